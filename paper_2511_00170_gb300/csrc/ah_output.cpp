// FASTA output (Supplementary "Headers and outputs"): one record per amplicon whose header carries
// the sequence id, source, coordinates, Tm, orientation, the matched primer sites and, when
// requested, the barcodes; the amplicon sequence follows on one line.  FASTQ output (the FASTQ
// support the paper lists as future work) adds a '+' line and the amplicon's qualities.  Host
// code: it formats what the device produced (ah_amplicons_copy, ah_amplicons_seq_copy,
// ah_amplicons_qual_copy) into a caller buffer.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "ah_internal.h"

namespace {

const char* const kOrient[4] = {"FR", "RF", "FF", "RR"};

void put_u64(std::string& s, uint64_t v) {
  char buf[24];
  int n = 0;
  do {
    buf[n++] = (char)('0' + v % 10);
    v /= 10;
  } while (v);
  while (n) s.push_back(buf[--n]);
}

// the sequence id: the header line up to its first blank
void put_id(std::string& s, const char* name) {
  for (const char* c = name; *c && *c != ' ' && *c != '\t'; ++c) s.push_back(*c);
}

void put_field(std::string& s, const char* arena, const uint64_t* off, uint64_t f) {
  s.append(arena + off[f], arena + off[f + 1]);
}

// FASTA (qarena NULL) or FASTQ records
ah_status write_records(uint64_t n_amps, const ah_amplicon* amps, const char* arena, const char* qarena,
                        const uint64_t* field_off, uint32_t n_records, const char* const* record_names,
                        const char* const* record_sources, int barcodes, char* out, uint64_t out_cap,
                        uint64_t* out_len) {
  if (!out_len || (n_amps && (!amps || !arena || !field_off || !record_names))) return AH_EINVAL;
  std::string s;
  s.reserve(n_amps * 128);
  for (uint64_t m = 0; m < n_amps; ++m) {
    const ah_amplicon& a = amps[m];
    if (a.record >= n_records || a.orient > 3 || a.end < a.start) return AH_EINVAL;
    const uint64_t* f = field_off + 5 * m;  // amplicon, fb, rb, site i, site j
    s.push_back(qarena ? '@' : '>');
    put_id(s, record_names[a.record]);
    if (record_sources && record_sources[a.record]) {
      s += ".source=";
      s += record_sources[a.record];
    }
    s += ".coordinates=";
    put_u64(s, (uint64_t)a.start + 1);  // 1-based, inclusive
    s.push_back('-');
    put_u64(s, a.end);
    s += ".Tm=";
    if (std::isnan(a.tm)) {
      s += "NA";
    } else {
      char buf[48];
      snprintf(buf, sizeof buf, "%.2f", a.tm);
      s += buf;
    }
    s += ".orientation=";
    s += kOrient[a.orient];
    // the forward primer's site and the reverse primer's: for RF the anchor i is the reverse one
    const uint64_t fs = a.orient == 1 ? 4 : 3, rs = a.orient == 1 ? 3 : 4;
    s += ".fprimer=";
    put_field(s, arena, f, fs);
    s += ".rprimer=";
    put_field(s, arena, f, rs);
    if (barcodes) {
      s += ".fb=";
      put_field(s, arena, f, 1);
      s += ".rb=";
      put_field(s, arena, f, 2);
    }
    s.push_back('\n');
    put_field(s, arena, f, 0);
    s.push_back('\n');
    if (qarena) {
      s += "+\n";
      put_field(s, qarena, f, 0);
      s.push_back('\n');
    }
  }
  *out_len = s.size();
  if (!out) return AH_OK;
  if (out_cap < s.size()) return AH_EOVERFLOW;
  memcpy(out, s.data(), s.size());
  return AH_OK;
}

}  // namespace

extern "C" {

ah_status ah_amplicons_fasta(uint64_t n_amps, const ah_amplicon* amps, const char* arena, const uint64_t* field_off,
                             uint32_t n_records, const char* const* record_names, const char* const* record_sources,
                             int barcodes, char* out, uint64_t out_cap, uint64_t* out_len) {
  return write_records(n_amps, amps, arena, nullptr, field_off, n_records, record_names, record_sources, barcodes, out,
                       out_cap, out_len);
}

ah_status ah_amplicons_fastq(uint64_t n_amps, const ah_amplicon* amps, const char* arena, const char* qual_arena,
                             const uint64_t* field_off, uint32_t n_records, const char* const* record_names,
                             const char* const* record_sources, int barcodes, char* out, uint64_t out_cap,
                             uint64_t* out_len) {
  if (n_amps && !qual_arena) return AH_EINVAL;
  return write_records(n_amps, amps, arena, qual_arena ? qual_arena : "", field_off, n_records, record_names,
                       record_sources, barcodes, out, out_cap, out_len);
}

}  // extern "C"
