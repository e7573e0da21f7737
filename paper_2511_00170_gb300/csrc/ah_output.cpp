// FASTA output (Supplementary "Headers and outputs"): one record per amplicon whose header carries
// the sequence id, source, coordinates, Tm, orientation, the matched primer sites and, when
// requested, the barcodes; the amplicon sequence follows on one line.  FASTQ output (the FASTQ
// support the paper lists as future work) adds a '+' line and the amplicon's qualities.  Host
// code: it formats what the device produced (ah_amplicons_copy, ah_amplicons_seq_copy,
// ah_amplicons_qual_copy) into a caller buffer.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ah_internal.h"

namespace {

const char* const kOrient[4] = {"FR", "RF", "FF", "RR"};

int digits(uint64_t v) {
  int n = 1;
  while (v >= 10) v /= 10, ++n;
  return n;
}

char* put_u64(char* o, uint64_t v) {
  const int n = digits(v);
  for (int i = n - 1; i >= 0; --i, v /= 10) o[i] = (char)('0' + v % 10);
  return o + n;
}

char* put_str(char* o, const char* s, size_t n) {
  memcpy(o, s, n);
  return o + n;
}

// the sequence id: the header line up to its first blank
size_t id_len(const char* name) {
  size_t n = 0;
  while (name[n] && name[n] != ' ' && name[n] != '\t') ++n;
  return n;
}

// the Tm field's text: two decimals, NA when undefined
int tm_text(double tm, char* buf) {
  if (std::isnan(tm)) {
    memcpy(buf, "NA", 2);
    return 2;
  }
  return snprintf(buf, 48, "%.2f", tm);
}

struct Fmt {
  const ah_amplicon* amps;
  const char *arena, *qarena;
  const uint64_t* field_off;
  const char* const* names;
  const char* const* sources;
  int barcodes;
};

uint64_t field_len(const uint64_t* f, int k) { return f[k + 1] - f[k]; }

// bytes of amplicon m's record; with out, the record written there
uint64_t record(const Fmt& F, uint64_t m, char* out) {
  const ah_amplicon& a = F.amps[m];
  const uint64_t* f = F.field_off + 5 * m;  // amplicon, fb, rb, site i, site j
  const char* name = F.names[a.record];
  const char* src = F.sources ? F.sources[a.record] : nullptr;
  char tmb[48];
  const int tl = tm_text(a.tm, tmb);
  const size_t il = id_len(name), sl = src ? strlen(src) : 0;
  // the forward primer's site and the reverse primer's: for RF the anchor i is the reverse one
  const int fs = a.orient == 1 ? 4 : 3, rs = a.orient == 1 ? 3 : 4;
  uint64_t n = 1 + il + (src ? 8 + sl : 0) + 13 + digits((uint64_t)a.start + 1) + 1 + digits(a.end) + 4 + tl + 13 + 2 +
               9 + field_len(f, fs) + 9 + field_len(f, rs) + (F.barcodes ? 4 + field_len(f, 1) + 4 + field_len(f, 2) : 0) +
               1 + field_len(f, 0) + 1 + (F.qarena ? 2 + field_len(f, 0) + 1 : 0);
  if (!out) return n;
  char* o = out;
  *o++ = F.qarena ? '@' : '>';
  o = put_str(o, name, il);
  if (src) o = put_str(put_str(o, ".source=", 8), src, sl);
  o = put_str(o, ".coordinates=", 13);
  o = put_u64(o, (uint64_t)a.start + 1);  // 1-based, inclusive
  *o++ = '-';
  o = put_u64(o, a.end);
  o = put_str(put_str(o, ".Tm=", 4), tmb, tl);
  o = put_str(put_str(o, ".orientation=", 13), kOrient[a.orient], 2);
  o = put_str(put_str(o, ".fprimer=", 9), F.arena + f[fs], field_len(f, fs));
  o = put_str(put_str(o, ".rprimer=", 9), F.arena + f[rs], field_len(f, rs));
  if (F.barcodes) {
    o = put_str(put_str(o, ".fb=", 4), F.arena + f[1], field_len(f, 1));
    o = put_str(put_str(o, ".rb=", 4), F.arena + f[2], field_len(f, 2));
  }
  *o++ = '\n';
  o = put_str(o, F.arena + f[0], field_len(f, 0));
  *o++ = '\n';
  if (F.qarena) {
    o = put_str(o, "+\n", 2);
    o = put_str(o, F.qarena + f[0], field_len(f, 0));
    *o++ = '\n';
  }
  return n;
}

// fn(begin, end) over [0, n) in chunks on up to hardware_concurrency threads
template <typename Fn>
void parallel_chunks(uint64_t n, Fn fn) {
  const uint64_t per = 1 << 14;
  const unsigned width = (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>(std::max(1u, std::thread::hardware_concurrency()), (n + per - 1) / per));
  if (width == 1) {
    fn(0, n);
    return;
  }
  std::atomic<uint64_t> next{0};
  std::vector<std::thread> pool;
  for (unsigned w = 0; w < width; ++w)
    pool.emplace_back([&] {
      for (uint64_t b = next.fetch_add(per); b < n; b = next.fetch_add(per)) fn(b, std::min(n, b + per));
    });
  for (auto& t : pool) t.join();
}

// FASTA (qarena NULL) or FASTQ records: lengths first (in parallel), then every record written at
// its offset (in parallel)
ah_status write_records(uint64_t n_amps, const ah_amplicon* amps, const char* arena, const char* qarena,
                        const uint64_t* field_off, uint32_t n_records, const char* const* record_names,
                        const char* const* record_sources, int barcodes, char* out, uint64_t out_cap,
                        uint64_t* out_len) {
  if (!out_len || (n_amps && (!amps || !arena || !field_off || !record_names))) return AH_EINVAL;
  for (uint64_t m = 0; m < n_amps; ++m)
    if (amps[m].record >= n_records || amps[m].orient > 3 || amps[m].end < amps[m].start) return AH_EINVAL;
  const Fmt F{amps, arena, qarena, field_off, record_names, record_sources, barcodes};
  std::vector<uint64_t> off(n_amps + 1, 0);
  parallel_chunks(n_amps, [&](uint64_t b, uint64_t e) {
    for (uint64_t m = b; m < e; ++m) off[m + 1] = record(F, m, nullptr);
  });
  for (uint64_t m = 0; m < n_amps; ++m) off[m + 1] += off[m];
  *out_len = off[n_amps];
  if (!out) return AH_OK;
  if (out_cap < off[n_amps]) return AH_EOVERFLOW;
  parallel_chunks(n_amps, [&](uint64_t b, uint64_t e) {
    for (uint64_t m = b; m < e; ++m) record(F, m, out + off[m]);
  });
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
