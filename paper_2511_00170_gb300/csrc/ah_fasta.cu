// FASTA input on the device (Abstract and Section "Implementations": the pipeline packs FASTA into
// 2-bit batches).  Raw FASTA text, a '>' header line per record followed by sequence lines, is
// parsed where it lies in HBM: a line-state pass per 4 KiB tile, the tiles' entry states chained on
// the host, then a counting pass and an emitting pass that compact the sequence bytes (line breaks
// and blanks dropped) and record every header.  The compacted sequences are packed like any other
// device source.
//
// Line state: LS at the start of a line, H inside a header line, S inside a sequence line.  A line
// whose first byte is '>' is a header and starts a record; '\n' ends a line; '\r', ' ' and '\t' in a
// sequence line are not bases.  Bytes before the first header belong to no record.
#include <algorithm>
#include <cstring>

#include "ah_internal.h"

struct ah_fasta {
  std::vector<std::string> names;  // header lines without '>' (or '@') and trailing '\r'
};

namespace ah {
namespace {

constexpr int kFaThreads = 256, kFaBytes = 16, kFaSegs = 4, kFaTile = kFaThreads * kFaBytes * kFaSegs;
// a thread takes kFaSegs consecutive 16-byte segments (64 bytes); a tile (one CTA) 16 KiB
enum : uint32_t { FS_LS = 0, FS_H = 1, FS_S = 2 };
// a transfer function over the three states: bits 2s..2s+1 hold the state after, from state s
constexpr uint32_t kIdentity = FS_LS | (FS_H << 2) | (FS_S << 4);

__device__ __forceinline__ uint32_t apply(uint32_t f, uint32_t s) { return (f >> (2 * s)) & 3u; }
// first a, then b
__device__ __forceinline__ uint32_t compose(uint32_t a, uint32_t b) {
  return apply(b, apply(a, FS_LS)) | (apply(b, apply(a, FS_H)) << 2) | (apply(b, apply(a, FS_S)) << 4);
}
__device__ __forceinline__ uint32_t step(uint32_t s, uint8_t c) {
  if (c == '\n') return FS_LS;
  if (s == FS_LS) return c == '>' ? FS_H : FS_S;
  return s;
}
__device__ __forceinline__ bool is_blank(uint8_t c) { return c == '\r' || c == ' ' || c == '\t'; }

// segment q of this thread: bytes [p0, p1)
__device__ __forceinline__ void seg_span(uint64_t n, int q, uint64_t* p0, uint64_t* p1) {
  *p0 = (uint64_t)blockIdx.x * kFaTile + ((uint64_t)threadIdx.x * kFaSegs + q) * kFaBytes;
  *p1 = min(n, *p0 + kFaBytes);
  if (*p0 > n) *p0 = n;
}

// A thread's segment: up to 16 bytes and per-byte class masks (bit j for byte j).
struct Seg {
  uint32_t w0, w1, w2, w3;  // the bytes, little-endian (registers: no indexed array)
  int len;
  uint32_t nl, gt, blank;
  __device__ __forceinline__ uint8_t at(int j) const {
    const uint32_t w = j < 8 ? (j < 4 ? w0 : w1) : (j < 12 ? w2 : w3);
    return (uint8_t)(w >> (8 * (j & 3)));
  }
};

// bits 7, 15, 23, 31 of m to bits 0-3 (the four partial products land on distinct bits below 28)
__device__ __forceinline__ uint32_t bit7_mask(uint32_t m) { return ((m & 0x80808080u) * 0x00204081u) >> 28; }

// bit j: byte j of w equals the byte in ch4 (exact per byte: no borrow crosses bytes)
__device__ __forceinline__ uint32_t bytes_eq(uint32_t w, uint32_t ch4) {
  const uint32_t y = w ^ ch4;
  return bit7_mask(~(((y & 0x7f7f7f7fu) + 0x7f7f7f7fu) | y));
}

__device__ __forceinline__ void classify_seg(const uint32_t* w, int len, Seg* g) {
  g->len = len;
  g->nl = g->gt = g->blank = 0;
  g->w0 = w[0], g->w1 = w[1], g->w2 = w[2], g->w3 = w[3];
  // bases and other letters have bit 7 clear and bit 6 set; line breaks, '>' and blanks do not,
  // so most segments skip the exact classification
  uint32_t other = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) other |= ~(~w[q] & (w[q] << 1)) & 0x80808080u;
  if (other == 0 && len == kFaBytes) return;
  // line breaks exactly; '>' and blanks only when some other non-letter byte is present
  uint32_t other16 = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    other16 |= bit7_mask(~(~w[q] & (w[q] << 1))) << (4 * q);
    g->nl |= bytes_eq(w[q], 0x0a0a0a0au) << (4 * q);
  }
  if (other16 != g->nl || len != kFaBytes) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      g->gt |= bytes_eq(w[q], 0x3e3e3e3eu) << (4 * q);
      g->blank |= (bytes_eq(w[q], 0x0d0d0d0du) | bytes_eq(w[q], 0x20202020u) | bytes_eq(w[q], 0x09090909u)) << (4 * q);
    }
  }
  const uint32_t valid = len >= 32 ? 0xffffffffu : ((1u << len) - 1u);
  g->nl &= valid, g->gt &= valid, g->blank &= valid;
}

// the thread's kFaSegs segments: whole and 16-byte aligned, four vector loads issued together;
// otherwise byte loads up to the end of the text
__device__ __forceinline__ void load_segs(const uint8_t* __restrict__ t, uint64_t n, Seg* g) {
  const uint64_t p = (uint64_t)blockIdx.x * kFaTile + (uint64_t)threadIdx.x * (kFaSegs * kFaBytes);
  uint32_t w[kFaSegs][4];
  if (p + kFaSegs * kFaBytes <= n && (((uint64_t)(uintptr_t)t) & 15) == 0) {
    const uint4* v = reinterpret_cast<const uint4*>(t + p);
    uint4 x[kFaSegs];
#pragma unroll
    for (int q = 0; q < kFaSegs; ++q) x[q] = __ldg(v + q);
#pragma unroll
    for (int q = 0; q < kFaSegs; ++q) {
      w[q][0] = x[q].x, w[q][1] = x[q].y, w[q][2] = x[q].z, w[q][3] = x[q].w;
      classify_seg(w[q], kFaBytes, &g[q]);
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) {
    const uint64_t p0 = min(n, p + (uint64_t)q * kFaBytes), p1 = min(n, p0 + kFaBytes);
    const int len = (int)(p1 - p0);
    w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0;
#pragma unroll
    for (int j = 0; j < kFaBytes; ++j)
      if (j < len) w[q][j >> 2] |= (uint32_t)t[p0 + j] << (8 * (j & 3));
    classify_seg(w[q], len, &g[q]);
  }
}

// the segment's transfer function
__device__ __forceinline__ uint32_t seg_function(const Seg& g) {
  if (g.len == 0) return kIdentity;
  if (g.nl) {
    const int last = 31 - __clz(g.nl);
    const uint32_t e = last == g.len - 1 ? FS_LS : (g.at(last + 1) == '>' ? FS_H : FS_S);
    return e | (e << 2) | (e << 4);
  }
  return (g.at(0) == '>' ? FS_H : FS_S) | (FS_H << 2) | (FS_S << 4);
}

// the segment needs the byte walk: a header starts in it or it starts inside a header line
__device__ __forceinline__ bool seg_has_header(const Seg& g, uint32_t s0) {
  const uint32_t line_start = (g.nl << 1) | (s0 == FS_LS ? 1u : 0u);
  return s0 == FS_H || (g.gt & line_start) != 0;
}

// exclusive composition of the block's thread functions (thread order) and the block's total
__device__ uint32_t block_exclusive_function(uint32_t f, uint32_t* total) {
  __shared__ uint32_t warp_f[kFaThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = f;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t other = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = compose(other, inc);
  }
  uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) exc = kIdentity;
  if (lane == 31) warp_f[warp] = inc;
  __syncthreads();
  uint32_t before = kIdentity;
  for (int w = 0; w < warp; ++w) before = compose(before, warp_f[w]);
  if (total) {
    uint32_t all = kIdentity;
    for (int w = 0; w < kFaThreads / 32; ++w) all = compose(all, warp_f[w]);
    *total = all;
  }
  __syncthreads();
  return compose(before, exc);
}

// exclusive sums of two per-thread counts over the block, and their totals
__device__ void block_exclusive_sums(uint32_t a, uint32_t b, uint32_t* ea, uint32_t* eb, uint32_t* ta, uint32_t* tb) {
  __shared__ uint32_t wa[kFaThreads / 32], wb[kFaThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t xa = __shfl_up_sync(0xffffffffu, ia, o), xb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) ia += xa, ib += xb;
  }
  if (lane == 31) wa[warp] = ia, wb[warp] = ib;
  __syncthreads();
  uint32_t ba = 0, bb = 0, sa = 0, sb = 0;
  for (int w = 0; w < kFaThreads / 32; ++w) {
    if (w < warp) ba += wa[w], bb += wb[w];
    sa += wa[w], sb += wb[w];
  }
  __syncthreads();
  *ea = ba + ia - a;
  *eb = bb + ib - b;
  *ta = sa;
  *tb = sb;
}

// pass 1: each tile's transfer function
__global__ void __launch_bounds__(kFaThreads) k_fa_tiles(const uint8_t* __restrict__ t, uint64_t n,
                                                         uint8_t* __restrict__ tile_f) {
  Seg g[kFaSegs];
  load_segs(t, n, g);
  uint32_t f = kIdentity;
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) f = compose(f, seg_function(g[q]));
  uint32_t total;
  block_exclusive_function(f, &total);
  if (threadIdx.x == 0) tile_f[blockIdx.x] = (uint8_t)total;
}

// passes 2 and 3: classify the tile's bytes from its entry state.  emit = false: per-tile counts of
// sequence bytes and headers.  emit = true: sequence bytes to out[rank], and per header (record r)
// hdr_pos[r] (first byte after '>'), seq_rank[r] (sequence bytes before it) and hdr_end[r] (its '\n').
// one segment from entry state s: counts (or, emitting, the bytes and header records); returns the
// state after it
template <bool emit>
__device__ __forceinline__ uint32_t seg_pass(const Seg& g, uint64_t p0, uint32_t s, uint32_t* n_seq, uint32_t* n_hdr,
                                             uint8_t* staged, uint32_t* local, uint64_t* rec, uint64_t seq_base0,
                                             uint64_t* __restrict__ hdr_pos, uint64_t* __restrict__ hdr_end,
                                             uint64_t* __restrict__ seq_rank) {
  if (!seg_has_header(g, s)) {  // no header: every byte that is not a line break or a blank
    const uint32_t valid = g.len >= 32 ? 0xffffffffu : ((1u << g.len) - 1u);
    const uint32_t seq_mask = ~(g.nl | g.blank) & valid;
    *n_seq += __popc(seq_mask);
    if (emit)
      for (uint32_t m = seq_mask; m; m &= m - 1) staged[(*local)++] = g.at(__ffs(m) - 1);
    return apply(seg_function(g), s);
  }
  for (int j = 0; j < g.len; ++j) {
    const uint8_t x = g.at(j);
    if (s == FS_LS && x == '>') {
      ++*n_hdr;
      if (emit) {
        hdr_pos[*rec] = p0 + j + 1;
        seq_rank[*rec] = seq_base0 + *local;
        ++*rec;
      }
    } else if (s == FS_H && x == '\n') {
      if (emit) hdr_end[*rec - 1] = p0 + j;  // a header line is open: *rec >= 1
    } else if ((s == FS_S || s == FS_LS) && x != '\n' && !is_blank(x)) {
      ++*n_seq;
      if (emit) staged[(*local)++] = x;
    }
    s = step(s, x);
  }
  return s;
}

template <bool emit>
__global__ void __launch_bounds__(kFaThreads) k_fa_pass(const uint8_t* __restrict__ t, uint64_t n,
                                                        const uint8_t* __restrict__ tile_entry,
                                                        uint32_t* __restrict__ tile_seq, uint32_t* __restrict__ tile_hdr,
                                                        const uint64_t* __restrict__ seq_base,
                                                        const uint64_t* __restrict__ hdr_base, uint8_t* __restrict__ out,
                                                        uint64_t* __restrict__ hdr_pos, uint64_t* __restrict__ hdr_end,
                                                        uint64_t* __restrict__ seq_rank, uint64_t pos_off, uint64_t seq_off,
                                                        uint64_t hdr_off) {
  // (a chunk of the text: positions, bases and records before it are pos_off, seq_off, hdr_off)
  __shared__ __align__(16) uint8_t staged[emit ? kFaTile + 32 : 16];  // the tile's sequence bytes, compacted
  Seg g[kFaSegs];
  load_segs(t, n, g);
  uint32_t f = kIdentity;
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) f = compose(f, seg_function(g[q]));
  const uint32_t before = block_exclusive_function(f, nullptr);
  const uint32_t s0 = apply(before, tile_entry[blockIdx.x]);
  uint32_t n_seq = 0, n_hdr = 0, s = s0;
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) {
    uint64_t p0, p1;
    seg_span(n, q, &p0, &p1);
    s = seg_pass<false>(g[q], p0, s, &n_seq, &n_hdr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr);
  }
  uint32_t e_seq, e_hdr, t_seq, t_hdr;
  block_exclusive_sums(n_seq, n_hdr, &e_seq, &e_hdr, &t_seq, &t_hdr);
  if (!emit) {
    if (threadIdx.x == 0) tile_seq[blockIdx.x] = t_seq, tile_hdr[blockIdx.x] = t_hdr;
    return;
  }
  const uint64_t base = seq_off + seq_base[blockIdx.x];
  const uint32_t lead = (uint32_t)(base & 15);  // staged[lead + i] goes to out[base + i]
  uint32_t local = lead + e_seq;                // this thread's first sequence byte, staged
  uint64_t rec = hdr_off + hdr_base[blockIdx.x] + e_hdr;  // headers started before this thread's bytes
  uint32_t cs = 0, ch = 0;
  s = s0;
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) {
    uint64_t p0, p1;
    seg_span(n, q, &p0, &p1);
    s = seg_pass<true>(g[q], pos_off + p0, s, &cs, &ch, staged, &local, &rec, base - lead, hdr_pos, hdr_end, seq_rank);
  }
  __syncthreads();
  // out[base, base + t_seq) from staged[lead, lead + t_seq): whole aligned 16-byte units as uint4,
  // the partial first and last units byte by byte (their other bytes belong to the next tiles)
  uint8_t* dst = out + (base - lead);
  const uint32_t end = lead + t_seq;
  const uint32_t full_lo = lead ? 16u : 0u, full_hi = end & ~15u;
  for (uint32_t u = full_lo + 16u * threadIdx.x; u < full_hi; u += 16u * kFaThreads)
    *reinterpret_cast<uint4*>(dst + u) = *reinterpret_cast<const uint4*>(staged + u);
  if (threadIdx.x < 32) {
    for (uint32_t i = lead + threadIdx.x; i < min(full_lo, end); i += 32) dst[i] = staged[i];
    for (uint32_t i = max(full_hi, full_lo) + threadIdx.x; i < end; i += 32) dst[i] = staged[i];
  }
}

// names of records [0, n_rec) into one buffer: name r is text[hdr_pos[r], hdr_pos[r] + len[r])
__global__ void k_fa_names(const uint8_t* __restrict__ t, const uint64_t* __restrict__ hdr_pos,
                           const uint64_t* __restrict__ name_off, uint32_t n_rec, uint8_t* __restrict__ names) {
  const uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= n_rec) return;
  const uint64_t len = name_off[r + 1] - name_off[r];
  for (uint64_t i = threadIdx.x & 31; i < len; i += 32) names[name_off[r] + i] = t[hdr_pos[r] + i];
}

// ------------------------------------------------------------------------------------------
// FASTQ (four lines per record: '@' header, bases, '+' line, qualities).  The line of a byte is the
// number of line breaks before it, so a tile needs only the line breaks before it (an exclusive
// sum) and no state machine; line 4r is record r's header, 4r + 1 its bases, 4r + 3 its qualities
// ('\r' dropped from all three).

// the thread's 64 bytes of tile `tile` as four segments with their line-break and '\r' masks
__device__ __forceinline__ void fq_load(const uint8_t* __restrict__ t, uint64_t n, uint64_t tile, Seg* g) {
  const uint64_t p = tile * kFaTile + (uint64_t)threadIdx.x * (kFaSegs * kFaBytes);
  const bool whole = p + kFaSegs * kFaBytes <= n && (((uint64_t)(uintptr_t)t) & 15) == 0;
  uint4 x[kFaSegs];
  if (whole) {
    const uint4* v = reinterpret_cast<const uint4*>(t + p);
#pragma unroll
    for (int q = 0; q < kFaSegs; ++q) x[q] = __ldg(v + q);
  }
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) {
    uint32_t w[4];
    int len = kFaBytes;
    if (whole) {
      w[0] = x[q].x, w[1] = x[q].y, w[2] = x[q].z, w[3] = x[q].w;
    } else {
      const uint64_t p0 = min(n, p + (uint64_t)q * kFaBytes), p1 = min(n, p0 + kFaBytes);
      len = (int)(p1 - p0);
      w[0] = w[1] = w[2] = w[3] = 0;
#pragma unroll
      for (int j = 0; j < kFaBytes; ++j)
        if (j < len) w[j >> 2] |= (uint32_t)t[p0 + j] << (8 * (j & 3));
    }
    Seg& s = g[q];
    s.len = len;
    s.w0 = w[0], s.w1 = w[1], s.w2 = w[2], s.w3 = w[3];
    s.nl = s.blank = s.gt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      s.nl |= bytes_eq(w[k], 0x0a0a0a0au) << (4 * k);
      s.blank |= bytes_eq(w[k], 0x0d0d0d0du) << (4 * k);
    }
    const uint32_t valid = len >= 32 ? 0xffffffffu : ((1u << len) - 1u);
    s.nl &= valid, s.blank &= valid;
  }
}

// pass 1: line breaks per tile, over tiles tile0 .. tile0 + gridDim.x - 1 of the text
__global__ void __launch_bounds__(kFaThreads) k_fq_lines(const uint8_t* __restrict__ t, uint64_t n, uint64_t tile0,
                                                         uint32_t* __restrict__ tile_nl) {
  const uint64_t tile = tile0 + blockIdx.x;
  Seg g[kFaSegs];
  fq_load(t, n, tile, g);
  uint32_t c = 0;
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) c += __popc(g[q].nl);
  uint32_t e0, e1, t0, t1;
  block_exclusive_sums(c, 0, &e0, &e1, &t0, &t1);
  if (threadIdx.x == 0) tile_nl[tile] = t0;
}

// passes 2 and 3 from each tile's line number: counts of bases, qualities and headers per tile, or
// (emit) the bases and qualities compacted and per record r: hdr_pos[r] (after '@'), hdr_end[r] (its
// line break), seq_rank[r] and qual_rank[r] (bases and qualities before the record).  Tiles tile0 ..
// tile0 + gridDim.x - 1 of the text; line_base, seq_base and qual_base count from the first of them,
// the lines, bases and qualities of the tiles before it are line_off, seq_off and qual_off.
template <bool emit>
__global__ void __launch_bounds__(kFaThreads) k_fq_pass(const uint8_t* __restrict__ t, uint64_t n, uint64_t tile0,
                                                        const uint64_t* __restrict__ line_base, uint64_t line_off,
                                                        uint64_t seq_off, uint64_t qual_off,
                                                        uint32_t* __restrict__ tile_seq, uint32_t* __restrict__ tile_qual,
                                                        uint32_t* __restrict__ tile_hdr, uint32_t* __restrict__ bad,
                                                        const uint64_t* __restrict__ seq_base,
                                                        const uint64_t* __restrict__ qual_base, uint8_t* __restrict__ seq_out,
                                                        uint8_t* __restrict__ qual_out, uint64_t* __restrict__ hdr_pos,
                                                        uint64_t* __restrict__ hdr_end, uint64_t* __restrict__ seq_rank,
                                                        uint64_t* __restrict__ qual_rank, uint64_t n_rec) {
  __shared__ __align__(16) uint8_t st_seq[emit ? kFaTile + 32 : 16], st_qual[emit ? kFaTile + 32 : 16];
  const uint64_t tile = tile0 + blockIdx.x;
  Seg g[kFaSegs];
  fq_load(t, n, tile, g);
  const uint64_t p = tile * kFaTile + (uint64_t)threadIdx.x * (kFaSegs * kFaBytes);
  uint32_t c = 0;
#pragma unroll
  for (int q = 0; q < kFaSegs; ++q) c += __popc(g[q].nl);
  uint32_t e_nl, e_x, t_nl, t_x;
  block_exclusive_sums(c, 0, &e_nl, &e_x, &t_nl, &t_x);
  const uint64_t line0 = line_off + line_base[tile] + e_nl;
  const bool start0 = p == 0 || (p < n && t[p - 1] == '\n');  // the thread's first byte starts a line
  // one walk over the runs between line breaks; emit = false counts, emit = true writes
  auto walk = [&](bool write, uint32_t* ns, uint32_t* nq, uint32_t* nh, uint32_t* nbad, uint32_t ls, uint32_t lq,
                  uint64_t sb, uint64_t qb) {
    uint64_t line = line0;
    bool at_start = start0;
    for (int q = 0; q < kFaSegs; ++q) {
      const Seg& s = g[q];
      const uint64_t p0 = p + (uint64_t)q * kFaBytes;
      uint32_t rest = s.nl;
      int a = 0;
      for (;;) {
        const int stop = rest ? __ffs(rest) - 1 : s.len;  // run [a, stop), then a line break at stop
        if (stop > a || (rest && stop == a)) {
          const uint32_t run = (stop >= 32 ? 0xffffffffu : ((1u << stop) - 1u)) & ~((1u << a) - 1u);
          const uint32_t kind = (uint32_t)(line & 3);
          if (kind == 1 || kind == 3) {
            const uint32_t m = run & ~s.blank;
            if (kind == 1) {
              *ns += __popc(m);
              if (write)
                for (uint32_t x = m; x; x &= x - 1) st_seq[ls++] = s.at(__ffs(x) - 1);
            } else {
              *nq += __popc(m);
              if (write)
                for (uint32_t x = m; x; x &= x - 1) st_qual[lq++] = s.at(__ffs(x) - 1);
            }
          } else if (kind == 0 && at_start && stop > a) {  // a non-empty header line starts here
            if (s.at(a) == '@') {
              ++*nh;
              if (write && (line >> 2) < n_rec) {  // records past n_rec are malformed text: caught on the host
                hdr_pos[line >> 2] = p0 + a + 1;
                seq_rank[line >> 2] = sb + ls;
                qual_rank[line >> 2] = qb + lq;
              }
            } else {
              ++*nbad;
            }
          }
          if (kind == 0 && rest && write && (line >> 2) < n_rec) hdr_end[line >> 2] = p0 + stop;
        }
        if (!rest) {
          if (stop > a) at_start = false;
          break;
        }
        rest &= rest - 1;
        a = stop + 1;
        ++line;
        at_start = true;
      }
    }
    return make_uint2(ls, lq);
  };
  uint32_t ns = 0, nq = 0, nh = 0, nb = 0;
  walk(false, &ns, &nq, &nh, &nb, 0, 0, 0, 0);
  uint32_t e_seq, e_qual, t_seq, t_qual;
  block_exclusive_sums(ns, nq, &e_seq, &e_qual, &t_seq, &t_qual);
  if (!emit) {
    uint32_t e_h, e_b, t_h, t_b;
    block_exclusive_sums(nh, nb, &e_h, &e_b, &t_h, &t_b);
    if (threadIdx.x == 0) {
      tile_seq[tile] = t_seq, tile_qual[tile] = t_qual, tile_hdr[tile] = t_h;
      if (t_b) atomicAdd(bad, t_b);
    }
    return;
  }
  const uint64_t sbase = seq_off + seq_base[tile], qbase = qual_off + qual_base[tile];
  const uint32_t slead = (uint32_t)(sbase & 15), qlead = (uint32_t)(qbase & 15);
  uint32_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
  walk(true, &d0, &d1, &d2, &d3, slead + e_seq, qlead + e_qual, sbase - slead, qbase - qlead);
  __syncthreads();
  // out[base, base + count) from staged[lead, lead + count) in aligned 16-byte units
  auto copy_out = [&](uint8_t* out, const uint8_t* st, uint64_t base, uint32_t lead, uint32_t cnt) {
    uint8_t* dst = out + (base - lead);
    const uint32_t end = lead + cnt, full_lo = lead ? 16u : 0u, full_hi = end & ~15u;
    for (uint32_t u = full_lo + 16u * threadIdx.x; u < full_hi; u += 16u * kFaThreads)
      *reinterpret_cast<uint4*>(dst + u) = *reinterpret_cast<const uint4*>(st + u);
    if (threadIdx.x < 32) {
      for (uint32_t i = lead + threadIdx.x; i < min(full_lo, end); i += 32) dst[i] = st[i];
      for (uint32_t i = max(full_hi, full_lo) + threadIdx.x; i < end; i += 32) dst[i] = st[i];
    }
  };
  copy_out(seq_out, st_seq, sbase, slead, t_seq);
  copy_out(qual_out, st_qual, qbase, qlead, t_qual);
}

// hdr_end[r] = the text's end before the emitting pass (a record whose header line ends the text)
__global__ void k_fill_u64(uint64_t* __restrict__ p, uint64_t n, uint64_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// every record has its header (its rank was written), fewer than 2^32 bases and as many qualities
// as bases; bad = 1 if not
__global__ void k_fq_check(const uint64_t* __restrict__ seq_rank, const uint64_t* __restrict__ qual_rank, uint64_t n,
                           uint64_t total_seq, uint64_t total_qual, uint32_t* bad) {
  const uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint64_t s0 = seq_rank[r], s1 = r + 1 < n ? seq_rank[r + 1] : total_seq;
  const uint64_t q0 = qual_rank[r], q1 = r + 1 < n ? qual_rank[r + 1] : total_qual;
  if (s0 == ~0ull || s1 < s0 || q1 < q0 || s1 - s0 != q1 - q0 || s1 - s0 > 0xffffffffull) atomicOr(bad, 1u);
}

// off[r] = rank[r] - rank[0] for r < n, off[n] = total - rank[0]
__global__ void k_rank_offsets(const uint64_t* __restrict__ rank, uint64_t n, uint64_t total, uint64_t* __restrict__ off) {
  const uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r <= n) off[r] = (r < n ? rank[r] : total) - rank[0];
}

uint32_t host_apply(uint32_t f, uint32_t s) { return (f >> (2 * s)) & 3u; }

}  // namespace
}  // namespace ah

using namespace ah;

namespace ah {
namespace {

// Parse and pack: into a new batch (*batch_out) or, with `into`, into an existing batch whose record
// lengths must equal the text's.
// hook (into mode only): after each chunk, the compacted record bases so far (the first record's first
// base at d_concat, `avail` of them, last = false), and once all are in and the records checked
// against the batch (last = true); it then packs them instead of the final pack
ah_status fasta_pack(ah_ctx* ctx, const char* text, uint64_t n_bytes, const uint32_t* genome_ids, ah_batch* into,
                     ah_batch** batch_out, ah_fasta** names_out, const FastaChunkHook* hook = nullptr) {
  cudaSetDevice(ctx->device);
  cudaPointerAttributes pa;
  const bool on_device = cudaPointerGetAttributes(&pa, text) == cudaSuccess &&
                         (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  ah_status st = AH_OK;
  const uint8_t* t = (const uint8_t*)text;
  uint8_t* staged = nullptr;
  const uint64_t n_tiles = (n_bytes + kFaTile - 1) / kFaTile;
  // host text is parsed in chunks as it lands: a copy stream moves chunk c + 1 while the passes run
  // on chunk c (each chunk's passes need only the entry state and totals of the chunks before it)
  const uint64_t chunk_tiles = on_device ? std::max<uint64_t>(1, n_tiles) : (kChunkBases / kFaTile);
  const uint64_t n_chunks = (n_tiles + chunk_tiles - 1) / chunk_tiles;
  uint8_t *tile_f = nullptr, *tile_entry = nullptr, *compact = nullptr, *h_f = nullptr, *h_entry = nullptr;
  uint32_t *tile_seq = nullptr, *tile_hdr = nullptr;
  uint64_t *seq_base = nullptr, *hdr_base = nullptr, *hdr_pos = nullptr, *hdr_end = nullptr, *seq_rank = nullptr;
  uint64_t hdr_cap = 0;
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> landed;
  uint64_t total_seq = 0, total_hdr = 0;
  uint64_t rank0 = ~0ull;  // the first record's first base in the compacted text (hook only)
  auto cleanup = [&] {
    if (cs) {
      cudaStreamSynchronize(cs);
      cudaStreamDestroy(cs);
    }
    for (cudaEvent_t e : landed) cudaEventDestroy(e);
    if (h_f) cudaFreeHost(h_f);
    if (h_entry) cudaFreeHost(h_entry);
    for (void* p : {(void*)staged, (void*)tile_f, (void*)tile_entry, (void*)compact, (void*)tile_seq,
                    (void*)tile_hdr, (void*)seq_base, (void*)hdr_base, (void*)hdr_pos, (void*)hdr_end, (void*)seq_rank})
      dfree(ctx, p);
  };
  // record arrays with room for `need` records, contents kept, a missing header end read as the end
  // of the text
  auto grow = [&](uint64_t need) -> ah_status {
    if (need <= hdr_cap) return AH_OK;
    const uint64_t cap = std::max<uint64_t>(need, std::max<uint64_t>(4096, 2 * hdr_cap));
    uint64_t *np = nullptr, *ne = nullptr, *nr = nullptr;
    ah_status e = AH_OK;
    if ((e = dalloc(ctx, &np, cap)) || (e = dalloc(ctx, &ne, cap)) || (e = dalloc(ctx, &nr, cap + 1))) {
      dfree(ctx, np), dfree(ctx, ne), dfree(ctx, nr);
      return e;
    }
    std::vector<uint64_t> fill(cap - hdr_cap, n_bytes);
    cudaMemcpyAsync(ne + hdr_cap, fill.data(), fill.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (hdr_cap) {
      cudaMemcpyAsync(np, hdr_pos, hdr_cap * 8, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(ne, hdr_end, hdr_cap * 8, cudaMemcpyDeviceToDevice, ctx->stream);
      cudaMemcpyAsync(nr, seq_rank, hdr_cap * 8, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    dfree(ctx, hdr_pos), dfree(ctx, hdr_end), dfree(ctx, seq_rank);
    hdr_pos = np, hdr_end = ne, seq_rank = nr, hdr_cap = cap;
    return cudaStreamSynchronize(ctx->stream) == cudaSuccess ? AH_OK : fail(ctx, AH_ECUDA, "ah_fasta_pack: grow");
  };
  do {
    if ((st = dalloc(ctx, &tile_f, n_tiles)) || (st = dalloc(ctx, &tile_entry, n_tiles)) ||
        (st = dalloc(ctx, &tile_seq, n_tiles)) || (st = dalloc(ctx, &tile_hdr, n_tiles)) ||
        (st = dalloc(ctx, &seq_base, n_tiles + 1)) || (st = dalloc(ctx, &hdr_base, n_tiles + 1)) ||
        (st = dalloc(ctx, &compact, n_bytes + 16)))
      break;
    if (cudaMallocHost(&h_f, chunk_tiles) != cudaSuccess || cudaMallocHost(&h_entry, chunk_tiles) != cudaSuccess) {
      st = fail(ctx, AH_ENOMEM, "ah_fasta_pack: page-locked buffers");
      break;
    }
    if (!on_device) {
      if ((st = dalloc(ctx, &staged, n_bytes + 16))) break;
      cudaEvent_t ready;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) {
        st = fail(ctx, AH_ECUDA, "ah_fasta_pack: copy stream");
        break;
      }
      landed.push_back(ready);  // the buffer was allocated in the context stream's order
      cudaEventRecord(ready, ctx->stream);
      cudaStreamWaitEvent(cs, ready, 0);
      for (uint64_t c = 0; c < n_chunks && !st; ++c) {
        const uint64_t b0 = c * chunk_tiles * kFaTile, b1 = std::min(n_bytes, b0 + chunk_tiles * kFaTile);
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
            cudaMemcpyAsync(staged + b0, text + b0, b1 - b0, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
            cudaEventRecord(e, cs) != cudaSuccess)
          st = fail(ctx, AH_ECUDA, "ah_fasta_pack: copy");
        landed.push_back(e);
      }
      if (st) break;
      t = staged;
    }
    uint32_t state = FS_LS;
    for (uint64_t c = 0; c < n_chunks && !st; ++c) {
      const uint64_t t0 = c * chunk_tiles, nt = std::min(chunk_tiles, n_tiles - t0);
      const uint64_t b0 = t0 * kFaTile, nb = std::min(n_bytes, b0 + nt * kFaTile) - b0;
      if (!on_device) cudaStreamWaitEvent(ctx->stream, landed[1 + c], 0);
      // pass 1 on the chunk; its tiles' entry states chained on the host
      k_fa_tiles<<<(unsigned)nt, kFaThreads, 0, ctx->stream>>>(t + b0, nb, tile_f + t0);
      launched(ctx);
      if (cudaMemcpyAsync(h_f, tile_f + t0, nt, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
          cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        st = fail(ctx, AH_ECUDA, "ah_fasta_pack: tile pass failed");
        break;
      }
      for (uint64_t i = 0; i < nt; ++i) h_entry[i] = (uint8_t)state, state = host_apply(h_f[i], state);
      if (cudaMemcpyAsync(tile_entry + t0, h_entry, nt, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
        st = fail(ctx, AH_ECUDA, "ah_fasta_pack: entry upload failed");
        break;
      }
      // pass 2: counts per tile, their sums within the chunk, the chunk's totals
      k_fa_pass<false><<<(unsigned)nt, kFaThreads, 0, ctx->stream>>>(t + b0, nb, tile_entry + t0, tile_seq + t0,
                                                                      tile_hdr + t0, nullptr, nullptr, nullptr, nullptr,
                                                                      nullptr, nullptr, 0, 0, 0);
      launched(ctx);
      uint64_t c_seq = 0, c_hdr = 0;
      if ((st = exclusive_scan_u32(ctx, tile_seq + t0, seq_base + t0, nt)) ||
          (st = exclusive_scan_u32(ctx, tile_hdr + t0, hdr_base + t0, nt)) ||
          (st = read_u64(ctx, seq_base + t0 + nt, &c_seq)) || (st = read_u64(ctx, hdr_base + t0 + nt, &c_hdr)))
        break;
      if (c_hdr && (st = grow(total_hdr + c_hdr))) break;
      // pass 3: the chunk's bases and headers at their places in the whole text
      k_fa_pass<true><<<(unsigned)nt, kFaThreads, 0, ctx->stream>>>(t + b0, nb, tile_entry + t0, nullptr, nullptr,
                                                                     seq_base + t0, hdr_base + t0, compact, hdr_pos,
                                                                     hdr_end, seq_rank, b0, total_seq, total_hdr);
      launched(ctx);
      total_seq += c_seq;
      total_hdr += c_hdr;
      if (hook && total_hdr) {
        if (rank0 == ~0ull && (st = read_u64(ctx, seq_rank, &rank0))) break;
        if ((st = (*hook)(compact + rank0, total_seq - rank0, false))) break;
      }
    }
    if (st) break;
    if (total_hdr == 0) {
      st = fail(ctx, AH_EINVAL, "ah_fasta_pack: no record (no line starts with '>')");
      break;
    }
    if (total_hdr > 0xffffffffull) {
      st = fail(ctx, AH_EINVAL, "ah_fasta_pack: more than 2^32 - 1 records");
      break;
    }
    std::vector<uint64_t> h_pos(total_hdr), h_end(total_hdr), h_rank(total_hdr + 1);
    AH_CUDA(ctx, cudaMemcpyAsync(h_pos.data(), hdr_pos, total_hdr * 8, cudaMemcpyDeviceToHost, ctx->stream));
    AH_CUDA(ctx, cudaMemcpyAsync(h_end.data(), hdr_end, total_hdr * 8, cudaMemcpyDeviceToHost, ctx->stream));
    AH_CUDA(ctx, cudaMemcpyAsync(h_rank.data(), seq_rank, total_hdr * 8, cudaMemcpyDeviceToHost, ctx->stream));
    AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    h_rank[total_hdr] = total_seq;
    const uint32_t n_rec = (uint32_t)total_hdr;
    // records: sequence offsets relative to the first record's first base
    std::vector<uint64_t> offs(n_rec + 1);
    for (uint32_t r = 0; r <= n_rec; ++r) offs[r] = h_rank[r] - h_rank[0];
    if (into) {
      bool same = into->n_records == n_rec;
      for (uint32_t r = 0; same && r < n_rec; ++r) same = into->h_rec_len[r] == offs[r + 1] - offs[r];
      if (!same) {
        st = fail(ctx, AH_EINVAL, "ah_fasta_pack_into: the text's records differ from the batch's in number or length");
        break;
      }
      st = hook ? (*hook)(compact + h_rank[0], offs[n_rec], true)
                : ah_batch_pack_range(ctx, into, 0, n_rec, compact + h_rank[0], offs.data());
    } else {
      st = ah_pack_batch_device(ctx, n_rec, compact + h_rank[0], offs.data(), genome_ids, batch_out);
    }
    if (st) break;
    if (names_out) {
      ah_fasta* f = new ah_fasta();
      f->names.resize(n_rec);
      std::vector<uint64_t> name_off(n_rec + 1, 0);
      for (uint32_t r = 0; r < n_rec; ++r) name_off[r + 1] = name_off[r] + (h_end[r] - h_pos[r]);
      std::vector<char> all(name_off[n_rec] + 1);
      if (on_device) {
        uint64_t* d_off = nullptr;
        uint8_t* d_names = nullptr;
        st = dalloc(ctx, &d_off, n_rec + 1);
        if (!st) st = dalloc(ctx, &d_names, name_off[n_rec] + 1);
        if (!st) {
          cudaMemcpyAsync(d_off, name_off.data(), (n_rec + 1) * 8, cudaMemcpyHostToDevice, ctx->stream);
          k_fa_names<<<(n_rec + 7) / 8, 256, 0, ctx->stream>>>(t, hdr_pos, d_off, n_rec, d_names);
          launched(ctx);
          cudaMemcpyAsync(all.data(), d_names, name_off[n_rec], cudaMemcpyDeviceToHost, ctx->stream);
          if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(ctx, AH_ECUDA, "ah_fasta_pack: names");
        }
        dfree(ctx, d_off);
        dfree(ctx, d_names);
      } else {
        for (uint32_t r = 0; r < n_rec; ++r) memcpy(all.data() + name_off[r], text + h_pos[r], h_end[r] - h_pos[r]);
      }
      for (uint32_t r = 0; r < n_rec && !st; ++r) {
        std::string nm(all.data() + name_off[r], name_off[r + 1] - name_off[r]);
        while (!nm.empty() && nm.back() == '\r') nm.pop_back();
        f->names[r] = std::move(nm);
      }
      if (st) {
        delete f;
        if (!into) {
          ah_batch_free(*batch_out);
          *batch_out = nullptr;
        }
        break;
      }
      *names_out = f;
    }
  } while (false);
  cleanup();
  return st;
}

}  // namespace

ah_status fasta_pack_hooked(ah_ctx* ctx, const char* text, uint64_t n_bytes, ah_batch* into, const FastaChunkHook& hook) {
  return fasta_pack(ctx, text, n_bytes, nullptr, into, nullptr, nullptr, &hook);
}
}  // namespace ah

extern "C" {

ah_status ah_fasta_pack(ah_ctx* ctx, const char* text, uint64_t n_bytes, const uint32_t* genome_ids,
                        ah_batch** batch_out, ah_fasta** names_out) {
  if (!ctx || !text || !batch_out || n_bytes == 0) return fail(ctx, AH_EINVAL, "ah_fasta_pack: bad arguments");
  *batch_out = nullptr;
  if (names_out) *names_out = nullptr;
  return fasta_pack(ctx, text, n_bytes, genome_ids, nullptr, batch_out, names_out);
}

ah_status ah_fasta_pack_into(ah_ctx* ctx, const char* text, uint64_t n_bytes, ah_batch* batch, ah_fasta** names_out) {
  if (!ctx || !text || !batch || n_bytes == 0 || batch->view)
    return fail(ctx, AH_EINVAL, "ah_fasta_pack_into: bad arguments");
  if (names_out) *names_out = nullptr;
  return fasta_pack(ctx, text, n_bytes, nullptr, batch, nullptr, names_out);
}

ah_status ah_fastq_pack(ah_ctx* ctx, const char* text, uint64_t n_bytes, const uint32_t* genome_ids,
                        ah_batch** batch_out, ah_quals** quals_out, ah_fasta** names_out) {
  if (!ctx || !text || !batch_out || !quals_out || n_bytes == 0) return fail(ctx, AH_EINVAL, "ah_fastq_pack: bad arguments");
  *batch_out = nullptr;
  *quals_out = nullptr;
  if (names_out) *names_out = nullptr;
  cudaSetDevice(ctx->device);
  cudaPointerAttributes pa;
  const bool on_device = cudaPointerGetAttributes(&pa, text) == cudaSuccess &&
                         (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  ah_status st = AH_OK;
  const uint8_t* t = (const uint8_t*)text;
  uint8_t *staged = nullptr, *seq = nullptr, *qual = nullptr;
  const uint64_t n_tiles = (n_bytes + kFaTile - 1) / kFaTile;
  // host text is parsed in chunks as it lands, as FASTA is: a copy stream moves chunk c + 1 while the
  // passes run on chunk c, which need only the lines, bases and qualities of the chunks before it
  const uint64_t chunk_tiles = on_device ? std::max<uint64_t>(1, n_tiles) : (kChunkBases / kFaTile);
  const uint64_t n_chunks = (n_tiles + chunk_tiles - 1) / chunk_tiles;
  uint32_t *tile_nl = nullptr, *tile_seq = nullptr, *tile_qual = nullptr, *tile_hdr = nullptr, *bad = nullptr;
  uint64_t *line_base = nullptr, *seq_base = nullptr, *qual_base = nullptr, *hdr_base = nullptr;
  uint64_t *hdr_pos = nullptr, *hdr_end = nullptr, *seq_rank = nullptr, *qual_rank = nullptr;
  uint64_t rec_cap = 0;
  ah_quals* q = nullptr;
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> landed;
  auto cleanup = [&] {
    if (cs) {
      cudaStreamSynchronize(cs);
      cudaStreamDestroy(cs);
    }
    for (cudaEvent_t e : landed) cudaEventDestroy(e);
    for (void* x : {(void*)staged, (void*)seq, (void*)tile_nl, (void*)tile_seq, (void*)tile_qual, (void*)tile_hdr,
                    (void*)bad, (void*)line_base, (void*)seq_base, (void*)qual_base, (void*)hdr_base, (void*)hdr_pos,
                    (void*)hdr_end, (void*)seq_rank, (void*)qual_rank})
      dfree(ctx, x);
  };
  auto fill = [&](uint64_t* p, uint64_t n, uint64_t v) {
    k_fill_u64<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 4096), 256, 0, ctx->stream>>>(p, n, v);
    launched(ctx);
  };
  // record arrays with room for `need` records, contents kept; a new record's header end reads as
  // the end of the text and its rank as missing (~0) until its header is seen
  auto grow = [&](uint64_t need) -> ah_status {
    if (need <= rec_cap) return AH_OK;
    const uint64_t cap = std::max<uint64_t>(need, std::max<uint64_t>(4096, 2 * rec_cap));
    uint64_t* nw[4] = {nullptr, nullptr, nullptr, nullptr};
    uint64_t** old[4] = {&hdr_pos, &hdr_end, &seq_rank, &qual_rank};
    ah_status e = AH_OK;
    for (int k = 0; k < 4 && !e; ++k) e = dalloc(ctx, &nw[k], cap);
    if (e) {
      for (uint64_t* x : nw) dfree(ctx, x);
      return e;
    }
    for (int k = 0; k < 4; ++k) {
      if (rec_cap) cudaMemcpyAsync(nw[k], *old[k], rec_cap * 8, cudaMemcpyDeviceToDevice, ctx->stream);
      dfree(ctx, *old[k]);
      *old[k] = nw[k];
    }
    fill(hdr_end + rec_cap, cap - rec_cap, n_bytes);
    fill(seq_rank + rec_cap, cap - rec_cap, ~0ull);
    rec_cap = cap;
    return cudaGetLastError() == cudaSuccess ? AH_OK : fail(ctx, AH_ECUDA, "ah_fastq_pack: record arrays");
  };
  // bases and qualities compacted: room for `need` bytes (and the packer's 16 of slack), the first
  // `used` kept.  Valid FASTQ has as many qualities as bases, at most half the text each, which is
  // the first size; other text may need more before it is refused.
  uint64_t seq_cap = 0, qual_cap = 0;
  auto grow_bytes = [&](uint8_t** buf, uint64_t* cap, uint64_t used, uint64_t need) -> ah_status {
    if (need + 16 <= *cap) return AH_OK;
    const uint64_t nc = std::max(need + 16, std::min(n_bytes + 16, 2 * *cap));
    uint8_t* nb = nullptr;
    ah_status e = dalloc(ctx, &nb, nc);
    if (e) return e;
    if (used) cudaMemcpyAsync(nb, *buf, used, cudaMemcpyDeviceToDevice, ctx->stream);
    dfree(ctx, *buf);
    *buf = nb;
    *cap = nc;
    return AH_OK;
  };
  do {
    if ((st = dalloc(ctx, &tile_nl, n_tiles)) || (st = dalloc(ctx, &tile_seq, n_tiles)) ||
        (st = dalloc(ctx, &tile_qual, n_tiles)) || (st = dalloc(ctx, &tile_hdr, n_tiles)) || (st = dalloc(ctx, &bad, 1)) ||
        (st = dalloc(ctx, &line_base, n_tiles + 1)) || (st = dalloc(ctx, &seq_base, n_tiles + 1)) ||
        (st = dalloc(ctx, &qual_base, n_tiles + 1)) || (st = dalloc(ctx, &hdr_base, n_tiles + 1)) ||
        (st = grow_bytes(&seq, &seq_cap, 0, n_bytes / 2)) || (st = grow_bytes(&qual, &qual_cap, 0, n_bytes / 2)))
      break;
    if (cudaMemsetAsync(bad, 0, 4, ctx->stream) != cudaSuccess) {
      st = fail(ctx, AH_ECUDA, "ah_fastq_pack: memset failed");
      break;
    }
    if (!on_device) {
      if ((st = dalloc(ctx, &staged, n_bytes + 16))) break;
      cudaEvent_t ready;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) {
        st = fail(ctx, AH_ECUDA, "ah_fastq_pack: copy stream");
        break;
      }
      landed.push_back(ready);  // the buffer was allocated in the context stream's order
      cudaEventRecord(ready, ctx->stream);
      cudaStreamWaitEvent(cs, ready, 0);
      for (uint64_t c = 0; c < n_chunks && !st; ++c) {
        const uint64_t b0 = c * chunk_tiles * kFaTile, b1 = std::min(n_bytes, b0 + chunk_tiles * kFaTile);
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
            cudaMemcpyAsync(staged + b0, text + b0, b1 - b0, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
            cudaEventRecord(e, cs) != cudaSuccess)
          st = fail(ctx, AH_ECUDA, "ah_fastq_pack: copy");
        landed.push_back(e);
      }
      if (st) break;
      t = staged;
    }
    uint64_t total_lines = 0, total_seq = 0, total_qual = 0, n_rec = 0;
    for (uint64_t c = 0; c < n_chunks && !st; ++c) {
      const uint64_t t0 = c * chunk_tiles, nt = std::min(chunk_tiles, n_tiles - t0);
      if (!on_device) cudaStreamWaitEvent(ctx->stream, landed[1 + c], 0);
      k_fq_lines<<<(unsigned)nt, kFaThreads, 0, ctx->stream>>>(t, n_bytes, t0, tile_nl);
      launched(ctx);
      if ((st = exclusive_scan_u32(ctx, tile_nl + t0, line_base + t0, nt))) break;
      k_fq_pass<false><<<(unsigned)nt, kFaThreads, 0, ctx->stream>>>(
          t, n_bytes, t0, line_base, total_lines, 0, 0, tile_seq, tile_qual, tile_hdr, bad, nullptr, nullptr, nullptr,
          nullptr, nullptr, nullptr, nullptr, nullptr, 0);
      launched(ctx);
      uint64_t c_lines = 0, c_seq = 0, c_qual = 0, c_hdr = 0;
      if ((st = exclusive_scan_u32(ctx, tile_seq + t0, seq_base + t0, nt)) ||
          (st = exclusive_scan_u32(ctx, tile_qual + t0, qual_base + t0, nt)) ||
          (st = exclusive_scan_u32(ctx, tile_hdr + t0, hdr_base + t0, nt)) ||
          (st = read_u64(ctx, line_base + t0 + nt, &c_lines)) || (st = read_u64(ctx, seq_base + t0 + nt, &c_seq)) ||
          (st = read_u64(ctx, qual_base + t0 + nt, &c_qual)) || (st = read_u64(ctx, hdr_base + t0 + nt, &c_hdr)))
        break;
      if ((st = grow(n_rec + c_hdr)) || (st = grow_bytes(&seq, &seq_cap, total_seq, total_seq + c_seq)) ||
          (st = grow_bytes(&qual, &qual_cap, total_qual, total_qual + c_qual)))
        break;
      k_fq_pass<true><<<(unsigned)nt, kFaThreads, 0, ctx->stream>>>(
          t, n_bytes, t0, line_base, total_lines, total_seq, total_qual, nullptr, nullptr, nullptr, nullptr, seq_base,
          qual_base, seq, qual, hdr_pos, hdr_end, seq_rank, qual_rank, rec_cap);
      launched(ctx);
      total_lines += c_lines;
      total_seq += c_seq;
      total_qual += c_qual;
      n_rec += c_hdr;
    }
    if (st) break;
    uint32_t h_bad = 0;
    if (cudaMemcpy(&h_bad, bad, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = fail(ctx, AH_ECUDA, "ah_fastq_pack: status read failed");
      break;
    }
    if (n_rec == 0 || h_bad || n_rec > 0xffffffffull) {
      st = fail(ctx, AH_EINVAL, "ah_fastq_pack: not FASTQ (every record is four lines, the first starting with '@')");
      break;
    }
    // records checked on the device; the sequence ranks come back for the batch's host record
    // table (the quality offsets equal the sequence offsets once the lengths match), header
    // positions only for the names
    AH_CUDA(ctx, cudaMemsetAsync(bad, 0, 4, ctx->stream));
    k_fq_check<<<(unsigned)((n_rec + 255) / 256), 256, 0, ctx->stream>>>(seq_rank, qual_rank, n_rec, total_seq,
                                                                         total_qual, bad);
    launched(ctx);
    std::vector<uint64_t> h_pos(names_out ? n_rec : 0), h_end(names_out ? n_rec : 0), h_srank(n_rec + 1);
    if ((st = copy_to_host(ctx, h_srank.data(), seq_rank, n_rec * 8))) break;
    if (names_out && ((st = copy_to_host(ctx, h_pos.data(), hdr_pos, n_rec * 8)) ||
                      (st = copy_to_host(ctx, h_end.data(), hdr_end, n_rec * 8))))
      break;
    if (cudaMemcpy(&h_bad, bad, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = fail(ctx, AH_ECUDA, "ah_fastq_pack: status read failed");
      break;
    }
    h_srank[n_rec] = total_seq;
    const uint32_t R = (uint32_t)n_rec;
    if (h_bad) {
      st = fail(ctx, AH_EINVAL, "ah_fastq_pack: a record lacks its header line or its qualities differ in length from its bases");
      break;
    }
    if ((st = pack_batch_ranked(ctx, R, seq, seq_rank, h_srank.data(), genome_ids, batch_out))) break;
    q = new ah_quals();
    q->ctx = ctx;
    q->n_records = R;
    if ((st = dalloc(ctx, &q->d_off, R + 1))) break;
    k_rank_offsets<<<(unsigned)((R + 256) / 256), 256, 0, ctx->stream>>>(qual_rank, R, total_qual, q->d_off);
    launched(ctx);
    // the qualities into a buffer of their own size: none come before the first record (line 0 is its
    // header), and their offsets are the bases' (the lengths match)
    if ((st = dalloc(ctx, &q->d_qual, total_qual + 16))) break;
    AH_CUDA(ctx, cudaMemcpyAsync(q->d_qual, qual, total_qual, cudaMemcpyDeviceToDevice, ctx->stream));
    q->h_off.resize(R + 1);
    for (uint32_t r = 0; r <= R; ++r) q->h_off[r] = h_srank[r] - h_srank[0];
    if (names_out) {
      ah_fasta* f = new ah_fasta();
      f->names.resize(R);
      std::vector<uint64_t> name_off(R + 1, 0);
      for (uint32_t r = 0; r < R; ++r) name_off[r + 1] = name_off[r] + (h_end[r] - h_pos[r]);
      std::vector<char> all(name_off[R] + 1);
      if (on_device) {
        uint64_t* d_off = nullptr;
        uint8_t* d_names = nullptr;
        st = dalloc(ctx, &d_off, R + 1);
        if (!st) st = dalloc(ctx, &d_names, name_off[R] + 1);
        if (!st) {
          cudaMemcpyAsync(d_off, name_off.data(), (R + 1) * 8, cudaMemcpyHostToDevice, ctx->stream);
          k_fa_names<<<(R + 7) / 8, 256, 0, ctx->stream>>>(t, hdr_pos, d_off, R, d_names);
          launched(ctx);
          cudaMemcpyAsync(all.data(), d_names, name_off[R], cudaMemcpyDeviceToHost, ctx->stream);
          if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(ctx, AH_ECUDA, "ah_fastq_pack: names");
        }
        dfree(ctx, d_off);
        dfree(ctx, d_names);
      } else {
        for (uint32_t r = 0; r < R; ++r) memcpy(all.data() + name_off[r], text + h_pos[r], h_end[r] - h_pos[r]);
      }
      for (uint32_t r = 0; r < R; ++r) {
        std::string nm(all.data() + name_off[r], name_off[r + 1] - name_off[r]);
        while (!nm.empty() && nm.back() == '\r') nm.pop_back();
        f->names[r] = std::move(nm);
      }
      if (st) {
        delete f;
        break;
      }
      *names_out = f;
    }
  } while (false);
  if (!st && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(ctx, AH_ECUDA, "ah_fastq_pack: copies failed");
  if (qual) dfree(ctx, qual);
  cleanup();
  if (st) {
    if (*batch_out) ah_batch_free(*batch_out);
    *batch_out = nullptr;
    ah_quals_free(q);
    return st;
  }
  *quals_out = q;
  return AH_OK;
}

uint32_t ah_quals_count(const ah_quals* q) { return q ? q->n_records : 0; }

ah_status ah_quals_copy(const ah_quals* q, char* out, uint64_t cap, uint64_t* offsets_out) {
  if (!q || !offsets_out) return AH_EINVAL;
  memcpy(offsets_out, q->h_off.data(), q->h_off.size() * sizeof(uint64_t));
  if (!out) return AH_OK;
  if (cap < q->h_off.back()) return fail(q->ctx, AH_EOVERFLOW, "ah_quals_copy: need %llu bytes",
                                         (unsigned long long)q->h_off.back());
  return copy_to_host(q->ctx, out, q->d_qual, q->h_off.back());
}

void ah_quals_free(ah_quals* q) {
  if (!q) return;
  if (q->ctx) {
    dfree(q->ctx, q->d_qual);
    dfree(q->ctx, q->d_off);
  }
  delete q;
}

uint32_t ah_fasta_count(const ah_fasta* f) { return f ? (uint32_t)f->names.size() : 0; }

const char* ah_fasta_name(const ah_fasta* f, uint32_t i) {
  return f && i < f->names.size() ? f->names[i].c_str() : nullptr;
}

ah_status ah_fasta_names_copy(const ah_fasta* f, char* out, uint64_t cap, uint64_t* offsets_out) {
  if (!f || !offsets_out) return AH_EINVAL;
  uint64_t total = 0;
  offsets_out[0] = 0;
  for (size_t i = 0; i < f->names.size(); ++i) offsets_out[i + 1] = total += f->names[i].size();
  if (!out) return AH_OK;
  if (cap < total) return AH_EOVERFLOW;
  for (size_t i = 0; i < f->names.size(); ++i) memcpy(out + offsets_out[i], f->names[i].data(), f->names[i].size());
  return AH_OK;
}

void ah_fasta_free(ah_fasta* f) { delete f; }

}  // extern "C"
