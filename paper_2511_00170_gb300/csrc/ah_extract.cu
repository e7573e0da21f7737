// Extraction stage (Supplementary, "Primer trimming and barcode extraction", "Headers and
// outputs"; "Amplicon calling and orientation": RF amplicons are reverse-complemented).
//
// Per amplicon five fields go into one byte arena: amplicon (or trimmed interior), forward barcode,
// reverse barcode, site i and site j in primer orientation.  A length pass and an exclusive scan
// place every amplicon; then one warp per amplicon decodes its fields from the 2-bit planes (lanes
// take consecutive output bytes, so stores are coalesced).
#include "ah_internal.h"

namespace ah {
namespace {

struct Fields {
  int64_t a[5], b[5];  // top-strand ranges [a, b) per field, clipped
  bool rc[5];          // write the range reverse-complemented
};

__device__ __forceinline__ int64_t clip(int64_t x, int64_t len) { return x < 0 ? 0 : (x > len ? len : x); }

__device__ Fields fields_of(const ah_amplicon& m, const ah_hit& hi, const ah_hit& hj, const uint8_t* plen,
                            int64_t len, int trim, int64_t fb, int64_t rb) {
  Fields f;
  const int64_t s_i = hi.pos, e_i = hi.pos + plen[hi.pattern], s_j = hj.pos, e_j = hj.pos + plen[hj.pattern];
  const bool rc = m.orient == 1;
  if (trim) {
    f.a[0] = e_i;
    f.b[0] = s_j < e_i ? e_i : s_j;
  } else {
    f.a[0] = s_i;
    f.b[0] = e_j;
  }
  f.rc[0] = rc;
  if (!rc) {
    f.a[1] = clip(s_i - fb, len), f.b[1] = clip(s_i, len);
    f.a[2] = clip(e_j, len), f.b[2] = clip(e_j + rb, len);
  } else {
    f.a[1] = clip(e_j, len), f.b[1] = clip(e_j + fb, len);
    f.a[2] = clip(s_i - rb, len), f.b[2] = clip(s_i, len);
  }
  f.rc[1] = f.rc[2] = rc;
  f.a[3] = s_i, f.b[3] = e_i, f.rc[3] = ((hi.pattern >> 1) & 1u) != 0;
  f.a[4] = s_j, f.b[4] = e_j, f.rc[4] = ((hj.pattern >> 1) & 1u) != 0;
  return f;
}

__global__ void k_extract_len(const ah_amplicon* __restrict__ amps, uint64_t n, const ah_hit* __restrict__ hits,
                              const uint32_t* __restrict__ rec_len, const uint8_t* __restrict__ plen, int trim,
                              int64_t fb, int64_t rb, uint64_t* __restrict__ total,
                              const uint64_t* __restrict__ d_n = nullptr) {
  const uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  if (d_n && m >= *d_n) {
    total[m] = 0;
    return;
  }
  const ah_amplicon A = amps[m];
  const Fields f = fields_of(A, hits[A.hit_i], hits[A.hit_j], plen, rec_len[A.record], trim, fb, rb);
  uint64_t t = 0;
  for (int q = 0; q < 5; ++q) t += (uint64_t)(f.b[q] - f.a[q]);
  total[m] = t;
}

__device__ __forceinline__ char decode(const uint2* planes, const uint32_t* invalid, uint64_t g0, int64_t x, bool comp) {
  const uint64_t g = g0 + ((uint64_t)x >> 5);
  const uint32_t bit = (uint32_t)(x & 31);
  if ((invalid[g] >> bit) & 1u) return 'N';
  const uint2 w = planes[g];
  uint32_t code = ((w.x >> bit) & 1u) | (((w.y >> bit) & 1u) << 1);
  if (comp) code ^= 2u;
  return "ACTG"[code];
}

__global__ void k_extract_write(const ah_amplicon* __restrict__ amps, uint64_t n, const ah_hit* __restrict__ hits,
                                const uint2* __restrict__ planes, const uint32_t* __restrict__ invalid,
                                const uint64_t* __restrict__ rec_group, const uint32_t* __restrict__ rec_len,
                                const uint8_t* __restrict__ plen, int trim, int64_t fb, int64_t rb,
                                const uint64_t* __restrict__ base, char* __restrict__ arena,
                                uint64_t* __restrict__ field_off, const uint64_t* __restrict__ d_n = nullptr,
                                uint64_t arena_cap = ~0ull, uint32_t* __restrict__ overflow = nullptr) {
  const int lane = threadIdx.x & 31;
  const uint64_t m = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (d_n) {
    const uint64_t live = min(*d_n, n);
    if (m == 0 && lane == 0 && live == 0) field_off[0] = 0;
    n = live;
  }
  if (m >= n) return;
  const ah_amplicon A = amps[m];
  const Fields f = fields_of(A, hits[A.hit_i], hits[A.hit_j], plen, rec_len[A.record], trim, fb, rb);
  const uint64_t g0 = rec_group[A.record];
  uint64_t w = base[m];
  if (base[m + 1] > arena_cap) {  // base[m + 1] is the end of this amplicon's fields
    if (lane == 0 && overflow) atomicOr(overflow, 8u);
    if (m == n - 1 && lane == 0) field_off[5 * n] = base[m + 1];
    return;
  }
  for (int q = 0; q < 5; ++q) {
    if (lane == 0) field_off[5 * m + q] = w;
    const int64_t len = f.b[q] - f.a[q];
    for (int64_t i = lane; i < len; i += 32) {
      // reverse complement: output i takes top-strand base b-1-i, complemented
      arena[w + i] = f.rc[q] ? decode(planes, invalid, g0, f.b[q] - 1 - i, true) : decode(planes, invalid, g0, f.a[q] + i, false);
    }
    w += (uint64_t)len;
  }
  if (m == n - 1 && lane == 0) field_off[5 * n] = w;
}

// qualities of field 0 (the amplicon or its trimmed interior) at the field's arena offset, reversed
// for RF like the bases (qualities are not complemented); one warp per amplicon
__global__ void k_extract_qual(const ah_amplicon* __restrict__ amps, uint64_t n, const ah_hit* __restrict__ hits,
                               const uint32_t* __restrict__ rec_len, const uint8_t* __restrict__ plen, int trim,
                               const uint8_t* __restrict__ qual, const uint64_t* __restrict__ qoff,
                               const uint64_t* __restrict__ field_off, char* __restrict__ qarena) {
  const int lane = threadIdx.x & 31;
  const uint64_t m = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= n) return;
  const ah_amplicon A = amps[m];
  const Fields f = fields_of(A, hits[A.hit_i], hits[A.hit_j], plen, rec_len[A.record], trim, 0, 0);
  const uint8_t* q = qual + qoff[A.record];
  const uint64_t w = field_off[5 * m];
  const int64_t len = f.b[0] - f.a[0];
  for (int64_t i = lane; i < len; i += 32) qarena[w + i] = (char)(f.rc[0] ? q[f.b[0] - 1 - i] : q[f.a[0] + i]);
}

}  // namespace

void launch_extract(cudaStream_t s, bool write, const ah_amplicon* amps, uint64_t cap, const uint64_t* d_n,
                    const ah_hit* hits, const uint2* planes, const uint32_t* invalid, const uint64_t* rec_group,
                    const uint32_t* rec_len, const uint8_t* plen, int trim, uint32_t fb, uint32_t rb, uint64_t* len_or_base,
                    char* arena, uint64_t* field_off, uint64_t arena_cap, uint32_t* overflow) {
  if (!write)
    k_extract_len<<<(unsigned)std::max<uint64_t>(1, (cap + 255) / 256), 256, 0, s>>>(amps, cap, hits, rec_len, plen, trim,
                                                                                    (int64_t)fb, (int64_t)rb,
                                                                                    len_or_base, d_n);
  else
    k_extract_write<<<(unsigned)std::max<uint64_t>(1, (cap + 7) / 8), 256, 0, s>>>(
        amps, cap, hits, planes, invalid, rec_group, rec_len, plen, trim, (int64_t)fb, (int64_t)rb, len_or_base, arena,
        field_off, d_n, arena_cap, overflow);
}

ah_status extract(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, ah_amplicons* a, int trim,
                  uint32_t fb, uint32_t rb) {
  ah_status st;
  dfree(ctx, a->d_arena);
  dfree(ctx, a->d_field_off);
  a->d_arena = nullptr;
  a->d_field_off = nullptr;
  a->arena_bytes = 0;
  const uint64_t n = a->n;
  uint64_t *tot = nullptr, *base = nullptr;
  if ((st = dalloc(ctx, &tot, n)) || (st = dalloc(ctx, &base, n + 1))) return st;
  if (n)
    k_extract_len<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(a->d, n, h->d, b->rec_len, p->d_plen, trim,
                                                                       (int64_t)fb, (int64_t)rb, tot);
  if (n) launched(ctx);
  if ((st = exclusive_scan_u64(ctx, tot, base, n))) return st;
  uint64_t bytes = 0;
  if ((st = read_u64(ctx, base + n, &bytes))) return st;
  if ((st = dalloc(ctx, &a->d_arena, bytes)) || (st = dalloc(ctx, &a->d_field_off, 5 * n + 1))) return st;
  if (n) {
    k_extract_write<<<(unsigned)((n + 7) / 8), 256, 0, ctx->stream>>>(a->d, n, h->d, b->planes, b->invalid, b->rec_group,
                                                                     b->rec_len, p->d_plen, trim, (int64_t)fb,
                                                                     (int64_t)rb, base, a->d_arena, a->d_field_off);
    launched(ctx);
  } else {
    AH_CUDA(ctx, cudaMemsetAsync(a->d_field_off, 0, sizeof(uint64_t), ctx->stream));
  }
  AH_CUDA(ctx, cudaGetLastError());
  a->arena_bytes = bytes;
  a->trim = trim;
  dfree(ctx, a->d_qarena);
  a->d_qarena = nullptr;
  dfree(ctx, tot);
  dfree(ctx, base);
  return AH_OK;
}

}  // namespace ah

using namespace ah;

extern "C" {

ah_status ah_extract_qualities(ah_ctx* ctx, const ah_quals* q, const ah_batch* b, const ah_primers* p,
                               const ah_hits* h, ah_amplicons* a) {
  if (!ctx || !q || !b || !p || !h || !a) return fail(ctx, AH_EINVAL, "ah_extract_qualities: NULL argument");
  if (!a->d_field_off) return fail(ctx, AH_EINVAL, "ah_extract_qualities: run ah_extract_barcodes first");
  bool same = q->n_records == b->n_records;
  for (uint32_t r = 0; same && r < b->n_records; ++r) same = q->h_off[r + 1] - q->h_off[r] == b->h_rec_len[r];
  if (!same) return fail(ctx, AH_EINVAL, "ah_extract_qualities: the qualities do not belong to this batch");
  cudaSetDevice(ctx->device);
  dfree(ctx, a->d_qarena);
  a->d_qarena = nullptr;
  ah_status st = dalloc(ctx, &a->d_qarena, a->arena_bytes + 1);
  if (st) return st;
  if (a->n) {
    k_extract_qual<<<(unsigned)((a->n + 7) / 8), 256, 0, ctx->stream>>>(a->d, a->n, h->d, b->rec_len, p->d_plen, a->trim,
                                                                        q->d_qual, q->d_off, a->d_field_off, a->d_qarena);
    launched(ctx);
  }
  AH_CUDA(ctx, cudaGetLastError());
  return AH_OK;
}

ah_status ah_amplicons_qual_copy(const ah_amplicons* a, char* out, uint64_t cap) {
  if (!a) return AH_EINVAL;
  if (!a->d_qarena) return fail(a->ctx, AH_EINVAL, "ah_amplicons_qual_copy: no qualities extracted");
  if (cap < a->arena_bytes) return fail(a->ctx, AH_EOVERFLOW, "ah_amplicons_qual_copy: need %llu bytes",
                                        (unsigned long long)a->arena_bytes);
  return copy_to_host(a->ctx, out, a->d_qarena, a->arena_bytes);
}

}  // extern "C"
