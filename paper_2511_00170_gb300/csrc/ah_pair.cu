// Pairing stage (Supplementary, "Amplicon calling and orientation"): sites are already sorted by
// (pair, record, pos, orient), so every + site walks the following sites of its record and pair
// directly.  A count pass, an exclusive scan and an emit pass give a deterministic order
// (by anchor, then partner) without atomics.
#include <cmath>

#include "ah_internal.h"

namespace ah {
namespace {

__device__ __forceinline__ uint8_t orientation(uint32_t primer_i, uint32_t primer_j) {
  // (F,R) FR=0, (R,F) RF=1, (F,F) FF=2, (R,R) RR=3
  return (uint8_t)(primer_i == primer_j ? 2u + primer_i : primer_i);
}

template <bool kEmit>
__global__ void k_pair_walk(const ah_hit* __restrict__ hits, uint64_t n, const uint64_t* __restrict__ pair_off,
                            const uint8_t* __restrict__ plen, uint32_t min_len, uint32_t max_len, uint32_t mask,
                            uint32_t* __restrict__ counts, const uint64_t* __restrict__ out_off,
                            ah_amplicon* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ah_hit a = hits[i];
  const uint32_t oa = a.pattern & 3u;
  uint32_t cnt = 0;
  uint64_t w = kEmit ? out_off[i] : 0;
  if (oa < 2) {  // anchors are + strand sites
    const uint32_t pair = a.pattern >> 2;
    const uint64_t seg_end = pair_off[pair + 1];
    for (uint64_t j = i + 1; j < seg_end; ++j) {
      const ah_hit b = hits[j];
      if (b.record != a.record) break;
      const uint32_t ob = b.pattern & 3u;
      if (ob < 2) break;  // a same-sense site stops the walk
      const uint64_t end = (uint64_t)b.pos + plen[b.pattern];
      const uint64_t length = end - a.pos;
      if (length > max_len) break;
      if (length < min_len) continue;
      const uint8_t o = orientation(oa & 1u, ob & 1u);
      if (!((mask >> o) & 1u)) continue;
      if (kEmit) {
        ah_amplicon m;
        m.hit_i = (uint32_t)i;
        m.hit_j = (uint32_t)j;
        m.record = a.record;
        m.start = a.pos;
        m.end = (uint32_t)end;
        m.pair = (uint16_t)pair;
        m.orient = o;
        m.flags = 0;
        m.tm = __longlong_as_double(0x7ff8000000000000ll);
        out[w++] = m;
      } else {
        ++cnt;
      }
    }
  }
  if (!kEmit) counts[i] = cnt;
}

}  // namespace

ah_status pair_amplicons(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, uint32_t min_len,
                         uint32_t max_len, uint32_t orient_mask, ah_amplicons** out) {
  (void)b;
  *out = nullptr;
  ah_status st;
  const uint64_t n = h->n;
  uint32_t* counts = nullptr;
  uint64_t* off = nullptr;
  if ((st = dalloc(ctx, &counts, n)) || (st = dalloc(ctx, &off, n + 1))) return st;
  const unsigned blocks = (unsigned)std::max<uint64_t>(1, (n + 255) / 256);
  if (n) {
    k_pair_walk<false><<<blocks, 256, 0, ctx->stream>>>(h->d, n, h->d_pair_off, p->d_plen, min_len, max_len,
                                                        orient_mask, counts, nullptr, nullptr);
    launched(ctx);
  }
  if ((st = exclusive_scan_u32(ctx, counts, off, n))) return st;
  uint64_t total = 0;
  if ((st = read_u64(ctx, off + n, &total))) return st;
  if (total > 0xffffffffull) return fail(ctx, AH_EOVERFLOW, "pairing: more than 2^32 amplicons");
  ah_amplicons* a = new ah_amplicons();
  a->ctx = ctx;
  a->n = total;
  if ((st = dalloc(ctx, &a->d, total))) {
    ah_amplicons_free(a);
    return st;
  }
  if (n && total) {
    k_pair_walk<true><<<blocks, 256, 0, ctx->stream>>>(h->d, n, h->d_pair_off, p->d_plen, min_len, max_len,
                                                       orient_mask, nullptr, off, a->d);
    launched(ctx);
  }
  AH_CUDA(ctx, cudaGetLastError());
  dfree(ctx, counts);
  dfree(ctx, off);
  *out = a;
  return AH_OK;
}

}  // namespace ah
