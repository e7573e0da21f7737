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

// d_n (optional): live site count in device memory, n is then the capacity; out_cap and overflow
// (optional) bound the emitted records
template <bool kEmit>
__global__ void k_pair_walk(const ah_hit* __restrict__ hits, uint64_t n, const uint64_t* __restrict__ pair_off,
                            const uint8_t* __restrict__ plen, uint32_t min_len, uint32_t max_len, uint32_t mask,
                            uint32_t* __restrict__ counts, const uint64_t* __restrict__ out_off,
                            ah_amplicon* __restrict__ out, const uint64_t* __restrict__ d_n = nullptr,
                            uint64_t out_cap = ~0ull, uint32_t* __restrict__ overflow = nullptr) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t n_live = d_n ? min(*d_n, n) : n;
  const uint32_t lane = threadIdx.x & 31u;
  const bool live = i < n_live;
  ah_hit a{};
  if (live) a = hits[i];
  const uint32_t oa = a.pattern & 3u;
  bool walking = live && oa < 2;  // anchors are + strand sites
  const uint32_t pair = a.pattern >> 2;
  const uint64_t seg_end = walking ? min(pair_off[pair + 1], n_live) : 0;
  uint32_t cnt = 0;
  uint64_t w = kEmit && live ? out_off[i] : 0;
  // partner j of the anchor: false when the walk ends there
  auto partner = [&](uint64_t j, uint32_t b_record, uint32_t b_pos, uint32_t b_pattern) -> bool {
    if (b_record != a.record) return false;
    const uint32_t ob = b_pattern & 3u;
    if (ob < 2) return false;  // a same-sense site stops the walk
    const uint64_t end = (uint64_t)b_pos + plen[b_pattern];
    const uint64_t length = end - a.pos;
    if (length > max_len) return false;
    if (length < min_len) return true;
    const uint8_t o = orientation(oa & 1u, ob & 1u);
    if (!((mask >> o) & 1u)) return true;
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
      if (w < out_cap)
        out[w] = m;
      else if (overflow)
        atomicOr(overflow, 4u);
      ++w;
    } else {
      ++cnt;
    }
    return true;
  };
  // the partners the warp's own lanes hold (site i + d is lane + d's), passed by shuffles; every
  // lane takes part until no walk can go on inside the warp
  uint64_t j = i + 1;
  for (uint32_t d = 1; d < 32; ++d) {
    const uint32_t b_record = __shfl_down_sync(0xffffffffu, a.record, d);
    const uint32_t b_pos = __shfl_down_sync(0xffffffffu, a.pos, d);
    const uint32_t b_pattern = __shfl_down_sync(0xffffffffu, (uint32_t)a.pattern, d);
    if (walking && lane + d < 32) {
      walking = j < seg_end && partner(j, b_record, b_pos, b_pattern);
      ++j;
    }
    if (!__any_sync(0xffffffffu, walking && lane + d + 1 < 32)) break;
  }
  // past the warp's sites: from memory
  for (; walking && j < seg_end; ++j) {
    const ah_hit b = hits[j];
    walking = partner(j, b.record, b.pos, b.pattern);
  }
  if (!kEmit && i < n) counts[i] = cnt;
}

}  // namespace

void launch_pair_walk(cudaStream_t s, bool emit, const ah_hit* hits, uint64_t cap, const uint64_t* d_n,
                      const uint64_t* pair_off, const uint8_t* plen, uint32_t min_len, uint32_t max_len, uint32_t mask,
                      uint32_t* counts, const uint64_t* out_off, ah_amplicon* out, uint64_t out_cap,
                      uint32_t* overflow) {
  const unsigned blocks = (unsigned)std::max<uint64_t>(1, (cap + 255) / 256);
  if (emit)
    k_pair_walk<true><<<blocks, 256, 0, s>>>(hits, cap, pair_off, plen, min_len, max_len, mask, nullptr, out_off, out,
                                             d_n, out_cap, overflow);
  else
    k_pair_walk<false><<<blocks, 256, 0, s>>>(hits, cap, pair_off, plen, min_len, max_len, mask, counts, nullptr,
                                              nullptr, d_n, out_cap, overflow);
}

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

// ------------------------------------------------------------------------------------------
// Allocation-free pairing.
//
// Some callers cannot allocate device memory while they run this step. One example is an
// application that hands all of the GPU's memory to its own pool before it loads this library.
// Another is a latency-bound loop where a cudaMalloc, with its implicit synchronisation, is not
// acceptable. ah_pair_amplicons_noalloc gives them the pairing stage with every buffer supplied by
// the caller. Its only scratch memory (per-site partner counts, their prefix sums and per-block
// partial sums) lives in the file-scope array below, sized for kNoAllocMaxSites sites and held by
// every GPU that loads the library until the process exits.
namespace ah {
namespace {

constexpr uint64_t kNoAllocMaxSites = 1ull << 20;
constexpr int kNaThreads = 256;
constexpr int kNaItems = 8;
constexpr uint64_t kNaTile = (uint64_t)kNaThreads * kNaItems;
constexpr uint64_t kNaBlocks = (kNoAllocMaxSites + kNaTile - 1) / kNaTile;  // 512
constexpr size_t kNaCountsOff = 0;
constexpr size_t kNaOffsetsOff = kNoAllocMaxSites * sizeof(uint32_t);
constexpr size_t kNaSumsOff = kNaOffsetsOff + ((kNoAllocMaxSites + 1) * sizeof(uint64_t) + 255) / 256 * 256;
constexpr size_t kNaScratchBytes = kNaSumsOff + kNaBlocks * sizeof(uint64_t);

static __device__ __align__(256) unsigned char g_pair_scratch[kNaScratchBytes];

// The device address of g_pair_scratch on the current device.  The first lookup on a device loads
// this file's device code there (CUDA loads modules lazily), which also allocates the array; later
// lookups only read the runtime's symbol table, so the address is looked up on every call rather
// than cached, and a call after a device reset sees the new one.
cudaError_t na_scratch(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_pair_scratch);
  *out = (unsigned char*)p;
  return e;
}

__device__ __forceinline__ uint64_t na_block_exclusive(uint64_t v, uint64_t* total) {
  __shared__ uint64_t ws[kNaThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t s = lane < kNaThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kNaThreads / 32) ws[lane] = s;
  }
  __syncthreads();
  const uint64_t before = (warp ? ws[warp - 1] : 0) + x - v;
  *total = ws[kNaThreads / 32 - 1];
  __syncthreads();
  return before;
}

// each thread owns kNaItems consecutive counts; pass 1 writes per-block sums
__global__ void k_na_sums(const uint32_t* __restrict__ counts, uint64_t n, uint64_t* __restrict__ sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kNaTile + (uint64_t)threadIdx.x * kNaItems;
  uint64_t s = 0;
  for (int i = 0; i < kNaItems; ++i)
    if (base + i < n) s += counts[base + i];
  uint64_t total;
  na_block_exclusive(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one CTA: exclusive scan of at most kNaBlocks block sums (two per thread); total -> offsets[n]
__global__ void k_na_scan_sums(uint64_t* __restrict__ sums, uint64_t nb, uint64_t* __restrict__ total_out) {
  const uint64_t i0 = 2 * (uint64_t)threadIdx.x, i1 = i0 + 1;
  const uint64_t a = i0 < nb ? sums[i0] : 0, b = i1 < nb ? sums[i1] : 0;
  uint64_t total;
  const uint64_t ex = na_block_exclusive(a + b, &total);
  if (i0 < nb) sums[i0] = ex;
  if (i1 < nb) sums[i1] = ex + a;
  if (threadIdx.x == 0) *total_out = total;
}

__global__ void k_na_apply(const uint32_t* __restrict__ counts, uint64_t n, const uint64_t* __restrict__ sums,
                           uint64_t* __restrict__ offsets) {
  const uint64_t base = (uint64_t)blockIdx.x * kNaTile + (uint64_t)threadIdx.x * kNaItems;
  uint64_t v[kNaItems], s = 0;
  for (int i = 0; i < kNaItems; ++i) {
    v[i] = base + i < n ? counts[base + i] : 0;
    s += v[i];
  }
  uint64_t total;
  uint64_t ex = na_block_exclusive(s, &total) + sums[blockIdx.x];
  for (int i = 0; i < kNaItems; ++i) {
    if (base + i < n) offsets[base + i] = ex;
    ex += v[i];
  }
}

}  // namespace

// Loads this file's device code, and with it the allocation-free pairing's scratch array, on the
// current device (called when a context is created, so that a caller who creates a context before
// handing the rest of the GPU's memory to its own pool never pays for it later).
cudaError_t noalloc_prepare() {
  unsigned char* p = nullptr;
  return na_scratch(&p);
}

}  // namespace ah

extern "C" ah_status ah_pair_amplicons_noalloc(void* cuda_stream, const ah_hit* d_hits, uint64_t n_hits,
                                               const uint64_t* d_pair_offsets, const uint8_t* d_pattern_len,
                                               uint32_t min_len, uint32_t max_len, uint32_t orient_mask,
                                               ah_amplicon* d_out, uint64_t out_capacity, uint64_t* n_out) {
  using namespace ah;
  if (!n_out || min_len > max_len) return AH_EINVAL;
  *n_out = 0;
  if (n_hits > kNoAllocMaxSites) return AH_EINVAL;
  if (n_hits && (!d_hits || !d_pair_offsets || !d_pattern_len)) return AH_EINVAL;
  // an error left on this thread by earlier, unrelated work is not ours to report or to clear:
  // refuse before enqueuing anything, and leave it in place
  if (cudaPeekAtLastError() != cudaSuccess) return AH_ECUDA;
  unsigned char* scratch = nullptr;
  if (na_scratch(&scratch) != cudaSuccess) return AH_ECUDA;
  if (n_hits == 0) return AH_OK;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  uint32_t* counts = (uint32_t*)(scratch + kNaCountsOff);
  uint64_t* offsets = (uint64_t*)(scratch + kNaOffsetsOff);
  uint64_t* sums = (uint64_t*)(scratch + kNaSumsOff);
  const unsigned blocks = (unsigned)((n_hits + 255) / 256);
  const unsigned nb = (unsigned)((n_hits + kNaTile - 1) / kNaTile);
  // every count, offset and block sum for the n_hits sites is written before it is read, so the
  // previous call's contents need no clearing
  // each launch is checked as it is made (the thread had no pending error on entry, so an error
  // now is this launch's); a failure returns with the passes before it still enqueued
  k_pair_walk<false><<<blocks, 256, 0, stream>>>(d_hits, n_hits, d_pair_offsets, d_pattern_len, min_len, max_len,
                                                 orient_mask & 15u, counts, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return AH_ECUDA;
  k_na_sums<<<nb, kNaThreads, 0, stream>>>(counts, n_hits, sums);
  if (cudaGetLastError() != cudaSuccess) return AH_ECUDA;
  k_na_scan_sums<<<1, kNaThreads, 0, stream>>>(sums, nb, offsets + n_hits);
  if (cudaGetLastError() != cudaSuccess) return AH_ECUDA;
  k_na_apply<<<nb, kNaThreads, 0, stream>>>(counts, n_hits, sums, offsets);
  if (cudaGetLastError() != cudaSuccess) return AH_ECUDA;
  uint64_t total = 0;
  if (cudaMemcpyAsync(&total, offsets + n_hits, sizeof total, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return AH_ECUDA;
  *n_out = total;
  if (total > out_capacity) return AH_EOVERFLOW;
  if (total && !d_out) return AH_EINVAL;
  if (total)
    k_pair_walk<true><<<blocks, 256, 0, stream>>>(d_hits, n_hits, d_pair_offsets, d_pattern_len, min_len, max_len,
                                                  orient_mask & 15u, nullptr, offsets, d_out);
  return cudaGetLastError() == cudaSuccess ? AH_OK : AH_ECUDA;
}
