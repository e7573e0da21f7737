// Shared device utilities: error reporting, status word, device-wide exclusive scan, packing.
#include <algorithm>
#include <cstdarg>
#include <cstring>

#include "ah_internal.h"

namespace ah {

ah_status fail(ah_ctx* ctx, ah_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[2048];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

void dfree(ah_ctx* ctx, void* p) {
  if (p) cudaFreeAsync(p, ctx->stream);
}

ah_status copy_to_host(ah_ctx* ctx, void* dst, const void* src, uint64_t bytes) {
  if (bytes) {
    cudaPointerAttributes pa;
    const bool locked = cudaPointerGetAttributes(&pa, dst) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if (locked || bytes <= (64u << 10)) {
      AH_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    } else {
      for (int b = 0; b < 2; ++b) {
        if (!ctx->bounce[b]) AH_CUDA(ctx, cudaMallocHost(&ctx->bounce[b], kBounceBytes));
        if (!ctx->bounce_ev[b]) AH_CUDA(ctx, cudaEventCreateWithFlags(&ctx->bounce_ev[b], cudaEventDisableTiming));
      }
      // chunk i lands in buffer i % 2 while the host copies chunk i - 1 out of the other
      uint64_t off[2] = {0, 0}, len[2] = {0, 0};
      int i = 0;
      for (uint64_t o = 0; o < bytes; o += kBounceBytes, ++i) {
        const int b = i & 1;
        if (len[b]) {
          AH_CUDA(ctx, cudaEventSynchronize(ctx->bounce_ev[b]));
          memcpy((char*)dst + off[b], ctx->bounce[b], len[b]);
        }
        off[b] = o;
        len[b] = std::min<uint64_t>(kBounceBytes, bytes - o);
        AH_CUDA(ctx, cudaMemcpyAsync(ctx->bounce[b], (const char*)src + o, len[b], cudaMemcpyDeviceToHost, ctx->stream));
        AH_CUDA(ctx, cudaEventRecord(ctx->bounce_ev[b], ctx->stream));
      }
      for (int k = 0; k < 2; ++k) {
        const int b = (i + k) & 1;  // the older chunk first
        if (!len[b]) continue;
        AH_CUDA(ctx, cudaEventSynchronize(ctx->bounce_ev[b]));
        memcpy((char*)dst + off[b], ctx->bounce[b], len[b]);
        len[b] = 0;
      }
    }
  }
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return AH_OK;
}

ah_status read_u64(ah_ctx* ctx, const uint64_t* d, uint64_t* h) {
  AH_CUDA(ctx, cudaMemcpyAsync(h, d, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return AH_OK;
}

ah_status check_status(ah_ctx* ctx) {
  AH_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  uint32_t s = *ctx->h_status;
  if (s) {
    AH_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream));
    if (s & ST_SCAN_MISMATCH)
      return fail(ctx, AH_EINTERNAL, "device self-check: bit-sliced matcher disagreed with the exact re-check");
    if (s & ST_BAD_INPUT) return fail(ctx, AH_EINVAL, "device input check: an index past the batch");
    if (s & ST_TM_LIMIT)
      return fail(ctx, AH_ELIMIT,
                  "degenerate site Tm: more qualifying primer variants than the enumeration bound, and the chain "
                  "method does not apply (salt method 6, or a variant whose entropy sum could reach zero)");
    return fail(ctx, AH_EINTERNAL, "device self-check failed (status 0x%x)", s);
  }
  return AH_OK;
}

ah_status drain_timings(ah_ctx* ctx) {
  if (ctx->ev_pending.empty()) return AH_OK;
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto& pr : ctx->ev_pending) {
    float ms = 0.f;
    AH_CUDA(ctx, cudaEventElapsedTime(&ms, pr.first, pr.second));
    ctx->scan_ms += ms;
  }
  ctx->ev_pending.clear();
  ctx->drain_gen++;
  return AH_OK;
}

// ------------------------------------------------------------------------------------------
// Exclusive scan of n counts into n+1 offsets (out[n] = total).  Three passes: per-block sums,
// a single-CTA scan of the block sums, and per-block scans with the block's offset.

namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ uint64_t block_exclusive(uint64_t v, uint64_t* total) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  uint64_t before = (warp ? warp_sums[warp - 1] : 0) + x - v;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

template <class T>
__global__ void k_block_sums(const T* __restrict__ in, uint64_t n, uint64_t* __restrict__ sums) {
  uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) s += (uint64_t)in[idx];
  }
  uint64_t total;
  block_exclusive<T>(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// exclusive scan of the block sums in place (one CTA, loops over chunks); writes the grand total
__global__ void k_scan_sums(uint64_t* sums, uint64_t nb, uint64_t* total_out) {
  uint64_t carry = 0;
  for (uint64_t base = 0; base < nb; base += kScanThreads) {
    uint64_t idx = base + threadIdx.x;
    uint64_t v = idx < nb ? sums[idx] : 0;
    uint64_t total;
    uint64_t ex = block_exclusive<uint64_t>(v, &total);
    if (idx < nb) sums[idx] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <class T>
__global__ void k_scan_apply(const T* __restrict__ in, uint64_t n, const uint64_t* __restrict__ sums,
                             uint64_t* __restrict__ out) {
  // each thread owns kScanItems consecutive elements
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? (uint64_t)in[base + i] : 0;
    s += v[i];
  }
  uint64_t total;
  uint64_t ex = block_exclusive<T>(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
}

template <class T>
ah_status exclusive_scan(ah_ctx* ctx, const T* d_in, uint64_t* d_out, uint64_t n) {
  if (n == 0) {
    AH_CUDA(ctx, cudaMemsetAsync(d_out, 0, sizeof(uint64_t), ctx->stream));
    return AH_OK;
  }
  uint64_t nb = (n + kScanTile - 1) / kScanTile;
  uint64_t* sums;
  ah_status st = dalloc(ctx, &sums, nb);
  if (st) return st;
  k_block_sums<T><<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(d_in, n, sums);
  k_scan_sums<<<1, kScanThreads, 0, ctx->stream>>>(sums, nb, d_out + n);
  k_scan_apply<T><<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(d_in, n, sums, d_out);
  launched(ctx, 3);
  dfree(ctx, sums);
  AH_CUDA(ctx, cudaGetLastError());
  return AH_OK;
}
template <class T>
void exclusive_scan_s(cudaStream_t s, const T* d_in, uint64_t* d_out, uint64_t n, uint64_t* sums) {
  if (n == 0) {
    cudaMemsetAsync(d_out, 0, sizeof(uint64_t), s);
    return;
  }
  const uint64_t nb = (n + kScanTile - 1) / kScanTile;
  k_block_sums<T><<<(unsigned)nb, kScanThreads, 0, s>>>(d_in, n, sums);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb, d_out + n);
  k_scan_apply<T><<<(unsigned)nb, kScanThreads, 0, s>>>(d_in, n, sums, d_out);
}
}  // namespace

uint64_t scan_scratch_elems(uint64_t n) { return std::max<uint64_t>(1, (n + kScanTile - 1) / kScanTile); }
void exclusive_scan_u32_s(cudaStream_t s, const uint32_t* d_in, uint64_t* d_out, uint64_t n, uint64_t* scratch) {
  exclusive_scan_s<uint32_t>(s, d_in, d_out, n, scratch);
}
void exclusive_scan_u64_s(cudaStream_t s, const uint64_t* d_in, uint64_t* d_out, uint64_t n, uint64_t* scratch) {
  exclusive_scan_s<uint64_t>(s, d_in, d_out, n, scratch);
}

ah_status exclusive_scan_u32(ah_ctx* ctx, const uint32_t* d_in, uint64_t* d_out, uint64_t n) {
  return exclusive_scan<uint32_t>(ctx, d_in, d_out, n);
}
ah_status exclusive_scan_u64(ah_ctx* ctx, const uint64_t* d_in, uint64_t* d_out, uint64_t n) {
  return exclusive_scan<uint64_t>(ctx, d_in, d_out, n);
}

}  // namespace ah
