/*
 * Seeded synthetic-input generator, device side: the same counter-based draws as _synth.c
 * (SplitMix64 output function of key + (i + 1) * GOLDEN), so a genome drawn here is byte-identical
 * to the one the host filler draws.  Runs of N are computed on the host (they use log) and only
 * written here; planted templates are built on the host and scattered here.  No in-silico PCR
 * arithmetic lives in this file.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct FillItem {
  uint64_t out_off;  /* where base `first` of the genome goes */
  uint64_t first;    /* counter of the first base */
  uint64_t count;
  uint64_t key;
  double gc;
};

__global__ void k_fill(uint8_t* __restrict__ out, const FillItem* __restrict__ items) {
  const FillItem it = items[blockIdx.y];
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < it.count; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = mix64(it.key + (it.first + i + 1) * GOLDEN);
    const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    uint8_t b;
    if (u < it.gc)
      b = (r & 1) ? 'G' : 'C';
    else
      b = (r & 1) ? 'A' : 'T';
    out[it.out_off + i] = b;
  }
}

__global__ void k_runs(uint8_t* __restrict__ out, const uint64_t* __restrict__ at, const uint32_t* __restrict__ len,
                       uint64_t n) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x)
    for (uint32_t j = 0; j < len[r]; ++j) out[at[r] + j] = 'N';
}

__global__ void k_scatter(uint8_t* __restrict__ out, const uint8_t* __restrict__ src, const uint64_t* __restrict__ src_off,
                          const uint64_t* __restrict__ dst, uint64_t n) {
  for (uint64_t t = blockIdx.x; t < n; t += gridDim.x) {
    const uint64_t a = src_off[t], b = src_off[t + 1];
    for (uint64_t i = a + threadIdx.x; i < b; i += blockDim.x) out[dst[t] + (i - a)] = src[i];
  }
}

extern "C" {
/* items: n_items FillItem records (host); copies them and fills on `stream`; returns a cudaError_t */
int synth_gpu_fill(uint8_t* d_out, const void* h_items, uint64_t n_items, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  FillItem* d_items = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d_items, n_items * sizeof(FillItem), s);
  if (e != cudaSuccess) return (int)e;
  e = cudaMemcpyAsync(d_items, h_items, n_items * sizeof(FillItem), cudaMemcpyHostToDevice, s);
  for (uint64_t i0 = 0; i0 < n_items && e == cudaSuccess; i0 += 65535) {
    const unsigned ny = (unsigned)((n_items - i0) < 65535 ? (n_items - i0) : 65535);
    k_fill<<<dim3(64, ny), 256, 0, s>>>(d_out, d_items + i0);
    e = cudaGetLastError();
  }
  cudaFreeAsync(d_items, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return (int)e;
}

int synth_gpu_runs(uint8_t* d_out, const uint64_t* d_at, const uint32_t* d_len, uint64_t n, void* stream) {
  if (!n) return 0;
  k_runs<<<1024, 256, 0, (cudaStream_t)stream>>>(d_out, d_at, d_len, n);
  return (int)cudaGetLastError();
}

int synth_gpu_scatter(uint8_t* d_out, const uint8_t* d_src, const uint64_t* d_src_off, const uint64_t* d_dst, uint64_t n,
                      void* stream) {
  if (!n) return 0;
  k_scatter<<<4096, 128, 0, (cudaStream_t)stream>>>(d_out, d_src, d_src_off, d_dst, n);
  return (int)cudaGetLastError();
}
}
