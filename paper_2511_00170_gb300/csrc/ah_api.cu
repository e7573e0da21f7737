// C ABI entry points: context, packing, primers, object accessors.  The path's stages live in
// ah_scan.cu, ah_pair.cu, ah_tm.cu and ah_extract.cu.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstring>

#include "ah_internal.h"

using namespace ah;

// ------------------------------------------------------------------------------------------
// packing kernels
//
// One CTA per item (a piece of one record, at most 2^20 bases); each warp turns 16 groups (512
// bases) into plane words at a time from 16-byte loads.  The source may be device memory or
// page-locked host memory, which the kernels then read over the host link.
namespace {

struct PackItem {
  uint64_t src_off;    // byte offset of the item's first base in the source buffer
  uint64_t dst_group;  // first output group
  uint32_t n_valid;    // bases present in the source for this item
  uint32_t n_groups;   // groups to write (padding included)
};

constexpr int kPackThreads = 256;

// Items whose source is 16-byte aligned: every lane converts 16 bases fetched with one 16-byte load
// (a warp covers 512 bases = 16 groups); the code bits of four bytes are gathered with one
// multiply each, and lanes 2l and 2l+1 join their halves of group l with a shuffle.
__device__ __forceinline__ uint32_t gather4(uint32_t b) {  // bit 0 of bytes 0..3 -> bits 0..3
  return (b * 0x10204080u) >> 28;
}
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {  // 0x80 in each zero byte, exactly
  return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
}

// Items to warps: per_warp = false, a block per item (its warps split the item; long records);
// per_warp = true, a warp per item over a grid-stride loop (many short records).
template <bool per_warp>
__global__ void k_pack16(const uint8_t* __restrict__ src, const PackItem* __restrict__ items, uint64_t n_items,
                         uint2* __restrict__ planes, uint32_t* __restrict__ invalid) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = per_warp ? ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x;
  const uint64_t wstep = per_warp ? ((uint64_t)gridDim.x * blockDim.x) >> 5 : n_items;
  const uint32_t warp = per_warp ? 0u : (threadIdx.x >> 5), nwarps = per_warp ? 1u : (blockDim.x >> 5);
  for (uint64_t ix = w0; ix < n_items; ix += wstep) {
  const PackItem it = items[ix];
  const uint8_t* base = (const uint8_t*)((uintptr_t)src + it.src_off);  // src may be null: offsets are then addresses
  for (uint32_t blk = warp; blk * 16u < it.n_groups; blk += nwarps) {
    const uint32_t x0 = blk * 512u + (uint32_t)lane * 16u;  // first base of this lane's 16
    uint32_t w[4] = {0x4E4E4E4Eu, 0x4E4E4E4Eu, 0x4E4E4E4Eu, 0x4E4E4E4Eu};  // 'N' past the record
    if (x0 + 16u <= it.n_valid) {
      const uint4 v = __ldg((const uint4*)(base + x0));
      w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
    } else if (x0 < it.n_valid) {
      for (uint32_t i = 0; i < it.n_valid - x0; ++i)
        w[i >> 2] = (w[i >> 2] & ~(0xFFu << (8 * (i & 3)))) | ((uint32_t)__ldg(base + x0 + i) << (8 * (i & 3)));
    }
    uint32_t lo = 0, hi = 0, inv = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t u = w[q] | 0x20202020u;  // lower case
      const uint32_t ok = zero_bytes(u ^ 0x61616161u) | zero_bytes(u ^ 0x63636363u) | zero_bytes(u ^ 0x67676767u) |
                          zero_bytes(u ^ 0x74747474u);
      const uint32_t bad = ((~ok) >> 7) & 0x01010101u;
      lo |= gather4((w[q] >> 1) & 0x01010101u) << (4 * q);
      hi |= gather4((w[q] >> 2) & 0x01010101u) << (4 * q);
      inv |= gather4(bad) << (4 * q);
    }
    lo &= ~inv;
    hi &= ~inv;
    const uint32_t lo2 = __shfl_xor_sync(0xffffffffu, lo, 1), hi2 = __shfl_xor_sync(0xffffffffu, hi, 1),
                   inv2 = __shfl_xor_sync(0xffffffffu, inv, 1);
    const uint32_t g = blk * 16u + ((uint32_t)lane >> 1);
    if (!(lane & 1) && g < it.n_groups) {
      planes[it.dst_group + g] = make_uint2(lo | (lo2 << 16), hi | (hi2 << 16));
      invalid[it.dst_group + g] = inv | (inv2 << 16);
    }
  }
  }
}

// the 16 bases of one 16-byte word as bit masks: lo | hi << 16 (code bits) and inv (non-ACGT)
__device__ __forceinline__ void word_masks(const uint4 v, uint32_t* lohi, uint32_t* inv_out) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t lo = 0, hi = 0, inv = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t u = w[q] | 0x20202020u;  // lower case
    const uint32_t ok = zero_bytes(u ^ 0x61616161u) | zero_bytes(u ^ 0x63636363u) | zero_bytes(u ^ 0x67676767u) |
                        zero_bytes(u ^ 0x74747474u);
    lo |= gather4((w[q] >> 1) & 0x01010101u) << (4 * q);
    hi |= gather4((w[q] >> 2) & 0x01010101u) << (4 * q);
    inv |= gather4(((~ok) >> 7) & 0x01010101u) << (4 * q);
  }
  *lohi = (lo & ~inv) | ((hi & ~inv) << 16);
  *inv_out = inv;
}

// Items at any byte alignment.  Word c of an item is the aligned 16 bytes at A + 16c, where A is
// the item's start rounded down to 16 and r = start - A; it holds item bases 16c - r .. 16c - r + 15.
// Only words that hold at least one of the item's bases are read (an aligned 16-byte word never
// crosses a page or an allocation boundary), bytes outside the item count as 'N', and group g is
// bits r .. r + 31 of words 2g, 2g+1, 2g+2: lane 2j builds group j of the warp's 16 from its own
// word and its two neighbours' (lane 31 also reads the word after the warp's 32).
template <bool per_warp>
__global__ void k_pack16u(const uint8_t* __restrict__ src, const PackItem* __restrict__ items, uint64_t n_items,
                          uint2* __restrict__ planes, uint32_t* __restrict__ invalid) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = per_warp ? ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x;
  const uint64_t wstep = per_warp ? ((uint64_t)gridDim.x * blockDim.x) >> 5 : n_items;
  const uint32_t warp = per_warp ? 0u : (threadIdx.x >> 5), nwarps = per_warp ? 1u : (blockDim.x >> 5);
  for (uint64_t ix = w0; ix < n_items; ix += wstep) {
  const PackItem it = items[ix];
  const uintptr_t start = (uintptr_t)src + it.src_off;  // src may be null: offsets are then addresses
  const uint4* A = (const uint4*)(start & ~(uintptr_t)15);
  const uint32_t r = (uint32_t)(start & 15);
  const uint64_t end = (uint64_t)it.n_valid + r;  // item bytes end here, counted from A
  auto masks = [&](uint64_t c, uint32_t* lohi, uint32_t* inv) {
    *lohi = 0;
    *inv = 0xFFFFu;
    if (16 * c >= end) return;
    word_masks(__ldg(A + c), lohi, inv);
    // keep bytes i with 0 <= 16c + i - r < n_valid
    const int64_t lo_i = (int64_t)r - 16 * (int64_t)c, hi_i = (int64_t)end - 16 * (int64_t)c;
    uint32_t keep = 0xFFFFu;
    if (hi_i < 16) keep &= (1u << hi_i) - 1u;
    if (lo_i > 0) keep &= ~((1u << lo_i) - 1u);
    *lohi &= keep | (keep << 16);
    *inv |= ~keep & 0xFFFFu;
  };
  for (uint32_t blk = warp; blk * 16u < it.n_groups; blk += nwarps) {
    const uint64_t c = (uint64_t)blk * 32u + (uint64_t)lane;
    uint32_t p, v, ph = 0, vh = 0xFFFFu;
    masks(c, &p, &v);
    if (lane == 31) masks(c + 1, &ph, &vh);
    const uint32_t p1 = __shfl_down_sync(0xffffffffu, p, 1), v1 = __shfl_down_sync(0xffffffffu, v, 1);
    uint32_t p2 = __shfl_down_sync(0xffffffffu, p, 2), v2 = __shfl_down_sync(0xffffffffu, v, 2);
    const uint32_t hp = __shfl_down_sync(0xffffffffu, ph, 1), hv = __shfl_down_sync(0xffffffffu, vh, 1);
    if (lane == 30) p2 = hp, v2 = hv;
    const uint32_t g = blk * 16u + ((uint32_t)lane >> 1);
    if (!(lane & 1) && g < it.n_groups) {
      // 48-bit windows (words 2g, 2g+1, 2g+2) of each mask, shifted right by r
      const uint32_t lo32 = (p & 0xFFFFu) | (p1 << 16), lo_hi = p2 & 0xFFFFu;
      const uint32_t hi32 = (p >> 16) | (p1 & 0xFFFF0000u), hi_hi = p2 >> 16;
      const uint32_t in32 = (v & 0xFFFFu) | (v1 << 16), in_hi = v2 & 0xFFFFu;
      planes[it.dst_group + g] = make_uint2(__funnelshift_r(lo32, lo_hi, r), __funnelshift_r(hi32, hi_hi, r));
      invalid[it.dst_group + g] = __funnelshift_r(in32, in_hi, r);
    }
  }
  }
}

// sparse invalid words back into a batch's bitmap; an index past the batch is refused (status bit)
__global__ void k_scatter_invalid(const uint64_t* __restrict__ groups, const uint32_t* __restrict__ words, uint64_t n,
                                  uint32_t* __restrict__ invalid, uint64_t n_groups, uint32_t* status) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g = groups[i];
    if (g < n_groups)
      invalid[g] = words[i];
    else
      atomicOr(status, (uint32_t)ST_BAD_INPUT);
  }
}

// Layout from device-resident record ranks (record r: source bytes [rank[r], rank[r + 1]), rank[n]
// = total): each record's length and group count; then, from the group offsets, its packing item
// and (without caller ids) its genome id.
__global__ void k_ranked_lengths(const uint64_t* __restrict__ rank, uint64_t total, uint32_t n,
                                 uint32_t* __restrict__ rec_len, uint32_t* __restrict__ groups) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint64_t len = (r + 1 < n ? rank[r + 1] : total) - rank[r];
  rec_len[r] = (uint32_t)len;
  groups[r] = (uint32_t)record_groups(len);
}

__global__ void k_ranked_items(const uint64_t* __restrict__ rank, const uint32_t* __restrict__ rec_len,
                               const uint32_t* __restrict__ groups, const uint64_t* __restrict__ rec_group, uint32_t n,
                               PackItem* __restrict__ items, uint32_t* __restrict__ genome_id) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  items[r] = PackItem{rank[r], rec_group[r], rec_len[r], groups[r]};
  if (genome_id) genome_id[r] = r;
}

void free_batch_arrays(ah_batch* b) {
  if (!b || !b->ctx) return;
  dfree(b->ctx, b->rec_group);
  if (b->view) return;
  dfree(b->ctx, b->planes);
  dfree(b->ctx, b->invalid);
  dfree(b->ctx, b->rec_len);
  dfree(b->ctx, b->genome_id);
}

// a batch made on another context may be read by any context on the same device
bool usable(const ah_ctx* ctx, const ah_batch* b) { return b->ctx == ctx || (b->ctx && b->ctx->device == ctx->device); }

// record layout shared by both packing paths
ah_status layout_batch(ah_ctx* ctx, uint32_t n_rec, const uint64_t* lens, const uint32_t* genome_ids, ah_batch* b) {
  b->ctx = ctx;
  b->n_records = n_rec;
  b->h_rec_group.resize(n_rec);
  b->h_rec_len.resize(n_rec);
  uint64_t cursor = 0, bases = 0;
  for (uint32_t r = 0; r < n_rec; ++r) {
    if (lens[r] > 0xffffffffull) return fail(ctx, AH_EINVAL, "record %u is longer than 2^32-1 bases", r);
    b->h_rec_group[r] = cursor;
    b->h_rec_len[r] = (uint32_t)lens[r];
    cursor += record_groups(lens[r]);
    bases += lens[r];
  }
  b->n_bases = bases;
  b->n_groups = cursor;
  b->alloc_groups = cursor + kTailGroups;
  ah_status st;
  if ((st = dalloc(ctx, &b->planes, b->alloc_groups))) return st;
  if ((st = dalloc(ctx, &b->invalid, b->alloc_groups))) return st;
  if ((st = dalloc(ctx, &b->rec_group, n_rec))) return st;
  if ((st = dalloc(ctx, &b->rec_len, n_rec))) return st;
  if ((st = dalloc(ctx, &b->genome_id, n_rec))) return st;
  std::vector<uint32_t> gid(n_rec);
  for (uint32_t r = 0; r < n_rec; ++r) gid[r] = genome_ids ? genome_ids[r] : r;
  AH_CUDA(ctx, cudaMemcpyAsync(b->rec_group, b->h_rec_group.data(), n_rec * sizeof(uint64_t), cudaMemcpyHostToDevice,
                               ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(b->rec_len, b->h_rec_len.data(), n_rec * sizeof(uint32_t), cudaMemcpyHostToDevice,
                               ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(b->genome_id, gid.data(), n_rec * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
  // the tail past the last record: code 0, invalid
  AH_CUDA(ctx, cudaMemsetAsync(b->planes + b->n_groups, 0, kTailGroups * sizeof(uint2), ctx->stream));
  AH_CUDA(ctx, cudaMemsetAsync(b->invalid + b->n_groups, 0xFF, kTailGroups * sizeof(uint32_t), ctx->stream));
  // host vectors above must outlive the async copies
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return AH_OK;
}

// items for record r's bases [from, to) placed at source offset src_off; the last piece of a
// record also writes the record's padding groups
void add_items(std::vector<PackItem>& items, const ah_batch* b, uint32_t r, uint64_t from, uint64_t to,
               uint64_t src_off) {
  // bases per item (a multiple of 32): a staged chunk of 256 Mi bases is then 1,024 blocks of the
  // packing kernel, enough to fill the GPU while the next chunk crosses the link
  const uint64_t piece = 1ull << 18;
  const uint64_t len = b->h_rec_len[r];
  const uint64_t rec_groups = record_groups(len);
  for (uint64_t a = from; a < to || (a == from && to == from && from == 0 && len == 0); a += piece) {
    uint64_t e = std::min(to, a + piece);
    PackItem it;
    it.src_off = src_off + (a - from);
    it.dst_group = b->h_rec_group[r] + a / 32;
    it.n_valid = (uint32_t)(e - a);
    uint64_t gend = (e == len) ? rec_groups : (e + 31) / 32;
    it.n_groups = (uint32_t)(gend - a / 32);
    if (it.n_groups) items.push_back(it);
    if (e == to) break;
  }
}

bool aligned16(const uint8_t* base, const PackItem* items, size_t n) {
  if ((uintptr_t)base & 15) return false;
  for (size_t i = 0; i < n; ++i)
    if (items[i].src_off & 15) return false;
  return true;
}

void launch_pack(cudaStream_t s, const uint8_t* d_src, const PackItem* d_items, const PackItem* h_items, size_t n,
                 ah_batch* b, ah_ctx* ctx) {
  const bool vec = aligned16(d_src, h_items, n);
  uint64_t groups = 0;
  for (size_t i = 0; i < n; ++i) groups += h_items[i].n_groups;
  if (n > 4096 && groups < 128ull * n) {
    // many short items (fewer than 128 groups, 4 Ki bases, on average): a warp per item
    const unsigned grid = (unsigned)std::min<uint64_t>((n + 7) / 8, 32ull * std::max(1, ctx->sm_count));
    if (vec)
      k_pack16<true><<<grid, kPackThreads, 0, s>>>(d_src, d_items, n, b->planes, b->invalid);
    else
      k_pack16u<true><<<grid, kPackThreads, 0, s>>>(d_src, d_items, n, b->planes, b->invalid);
    launched(ctx);
    return;
  }
  for (size_t i = 0; i < n; i += 65535) {
    const unsigned m = (unsigned)std::min<size_t>(65535, n - i);
    if (vec)
      k_pack16<false><<<m, kPackThreads, 0, s>>>(d_src, d_items + i, m, b->planes, b->invalid);
    else
      k_pack16u<false><<<m, kPackThreads, 0, s>>>(d_src, d_items + i, m, b->planes, b->invalid);
    launched(ctx);
  }
}

ah_status run_pack(ah_ctx* ctx, const uint8_t* d_src, const std::vector<PackItem>& items, ah_batch* b) {
  if (items.empty()) return AH_OK;
  PackItem* d_items;
  ah_status st = dalloc(ctx, &d_items, items.size());
  if (st) return st;
  AH_CUDA(ctx, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(PackItem), cudaMemcpyHostToDevice,
                               ctx->stream));
  launch_pack(ctx->stream, d_src, d_items, items.data(), items.size(), b, ctx);
  AH_CUDA(ctx, cudaGetLastError());
  // items (host) must stay alive until the copy has been consumed
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  dfree(ctx, d_items);
  return AH_OK;
}

// IUPAC nomenclature -> set over the packed codes (A=1, C=2, T=4, G=8); 0 if not a code
uint8_t iupac(char ch) {
  switch (std::toupper((unsigned char)ch)) {
    case 'A': return SET_A;
    case 'C': return SET_C;
    case 'G': return SET_G;
    case 'T': return SET_T;
    case 'R': return SET_A | SET_G;
    case 'Y': return SET_C | SET_T;
    case 'S': return SET_C | SET_G;
    case 'W': return SET_A | SET_T;
    case 'K': return SET_G | SET_T;
    case 'M': return SET_A | SET_C;
    case 'B': return SET_C | SET_G | SET_T;
    case 'D': return SET_A | SET_G | SET_T;
    case 'H': return SET_A | SET_C | SET_T;
    case 'V': return SET_A | SET_C | SET_G;
    case 'N': return SET_A | SET_C | SET_G | SET_T;
    default: return 0;
  }
}

// complement of a set: code c pairs with code c ^ 2 (A<->T, C<->G)
uint8_t set_complement(uint8_t s) {
  return (uint8_t)(((s & 1) << 2) | ((s & 4) >> 2) | ((s & 2) << 2) | ((s & 8) >> 2));
}

}  // namespace

// ------------------------------------------------------------------------------------------
namespace ah {

ah_status pack_batch_ranked(ah_ctx* ctx, uint32_t n, const uint8_t* d_seq, const uint64_t* d_rank,
                            const uint64_t* h_rank, const uint32_t* genome_ids, ah_batch** out) {
  *out = nullptr;
  if (n == 0) return fail(ctx, AH_EINVAL, "a batch needs at least one record");
  ah_batch* b = new ah_batch();
  b->ctx = ctx;
  b->n_records = n;
  uint32_t* groups = nullptr;
  PackItem* items = nullptr;
  const unsigned grid = (n + 255) / 256;
  // the device first: lengths, group offsets (their total sizes the planes), items, packing; the
  // host record table is filled while the device packs
  ah_status st = dalloc(ctx, &b->rec_group, (uint64_t)n + 1);  // the scan also writes the total
  if (!st) st = dalloc(ctx, &b->rec_len, n);
  if (!st) st = dalloc(ctx, &b->genome_id, n);
  if (!st) st = dalloc(ctx, &groups, n);
  if (!st) st = dalloc(ctx, &items, n);
  if (!st && genome_ids &&
      cudaMemcpyAsync(b->genome_id, genome_ids, n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
    st = fail(ctx, AH_ECUDA, "genome id copy failed");
  if (!st) {
    k_ranked_lengths<<<grid, 256, 0, ctx->stream>>>(d_rank, h_rank[n], n, b->rec_len, groups);
    launched(ctx);
    st = exclusive_scan_u32(ctx, groups, b->rec_group, n);
  }
  uint64_t dev_groups = 0;
  if (!st) st = read_u64(ctx, b->rec_group + n, &dev_groups);
  b->n_groups = dev_groups;
  b->alloc_groups = dev_groups + kTailGroups;
  if (!st) st = dalloc(ctx, &b->planes, b->alloc_groups);
  if (!st) st = dalloc(ctx, &b->invalid, b->alloc_groups);
  if (!st) {
    k_ranked_items<<<grid, 256, 0, ctx->stream>>>(d_rank, b->rec_len, groups, b->rec_group, n, items,
                                                   genome_ids ? nullptr : b->genome_id);
    launched(ctx);
    // a warp per record (any alignment), as launch_pack does for many short items
    const unsigned pgrid = (unsigned)std::min<uint64_t>((n + 7) / 8, 32ull * std::max(1, ctx->sm_count));
    k_pack16u<true><<<pgrid, kPackThreads, 0, ctx->stream>>>(d_seq, items, n, b->planes, b->invalid);
    launched(ctx);
    cudaMemsetAsync(b->planes + b->n_groups, 0, kTailGroups * sizeof(uint2), ctx->stream);
    cudaMemsetAsync(b->invalid + b->n_groups, 0xFF, kTailGroups * sizeof(uint32_t), ctx->stream);
    if (cudaGetLastError() != cudaSuccess) st = fail(ctx, AH_ECUDA, "ranked packing failed");
  }
  b->h_rec_group.resize(n);
  b->h_rec_len.resize(n);
  uint64_t cursor = 0;
  bool bad = false;
  for (uint32_t r = 0; r < n; ++r) {
    const uint64_t len = h_rank[r + 1] - h_rank[r];
    bad |= h_rank[r + 1] < h_rank[r] || len > 0xffffffffull;
    b->h_rec_group[r] = cursor;
    b->h_rec_len[r] = (uint32_t)len;
    cursor += record_groups(len);
  }
  b->n_bases = h_rank[n] - h_rank[0];
  if (!st && (bad || cursor != dev_groups)) st = fail(ctx, AH_EINTERNAL, "pack_batch_ranked: bad record ranks");
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && !st) st = fail(ctx, AH_ECUDA, "ranked packing failed");
  dfree(ctx, groups);
  dfree(ctx, items);
  if (st) {
    free_batch_arrays(b);
    delete b;
    return st;
  }
  *out = b;
  return AH_OK;
}

}  // namespace ah

extern "C" {

ah_status ah_ctx_create(ah_ctx** out, int device, void* cuda_stream) {
  if (!out) return AH_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return AH_ECUDA;
  ah_ctx* ctx = new ah_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
    delete ctx;
    return AH_ECUDA;
  }
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return AH_ECUDA;
    }
    ctx->own_stream = true;
  }
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (ah::noalloc_prepare() != cudaSuccess) {
    ah_ctx_destroy(ctx);
    return AH_ECUDA;
  }
  if (cudaMalloc(&ctx->d_status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess) {
    ah_ctx_destroy(ctx);
    return AH_ENOMEM;
  }
  // the context's own stream-ordered pool: contexts never reuse each other's freed blocks, which
  // would make one context's allocations wait for another's stream; freed memory stays cached for
  // reuse across steps
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) {
    ctx->pool = nullptr;
    ah_ctx_destroy(ctx);
    return AH_ENOMEM;
  }
  uint64_t threshold = UINT64_MAX;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  ctx->jit = &JitCache::global();
  *out = ctx;
  return AH_OK;
}

void ah_ctx_destroy(ah_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& c : ctx->compiles) c.first.join();
  ctx->jit = nullptr;
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  // blocks still held by objects of this context are released with them
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  for (int b = 0; b < 2; ++b) {
    if (ctx->bounce[b]) cudaFreeHost(ctx->bounce[b]);
    if (ctx->bounce_ev[b]) cudaEventDestroy(ctx->bounce_ev[b]);
  }
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* ah_last_error(const ah_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

ah_status ah_ctx_synchronize(ah_ctx* ctx) {
  if (!ctx) return AH_EINVAL;
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ah_status st = drain_timings(ctx);
  return st ? st : check_status(ctx);
}

void* ah_ctx_stream(const ah_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

ah_status ah_ctx_stats_get(const ah_ctx* ctx, ah_ctx_stats* out) {
  if (!ctx || !out) return AH_EINVAL;
  out->kernel_launches = ctx->n_launches;
  out->scan_launches = ctx->n_scan_launches;
  out->scan_ms = ctx->scan_ms;
  out->scan_bases = ctx->scan_bases;
  out->jit_compiles = ctx->jit_compiles;
  out->jit_ms = ctx->jit_ms;
  out->scan_ops_per_group = ctx->scan_ops_per_group;
  out->generic_scans = ctx->n_generic_scans;
  out->tm_generated = ctx->n_tm_generated;
  out->tm_builtin = ctx->n_tm_builtin;
  out->generic_bases = ctx->generic_bases;
  return AH_OK;
}

ah_status ah_ctx_stats_reset(ah_ctx* ctx) {
  if (!ctx) return AH_EINVAL;
  ah_status st = drain_timings(ctx);  // timings of replays before the reset do not count after it
  if (st) return st;
  ctx->n_launches = ctx->n_scan_launches = ctx->scan_bases = ctx->jit_compiles = ctx->n_generic_scans = ctx->generic_bases = 0;
  ctx->n_tm_generated = ctx->n_tm_builtin = 0;
  ctx->scan_ms = ctx->jit_ms = 0.0;
  return AH_OK;
}

ah_status ah_ctx_set_scan_config(ah_ctx* ctx, int threads, int groups_per_thread, int slot_cap, int shift_mode) {
  if (!ctx) return AH_EINVAL;
  if (threads < 32 || threads > 1024 || threads % 32 || groups_per_thread < 1 || groups_per_thread > 16 ||
      slot_cap < 16 || slot_cap > 4096 || (slot_cap & (slot_cap - 1)) || shift_mode < 0 || shift_mode > 2)
    return fail(ctx, AH_EINVAL, "ah_ctx_set_scan_config: values out of range");
  ctx->scan_cfg.threads = threads;
  ctx->scan_cfg.groups_per_thread = groups_per_thread;
  ctx->scan_cfg.slot_cap = slot_cap;
  ctx->scan_cfg.shift_mode = shift_mode;
  return AH_OK;
}

ah_status ah_ctx_set_scan_circuit(ah_ctx* ctx, int min_blocks, int vote_windows, int emit_queue) {
  if (!ctx) return AH_EINVAL;
  if (min_blocks < 0 || min_blocks > 32 || vote_windows < 1 || vote_windows > (1 << 20) || emit_queue < 0 ||
      emit_queue > 1)
    return fail(ctx, AH_EINVAL, "ah_ctx_set_scan_circuit: values out of range");
  ctx->scan_cfg.min_blocks = min_blocks;
  ctx->scan_cfg.vote_windows = vote_windows;
  ctx->scan_cfg.emit_queue = emit_queue;
  return AH_OK;
}

ah_status ah_ctx_set_pairs_per_kernel(ah_ctx* ctx, int pairs) {
  if (!ctx) return AH_EINVAL;
  if (pairs < 0 || pairs > 256) return fail(ctx, AH_EINVAL, "ah_ctx_set_pairs_per_kernel: 0..256");
  ctx->scan_cfg.pairs_per_kernel = pairs;
  return AH_OK;
}

ah_status ah_ctx_set_tm_kernel(ah_ctx* ctx, int mode) {
  if (!ctx) return AH_EINVAL;
  if (mode < 0 || mode > 2) return fail(ctx, AH_EINVAL, "ah_ctx_set_tm_kernel: mode 0 to 2");
  ctx->tm_kernel = mode;
  return AH_OK;
}

ah_status ah_ctx_set_tm_split(ah_ctx* ctx, uint64_t sites) {
  if (!ctx) return AH_EINVAL;
  ctx->tm_split_sites = sites ? sites : ah::kTmSplitSitesDefault;
  return AH_OK;
}

ah_status ah_ctx_set_generic_scan(ah_ctx* ctx, int mode) {
  if (!ctx) return AH_EINVAL;
  if (mode < 0 || mode > 3) return fail(ctx, AH_EINVAL, "ah_ctx_set_generic_scan: mode 0 to 3");
  ctx->generic_scan = mode;
  return AH_OK;
}

ah_status ah_ctx_inject_alloc_failures(ah_ctx* ctx, int n) {
  if (!ctx || n < 0) return AH_EINVAL;
  ctx->fail_allocs = n;
  return AH_OK;
}

ah_status ah_ctx_set_timing(ah_ctx* ctx, int enable) {
  if (!ctx) return AH_EINVAL;
  cudaSetDevice(ctx->device);
  for (int i = 0; i < 2 && enable; ++i)
    if (!ctx->ev[i]) AH_CUDA(ctx, cudaEventCreate(&ctx->ev[i]));
  ah_status st = drain_timings(ctx);
  ctx->timing = enable != 0;
  return st;
}

// ------------------------------------------------------------------------------------------
namespace {

// Pack records first .. first + n - 1 of b, record first + i read from src[i] (b's layout gives the
// lengths).  Records in device memory are read in place by the packing kernel.  Host records (page-
// locked or not) go through the copy engines: consecutive pieces that are contiguous in host memory
// become one copy per chunk of up to kChunkBases bases, into one of two staging buffers on a second
// stream, while the context's stream packs the previous chunk from HBM.  Synchronises.
// src[i]: record first + i.  one_buffer: every src lies in one allocation (its kind is checked once)
// on_chunk (may be empty): called after each staged chunk's packing is enqueued on ctx->stream with
// the end of the groups it completes (the pieces come in batch order, so with first == 0 every group
// below it holds its final contents once the stream reaches that point); with it set, the call
// returns without waiting for the context's stream.
ah_status pack_records(ah_ctx* ctx, ah_batch* b, uint32_t first, uint32_t n, const char* const* src,
                       bool one_buffer = false, const std::function<void(uint64_t)>& on_chunk = {}) {
  bool on_device = true;
  std::vector<uint64_t> dev_addr(n, 0);
  bool checked = false;
  for (uint32_t i = 0; i < n && on_device; ++i) {
    if (!b->h_rec_len[first + i]) continue;
    if (one_buffer && checked) {
      dev_addr[i] = (uint64_t)(uintptr_t)src[i];  // device memory of this device: the first check
      continue;
    }
    checked = true;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, src[i]) != cudaSuccess) {
      cudaGetLastError();
      on_device = false;
      break;
    }
    if ((pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) && pa.devicePointer &&
        pa.device == ctx->device && pa.devicePointer == (const void*)src[i])
      dev_addr[i] = (uint64_t)(uintptr_t)pa.devicePointer;
    else
      on_device = false;
  }
  if (on_device) {
    std::vector<PackItem> items;
    for (uint32_t i = 0; i < n; ++i) add_items(items, b, first + i, 0, b->h_rec_len[first + i], dev_addr[i]);
    ah_status st = run_pack(ctx, nullptr, items, b);
    if (!st && on_chunk) on_chunk(b->n_groups);
    return st;
  }
  // chunks of host pieces (records split on group boundaries), each piece at the staging offset that
  // continues the previous one, so a run of pieces contiguous in host memory is one copy.  A chunk's
  // first copy starts at the page boundary below its first byte when the bytes in between belong to
  // the same contiguous stretch of records: copies from an address inside a page crossed the link
  // at 189 GB/s on GB300, page-aligned ones at 211 GB/s.
  struct Run {
    const char* src;
    uint64_t bytes, stage_off;
  };
  constexpr uint64_t kPage = 4096;
  std::vector<std::vector<Run>> runs(1);
  std::vector<std::vector<PackItem>> items(1);
  uint64_t fill = 0, stage_max = 0;
  const char* stretch = nullptr;  // start of the contiguous stretch of records holding record i
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t r = first + i;
    const uint64_t len = b->h_rec_len[r];
    if (i == 0 || src[i] != src[i - 1] + b->h_rec_len[r - 1]) stretch = src[i];
    uint64_t done = 0;
    if (len == 0) add_items(items.back(), b, r, 0, 0, 0);  // its padding groups (nothing is read)
    while (done < len) {
      const char* sp = src[i] + done;
      uint64_t lead = 0;
      if (fill == 0) {  // a new chunk: its copy starts on a page boundary where that stays in the stretch
        lead = (uint64_t)((uintptr_t)sp % kPage);
        if (lead > (uint64_t)(sp - stretch)) lead = 0;
        fill = lead;
      }
      uint64_t take = std::min(kChunkBases - std::min(fill, kChunkBases), len - done);
      if (take < len - done) take &= ~uint64_t(31);  // split records on group boundaries
      if (take == 0) {
        runs.emplace_back();
        items.emplace_back();
        fill = 0;
        continue;
      }
      std::vector<Run>& rv = runs.back();
      if (!rv.empty() && rv.back().src + rv.back().bytes == sp && rv.back().stage_off + rv.back().bytes == fill)
        rv.back().bytes += take;
      else if (lead)
        rv.push_back({sp - lead, take + lead, 0});
      else
        rv.push_back({sp, take, fill});
      add_items(items.back(), b, r, done, done + take, fill);
      fill += take;
      stage_max = std::max(stage_max, fill);
      done += take;
    }
  }
  std::vector<PackItem> all;
  std::vector<size_t> at;
  for (auto& v : items) {
    at.push_back(all.size());
    all.insert(all.end(), v.begin(), v.end());
  }
  if (all.empty()) return AH_OK;
  ah_status st = AH_OK;
  uint8_t* staging[2] = {nullptr, nullptr};
  PackItem* d_items = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, packed[2] = {nullptr, nullptr}, ready = nullptr;
  // 16 bytes of slack: the packing kernel reads whole aligned 16-byte words around its bytes
  if (!st) st = dalloc(ctx, &staging[0], stage_max + 16);
  if (!st && runs.size() > 1) st = dalloc(ctx, &staging[1], stage_max + 16);
  if (!st) st = dalloc(ctx, &d_items, all.size());
  cudaError_t e = cudaSuccess;
  if (!st) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess && !st; ++k) {
    e = cudaEventCreateWithFlags(&copied[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&packed[k], cudaEventDisableTiming);
  }
  if (!st && e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (!st && e == cudaSuccess)
    e = cudaMemcpyAsync(d_items, all.data(), all.size() * sizeof(PackItem), cudaMemcpyHostToDevice, ctx->stream);
  // the staging buffers were allocated in the context stream's order: the copy stream starts after that
  if (!st && e == cudaSuccess) e = cudaEventRecord(ready, ctx->stream);
  if (!st && e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
  for (size_t c = 0; c < runs.size() && !st && e == cudaSuccess; ++c) {
    const int w = (int)(c & 1);
    if (c >= 2) e = cudaStreamWaitEvent(cs, packed[w], 0);  // the buffer's previous chunk is packed
    for (const Run& rn : runs[c]) {
      if (e != cudaSuccess) break;
      e = cudaMemcpyAsync(staging[w] + rn.stage_off, rn.src, rn.bytes, cudaMemcpyHostToDevice, cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(copied[w], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, copied[w], 0);
    if (e == cudaSuccess && !items[c].empty())
      launch_pack(ctx->stream, staging[w], d_items + at[c], items[c].data(), items[c].size(), b, ctx);
    if (e == cudaSuccess) e = cudaEventRecord(packed[w], ctx->stream);
    if (e == cudaSuccess && on_chunk) {
      uint64_t done = 0;
      for (const PackItem& it : items[c]) done = std::max(done, it.dst_group + it.n_groups);
      on_chunk(c + 1 == runs.size() ? b->n_groups : done);
    }
  }
  if (!st && e == cudaSuccess && !on_chunk) e = cudaStreamSynchronize(ctx->stream);
  if (!st && e != cudaSuccess) st = fail(ctx, AH_ECUDA, "packing failed: %s", cudaGetErrorString(e));
  if (cs) {
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  for (int k = 0; k < 2; ++k) {
    if (copied[k]) cudaEventDestroy(copied[k]);
    if (packed[k]) cudaEventDestroy(packed[k]);
  }
  if (ready) cudaEventDestroy(ready);
  dfree(ctx, staging[0]);
  dfree(ctx, staging[1]);
  dfree(ctx, d_items);
  return st;
}

}  // namespace

}  // extern "C"

namespace ah {
ah_status pack_host_staged(ah_ctx* ctx, ah_batch* b, const uint8_t* h_seq, const uint64_t* h_offsets,
                           const std::function<void(uint64_t)>& on_chunk) {
  std::vector<const char*> src(b->n_records);
  for (uint32_t i = 0; i < b->n_records; ++i) {
    if (h_offsets[i + 1] < h_offsets[i] || h_offsets[i + 1] - h_offsets[i] != b->h_rec_len[i])
      return fail(ctx, AH_EINVAL, "record %u length differs from the batch layout", i);
    src[i] = (const char*)h_seq + h_offsets[i];
  }
  return pack_records(ctx, b, 0, b->n_records, src.data(), true, on_chunk);
}

ah_status pack_concat_upto(ah_ctx* ctx, ah_batch* b, const uint8_t* d_src, const uint64_t* start, uint64_t to,
                           ConcatCursor* cur, uint64_t* done_groups) {
  std::vector<PackItem> items;
  while (cur->r < b->n_records) {
    const uint32_t r = cur->r;
    const uint64_t s = start[r], len = b->h_rec_len[r];
    uint64_t avail = to > s ? std::min(len, to - s) : 0;
    if (avail < len) avail &= ~uint64_t(31);  // a record not yet complete: whole groups only
    if (len == 0) {
      add_items(items, b, r, 0, 0, 0);  // its padding groups (nothing is read)
    } else if (avail > cur->off) {
      add_items(items, b, r, cur->off, avail, s + cur->off);
      cur->off = avail;
    }
    if (cur->off < len) break;
    cur->r++, cur->off = 0;
  }
  *done_groups = cur->r < b->n_records ? b->h_rec_group[cur->r] + cur->off / 32 : b->n_groups;
  if (items.empty()) return AH_OK;
  PackItem* d_items = nullptr;
  ah_status st = dalloc(ctx, &d_items, items.size());
  if (st) return st;
  // pageable source: the copy is staged before the call returns, so `items` may go
  AH_CUDA(ctx, cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(PackItem), cudaMemcpyHostToDevice,
                               ctx->stream));
  launch_pack(ctx->stream, d_src, d_items, items.data(), items.size(), b, ctx);
  AH_CUDA(ctx, cudaGetLastError());
  dfree(ctx, d_items);
  return AH_OK;
}
}  // namespace ah

extern "C" {

ah_status ah_pack_batch(ah_ctx* ctx, uint32_t n_rec, const char* const* seqs, const uint64_t* lens,
                        const uint32_t* genome_ids, ah_batch** out) {
  if (!ctx || !out || !lens || (n_rec && !seqs) || n_rec == 0) return fail(ctx, AH_EINVAL, "ah_pack_batch: bad arguments");
  for (uint32_t r = 0; r < n_rec; ++r)
    if (lens[r] && !seqs[r]) return fail(ctx, AH_EINVAL, "ah_pack_batch: record %u has no data", r);
  *out = nullptr;
  cudaSetDevice(ctx->device);
  ah_batch* b = new ah_batch();
  ah_status st = layout_batch(ctx, n_rec, lens, genome_ids, b);
  if (!st) st = pack_records(ctx, b, 0, n_rec, seqs);
  if (st) {
    free_batch_arrays(b);
    delete b;
    return st;
  }
  *out = b;
  return AH_OK;
}

ah_status ah_pack_batch_device(ah_ctx* ctx, uint32_t n_rec, const uint8_t* d_seq, const uint64_t* h_offsets,
                               const uint32_t* genome_ids, ah_batch** out) {
  if (!ctx || !out || !h_offsets || n_rec == 0 || !d_seq) return fail(ctx, AH_EINVAL, "ah_pack_batch_device: bad arguments");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  std::vector<uint64_t> lens(n_rec);
  for (uint32_t r = 0; r < n_rec; ++r) {
    if (h_offsets[r + 1] < h_offsets[r]) return fail(ctx, AH_EINVAL, "ah_pack_batch_device: offsets decrease");
    lens[r] = h_offsets[r + 1] - h_offsets[r];
  }
  ah_batch* b = new ah_batch();
  ah_status st = layout_batch(ctx, n_rec, lens.data(), genome_ids, b);
  std::vector<PackItem> items;
  for (uint32_t r = 0; r < n_rec && !st; ++r) add_items(items, b, r, 0, lens[r], h_offsets[r]);
  if (!st) st = run_pack(ctx, d_seq, items, b);
  if (st) {
    free_batch_arrays(b);
    delete b;
    return st;
  }
  *out = b;
  return AH_OK;
}

ah_status ah_batch_slice(ah_ctx* ctx, const ah_batch* db, uint32_t first, uint32_t count, ah_batch** out) {
  if (!ctx || !db || !out) return fail(ctx, AH_EINVAL, "ah_batch_slice: NULL argument");
  if (!usable(ctx, db)) return fail(ctx, AH_EINVAL, "ah_batch_slice: batch is on another device");
  if (count == 0 || (uint64_t)first + count > db->n_records) return fail(ctx, AH_EINVAL, "ah_batch_slice: bad range");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  ah_batch* s = new ah_batch();
  s->ctx = ctx;
  s->view = true;
  s->n_records = count;
  const uint64_t g0 = db->h_rec_group[first];
  const uint64_t g1 = (uint64_t)first + count < db->n_records ? db->h_rec_group[first + count] : db->n_groups;
  s->n_groups = g1 - g0;
  s->alloc_groups = db->alloc_groups - g0;
  s->planes = db->planes + g0;
  s->invalid = db->invalid + g0;
  s->rec_len = db->rec_len + first;
  s->genome_id = db->genome_id + first;
  s->h_rec_group.resize(count);
  s->h_rec_len.assign(db->h_rec_len.begin() + first, db->h_rec_len.begin() + first + count);
  uint64_t bases = 0;
  for (uint32_t i = 0; i < count; ++i) {
    s->h_rec_group[i] = db->h_rec_group[first + i] - g0;
    bases += s->h_rec_len[i];
  }
  s->n_bases = bases;
  ah_status st = dalloc(ctx, &s->rec_group, count);
  if (!st) {
    cudaError_t e = cudaMemcpyAsync(s->rec_group, s->h_rec_group.data(), count * sizeof(uint64_t), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = fail(ctx, AH_ECUDA, "ah_batch_slice: %s", cudaGetErrorString(e));
  }
  if (st) {
    free_batch_arrays(s);
    delete s;
    return st;
  }
  *out = s;
  return AH_OK;
}

ah_status ah_batch_create(ah_ctx* ctx, uint32_t n_rec, const uint64_t* lens, const uint32_t* genome_ids, ah_batch** out) {
  if (!ctx || !out || !lens || n_rec == 0) return fail(ctx, AH_EINVAL, "ah_batch_create: bad arguments");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  ah_batch* b = new ah_batch();
  ah_status st = layout_batch(ctx, n_rec, lens, genome_ids, b);
  if (st) {
    free_batch_arrays(b);
    delete b;
    return st;
  }
  *out = b;
  return AH_OK;
}

ah_status ah_batch_pack_range(ah_ctx* ctx, ah_batch* b, uint32_t first, uint32_t count, const uint8_t* d_seq,
                              const uint64_t* h_offsets) {
  if (!ctx || !b || !d_seq || !h_offsets || b->view) return fail(ctx, AH_EINVAL, "ah_batch_pack_range: bad arguments");
  if (!usable(ctx, b) || count == 0 || (uint64_t)first + count > b->n_records)
    return fail(ctx, AH_EINVAL, "ah_batch_pack_range: bad record range");
  cudaSetDevice(ctx->device);
  std::vector<const char*> src(count);
  for (uint32_t i = 0; i < count; ++i) {
    if (h_offsets[i + 1] < h_offsets[i] || h_offsets[i + 1] - h_offsets[i] != b->h_rec_len[first + i])
      return fail(ctx, AH_EINVAL, "ah_batch_pack_range: record %u length differs from the layout", first + i);
    src[i] = (const char*)d_seq + h_offsets[i];
  }
  return pack_records(ctx, b, first, count, src.data(), true);
}


ah_status ah_batch_export(const ah_batch* b, void* planes_out, uint64_t* n_invalid, uint64_t* inv_groups,
                          uint32_t* inv_words) {
  if (!b || !b->ctx || !n_invalid) return AH_EINVAL;
  ah_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  std::vector<uint32_t> inv(b->n_groups);
  AH_CUDA(ctx, cudaMemcpyAsync(inv.data(), b->invalid, b->n_groups * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                               ctx->stream));
  if (planes_out)
    AH_CUDA(ctx, cudaMemcpyAsync(planes_out, b->planes, b->n_groups * sizeof(uint2), cudaMemcpyDeviceToHost, ctx->stream));
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  uint64_t n = 0;
  for (uint64_t g = 0; g < b->n_groups; ++g) n += inv[g] != 0;
  const uint64_t cap = *n_invalid;
  *n_invalid = n;
  if (!inv_groups || !inv_words) return AH_OK;
  if (cap < n) return fail(ctx, AH_EOVERFLOW, "ah_batch_export: %llu invalid words, room for %llu", (unsigned long long)n,
                           (unsigned long long)cap);
  uint64_t j = 0;
  for (uint64_t g = 0; g < b->n_groups; ++g)
    if (inv[g]) inv_groups[j] = g, inv_words[j] = inv[g], ++j;
  return AH_OK;
}

}  // extern "C"

// the batch's invalid words from a sparse list (groups checked by the caller), enqueued on the
// context's stream: every word cleared, then the listed ones written
ah_status ah::upload_invalid_list(ah_ctx* ctx, uint64_t n_invalid, const uint64_t* inv_groups, const uint32_t* inv_words,
                                  InvalidList* out) {
  *out = InvalidList{};
  out->n = n_invalid;
  if (!n_invalid) return AH_OK;
  ah_status st;
  if ((st = dalloc(ctx, &out->groups, n_invalid)) || (st = dalloc(ctx, &out->words, n_invalid))) return st;
  AH_CUDA(ctx, cudaMemcpyAsync(out->groups, inv_groups, n_invalid * sizeof(uint64_t), cudaMemcpyHostToDevice,
                               ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(out->words, inv_words, n_invalid * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
  return AH_OK;
}

ah_status ah::scatter_invalid_list(ah_ctx* ctx, ah_batch* b, InvalidList* l) {
  AH_CUDA(ctx, cudaMemsetAsync(b->invalid, 0, b->n_groups * sizeof(uint32_t), ctx->stream));
  if (!l->n) return AH_OK;
  k_scatter_invalid<<<(unsigned)std::min<uint64_t>((l->n + 255) / 256, 65535), 256, 0, ctx->stream>>>(
      l->groups, l->words, l->n, b->invalid, b->n_groups, ctx->d_status);
  launched(ctx);
  AH_CUDA(ctx, cudaGetLastError());
  dfree(ctx, l->groups);
  dfree(ctx, l->words);
  *l = InvalidList{};
  return AH_OK;
}

extern "C" {

ah_status ah_batch_import(ah_ctx* ctx, ah_batch* b, const void* planes, uint64_t n_invalid, const uint64_t* inv_groups,
                          const uint32_t* inv_words) {
  if (!ctx || !b || !planes || (n_invalid && (!inv_groups || !inv_words)) || b->view)
    return fail(ctx, AH_EINVAL, "ah_batch_import: bad arguments");
  if (!usable(ctx, b)) return fail(ctx, AH_EINVAL, "ah_batch_import: batch of another device");
  for (uint64_t i = 0; i < n_invalid; ++i)
    if (inv_groups[i] >= b->n_groups)
      return fail(ctx, AH_EINVAL, "ah_batch_import: invalid word %llu at group %llu, past the batch's %llu groups",
                  (unsigned long long)i, (unsigned long long)inv_groups[i], (unsigned long long)b->n_groups);
  cudaSetDevice(ctx->device);
  AH_CUDA(ctx, cudaMemcpyAsync(b->planes, planes, b->n_groups * sizeof(uint2), cudaMemcpyHostToDevice, ctx->stream));
  InvalidList l;
  ah_status st = upload_invalid_list(ctx, n_invalid, inv_groups, inv_words, &l);
  if (!st) st = scatter_invalid_list(ctx, b, &l);
  if (st) return st;
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

ah_status ah_batch_view_get(const ah_batch* b, ah_batch_view* out) {
  if (!b || !out) return AH_EINVAL;
  out->n_records = b->n_records;
  out->n_bases = b->n_bases;
  out->n_groups = b->n_groups;
  out->planes = b->planes;
  out->invalid = b->invalid;
  out->rec_group = b->rec_group;
  out->rec_len = b->rec_len;
  out->genome_id = b->genome_id;
  return AH_OK;
}

void ah_batch_free(ah_batch* b) {
  if (!b) return;
  free_batch_arrays(b);
  delete b;
}

// ------------------------------------------------------------------------------------------
ah_status ah_primers_create(ah_ctx* ctx, uint32_t n_pairs, const char* const* fwd, const char* const* rev,
                            const uint8_t* k, uint8_t clamp, ah_primers** out) {
  if (!ctx || !out || !fwd || !rev || !k) return fail(ctx, AH_EINVAL, "ah_primers_create: NULL argument");
  if (n_pairs == 0 || n_pairs > 256) return fail(ctx, AH_EINVAL, "ah_primers_create: n_pairs must be 1..256");
  *out = nullptr;
  ah_primers* p = new ah_primers();
  p->ctx = ctx;
  p->n_pairs = n_pairs;
  p->clamp = clamp;
  std::vector<uint8_t> plen(4 * n_pairs), psets(n_pairs * 2 * 32, 0);
  for (uint32_t i = 0; i < n_pairs; ++i) {
    for (int x = 0; x < 2; ++x) {
      const char* s = x == 0 ? fwd[i] : rev[i];
      if (!s) {
        delete p;
        return fail(ctx, AH_EINVAL, "pair %u: NULL primer", i);
      }
      size_t L = strlen(s);
      if (L < 2 || L > 32 || L < clamp) {
        delete p;
        return fail(ctx, AH_EINVAL, "pair %u: primer length %zu outside [max(2, clamp), 32]", i, L);
      }
      if (k[i] > 15 || k[i] > L) {
        delete p;
        return fail(ctx, AH_EINVAL, "pair %u: k=%u exceeds 15 or the primer length", i, (unsigned)k[i]);
      }
      std::string up(L, ' ');
      for (size_t j = 0; j < L; ++j) {
        uint8_t set = iupac(s[j]);
        if (!set) {
          delete p;
          return fail(ctx, AH_EINVAL, "pair %u: '%c' is not an IUPAC nucleotide code", i, s[j]);
        }
        up[j] = (char)std::toupper((unsigned char)s[j]);
        psets[(i * 2 + x) * 32 + j] = set;
      }
      (x == 0 ? p->fwd : p->rev).push_back(up);
    }
    p->k.push_back(k[i]);
  }
  // oriented patterns: orient = 2 * strand + primer
  p->pats.resize(4 * n_pairs);
  for (uint32_t i = 0; i < n_pairs; ++i) {
    for (int strand = 0; strand < 2; ++strand) {
      for (int x = 0; x < 2; ++x) {
        const std::string& s = x == 0 ? p->fwd[i] : p->rev[i];
        const int L = (int)s.size();
        Pattern& P = p->pats[4 * i + 2 * strand + x];
        memset(&P, 0, sizeof P);
        P.len = (uint8_t)L;
        P.k = k[i];
        P.id = (uint16_t)(4 * i + 2 * strand + x);
        for (int j = 0; j < L; ++j)
          P.set[j] = strand == 0 ? iupac(s[j]) : set_complement(iupac(s[L - 1 - j]));
        // the primer's 3' end: last c positions as written, first c of the reverse complement
        P.clamp_lo = (uint8_t)(strand == 0 ? L - clamp : 0);
        P.clamp_hi = (uint8_t)(strand == 0 ? L : clamp);
        plen[P.id] = (uint8_t)L;
      }
    }
  }
  // each primer as four position masks, bit j of mask c: position j allows base code c
  std::vector<uint4> pmask(2 * (size_t)n_pairs);
  for (size_t q = 0; q < pmask.size(); ++q) {
    uint32_t m[4] = {0, 0, 0, 0};
    for (int j = 0; j < 32; ++j)
      for (int c = 0; c < 4; ++c) m[c] |= (uint32_t)((psets[q * 32 + j] >> c) & 1u) << j;
    pmask[q] = make_uint4(m[0], m[1], m[2], m[3]);
  }
  ah_status st = dalloc(ctx, &p->d_plen, plen.size());
  if (!st) st = dalloc(ctx, &p->d_psets, psets.size());
  if (!st) st = dalloc(ctx, &p->d_pk, p->k.size());
  if (!st) st = dalloc(ctx, &p->d_pmask, pmask.size());
  const std::vector<GenPattern> gen = gen_table(p->pats);
  if (!st) st = dalloc(ctx, &p->d_gen, gen.size());
  if (!st) {
    cudaMemcpyAsync(p->d_gen, gen.data(), gen.size() * sizeof(GenPattern), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(p->d_plen, plen.data(), plen.size(), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(p->d_psets, psets.data(), psets.size(), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(p->d_pk, p->k.data(), p->k.size(), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(p->d_pmask, pmask.data(), pmask.size() * sizeof(uint4), cudaMemcpyHostToDevice, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = fail(ctx, AH_ECUDA, "primer upload failed");
  }
  if (st) {
    ah_primers_free(p);
    return st;
  }
  *out = p;
  return AH_OK;
}

void ah_primers_free(ah_primers* p) {
  if (!p) return;
  if (p->ctx) {
    dfree(p->ctx, p->d_plen);
    dfree(p->ctx, p->d_psets);
    dfree(p->ctx, p->d_pk);
    dfree(p->ctx, p->d_pmask);
    dfree(p->ctx, p->d_gen);
  }
  delete p;
}

// ------------------------------------------------------------------------------------------
ah_status ah_scan_primers(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out) {
  if (!ctx || !b || !p || !out) return fail(ctx, AH_EINVAL, "ah_scan_primers: NULL argument");
  if (!usable(ctx, b) || p->ctx != ctx) return fail(ctx, AH_EINVAL, "ah_scan_primers: object from another context");
  cudaSetDevice(ctx->device);
  return scan_primers(ctx, b, p, out);
}

ah_status ah_scan_primers_per_record(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out) {
  if (!ctx || !b || !p || !out) return fail(ctx, AH_EINVAL, "ah_scan_primers_per_record: NULL argument");
  if (!usable(ctx, b) || p->ctx != ctx)
    return fail(ctx, AH_EINVAL, "ah_scan_primers_per_record: object from another context");
  cudaSetDevice(ctx->device);
  return scan_primers_per_record(ctx, b, p, out);
}

ah_status ah_hits_count(const ah_hits* h, uint64_t* n) {
  if (!h || !n) return AH_EINVAL;
  *n = h->n;
  return AH_OK;
}

ah_status ah_hits_device(const ah_hits* h, const ah_hit** d_hits, const uint64_t** d_pair_offsets) {
  if (!h) return AH_EINVAL;
  if (d_hits) *d_hits = h->d;
  if (d_pair_offsets) *d_pair_offsets = h->d_pair_off;
  return AH_OK;
}

ah_status ah_hits_copy(const ah_hits* h, ah_hit* host_out, uint64_t cap) {
  if (!h || (!host_out && cap)) return AH_EINVAL;
  uint64_t n = std::min(cap, h->n);
  return copy_to_host(h->ctx, host_out, h->d, n * sizeof(ah_hit));
}

void ah_hits_free(ah_hits* h) {
  if (!h) return;
  dfree(h->ctx, h->d);
  dfree(h->ctx, h->d_pair_off);
  delete h;
}

ah_status ah_pair_amplicons(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, uint32_t min_len,
                            uint32_t max_len, uint32_t orient_mask, ah_amplicons** out) {
  if (!ctx || !b || !p || !h || !out) return fail(ctx, AH_EINVAL, "ah_pair_amplicons: NULL argument");
  if (min_len > max_len) return fail(ctx, AH_EINVAL, "ah_pair_amplicons: min_len > max_len");
  if (h->n_pairs != p->n_pairs) return fail(ctx, AH_EINVAL, "ah_pair_amplicons: hits come from another primer set");
  cudaSetDevice(ctx->device);
  return pair_amplicons(ctx, b, p, h, min_len, max_len, orient_mask & 15u, out);
}

ah_status ah_tm_filter(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, ah_amplicons* a,
                       const ah_tm_params* params) {
  if (!ctx || !b || !p || !h || !a || !params) return fail(ctx, AH_EINVAL, "ah_tm_filter: NULL argument");
  if (params->saltcorr < 0 || params->saltcorr > 7)
    return fail(ctx, AH_EINVAL, "ah_tm_filter: salt correction method %d is not supported (0-7)", params->saltcorr);
  cudaSetDevice(ctx->device);
  return tm_filter(ctx, b, p, h, a, params);
}

ah_status ah_tm_duplexes(ah_ctx* ctx, uint32_t n, const char* const* seqs, const char* const* cseqs,
                         const ah_tm_params* params, double* tm_out) {
  if (!ctx || (n && (!seqs || !cseqs || !tm_out)) || !params) return fail(ctx, AH_EINVAL, "ah_tm_duplexes: NULL argument");
  if (params->saltcorr < 0 || params->saltcorr > 7)
    return fail(ctx, AH_EINVAL, "ah_tm_duplexes: salt correction method %d is not supported (0-7)", params->saltcorr);
  cudaSetDevice(ctx->device);
  return tm_duplexes(ctx, n, seqs, cseqs, params, tm_out);
}

ah_status ah_tm_sites(ah_ctx* ctx, uint32_t n, const char* const* primers, const char* const* sites, const uint8_t* k,
                      const uint8_t* clamp,
                      const ah_tm_params* params, double* tm_out) {
  if (!ctx || (n && (!primers || !sites || !tm_out)) || !params) return fail(ctx, AH_EINVAL, "ah_tm_sites: NULL argument");
  if (params->saltcorr < 0 || params->saltcorr > 7)
    return fail(ctx, AH_EINVAL, "ah_tm_sites: salt correction method %d is not supported (0-7)", params->saltcorr);
  cudaSetDevice(ctx->device);
  return tm_sites(ctx, n, primers, sites, k, clamp, params, tm_out);
}

ah_status ah_extract_barcodes(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, ah_amplicons* a,
                              int trim, uint32_t fb_len, uint32_t rb_len) {
  if (!ctx || !b || !p || !h || !a) return fail(ctx, AH_EINVAL, "ah_extract_barcodes: NULL argument");
  cudaSetDevice(ctx->device);
  return extract(ctx, b, p, h, a, trim, fb_len, rb_len);
}

ah_status ah_amplicons_count(const ah_amplicons* a, uint64_t* n) {
  if (!a || !n) return AH_EINVAL;
  *n = a->n;
  return AH_OK;
}

ah_status ah_amplicons_copy(const ah_amplicons* a, ah_amplicon* host_out, uint64_t cap) {
  if (!a || (!host_out && cap)) return AH_EINVAL;
  uint64_t n = std::min(cap, a->n);
  return copy_to_host(a->ctx, host_out, a->d, n * sizeof(ah_amplicon));
}

ah_status ah_amplicons_arena_size(const ah_amplicons* a, uint64_t* bytes) {
  if (!a || !bytes) return AH_EINVAL;
  *bytes = a->arena_bytes;
  return AH_OK;
}

ah_status ah_amplicons_seq_copy(const ah_amplicons* a, char* arena_out, uint64_t arena_cap, uint64_t* offsets_out,
                                uint64_t offsets_cap) {
  if (!a) return AH_EINVAL;
  if (!a->d_field_off) return fail(a->ctx, AH_EINVAL, "ah_amplicons_seq_copy: sequences were not extracted");
  if (arena_cap < a->arena_bytes || offsets_cap < 5 * a->n + 1)
    return fail(a->ctx, AH_EOVERFLOW, "ah_amplicons_seq_copy: need %llu arena bytes and %llu offsets",
                (unsigned long long)a->arena_bytes, (unsigned long long)(5 * a->n + 1));
  ah_status st = copy_to_host(a->ctx, arena_out, a->d_arena, a->arena_bytes);
  return st ? st : copy_to_host(a->ctx, offsets_out, a->d_field_off, (5 * a->n + 1) * sizeof(uint64_t));
}

void ah_amplicons_free(ah_amplicons* a) {
  if (!a) return;
  dfree(a->ctx, a->d);
  dfree(a->ctx, a->d_arena);
  dfree(a->ctx, a->d_field_off);
  dfree(a->ctx, a->d_qarena);
  delete a;
}

}  // extern "C"
