// Scan stage (Supplementary, "Primer matching and clamp logic"; "We sort candidate sites"):
//   1. the run-time specialised bit-sliced kernel marks candidate sites and appends a 64-bit key
//      (pair | tile-local position | orient | mismatches) to its tile's slot list;
//   2. each tile's keys are sorted (a warp's bitonic network in registers, or a block's in shared
//      memory for tiles of more than 256 keys) and counted per pair;
//   3. an exclusive scan over the pair-major (pair, tile) counts gives every tile's output range;
//   4. keys become ah_hit records (record lookup by binary search within the tile's records) in
//      (pair, record, pos, orient) order, so pairing needs no global sort.
#include <algorithm>
#include <thread>

#include "ah_internal.h"

namespace ah {
namespace {

// must match the ScanParams of the generated source
struct ScanParamsHost {
  const uint2* planes;
  const uint32_t* invalid;
  const uint64_t* rec_group;
  const uint32_t* rec_len;
  uint32_t n_rec;
  uint32_t slot_cap;
  uint64_t group_begin;
  uint64_t n_groups;
  uint64_t* slots;
  uint32_t* tile_count;
  uint32_t* status;
  uint64_t tile_groups;      // groups per slot-list tile: the tile of group g is g / tile_groups
  unsigned long long* work;  // persistent kernels: next block to take
  uint64_t n_blocks;         // persistent kernels: blocks of threads * groups_per_thread groups
};

__global__ void k_tile_max(const uint32_t* __restrict__ tile_count, uint64_t n_tiles, uint32_t* __restrict__ out) {
  uint32_t m = 0;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_tiles; t += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, tile_count[t]);
#pragma unroll
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t* a, uint32_t n, uint64_t key) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Bitonic sort of 32 R keys held by one warp, key r * 32 + lane in v[r] of that lane: exchanges
// between lanes (distance below 32) by shuffles, between a lane's own registers (distance 32 and
// above) in place.  The loops have constant bounds, so every register index is resolved at compile
// time.
template <int R>
__device__ __forceinline__ void warp_bitonic(uint64_t (&v)[R], int lane, int m = 32 * R) {
#pragma unroll
  for (int k = 2; k <= m; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int d = j >> 5;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r & d) continue;
          const bool up = (((r << 5) | lane) & k) == 0;
          const uint64_t x = v[r], y = v[r | d];
          if ((x > y) == up) {
            v[r] = y;
            v[r | d] = x;
          }
        }
      } else {
        const bool lower = (lane & j) == 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint64_t o = __shfl_xor_sync(0xffffffffu, v[r], j);
          const bool up = (((r << 5) | lane) & k) == 0;
          // keep the smaller of the two when this lane holds the lower index of an ascending pair
          // or the upper of a descending one, else the larger: one comparison and a select
          if ((o < v[r]) == (lower == up)) v[r] = o;
        }
      }
    }
  }
}

// Sorts n <= 32 R keys in the warp's registers and writes them back; returns (to every lane) the
// pairs of the first and last keys.  With one key per lane the network spans only the next power of
// two above n (lanes past it hold padding and stay put).
template <int R>
__device__ __forceinline__ uint2 sort_regs(uint64_t* tk, uint32_t n, int lane) {
  uint64_t v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t i = (uint32_t)(r << 5) | (uint32_t)lane;
    v[r] = i < n ? tk[i] : ~0ull;
  }
  if (R == 1) {
    int m = 1;
    while (m < (int)n) m <<= 1;
    warp_bitonic<R>(v, lane, m);
  } else {
    warp_bitonic<R>(v, lane);
  }
  uint64_t last = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const uint32_t i = (uint32_t)(r << 5) | (uint32_t)lane;
    if (i < n) tk[i] = v[r];
    const uint64_t x = __shfl_sync(0xffffffffu, v[r], (int)((n - 1) & 31u));
    if (r == (int)((n - 1) >> 5)) last = x;
  }
  return make_uint2((uint32_t)(__shfl_sync(0xffffffffu, v[0], 0) >> 48), (uint32_t)(last >> 48));
}

// Sort one tile's n <= kSmallTile keys in the registers of one warp, write them back and count them
// per pair (pair in the top 16 bits).  A tile of one pair needs no search for the counts.
__device__ __forceinline__ void sort_tile(uint64_t* tk, uint32_t n, uint64_t t, uint64_t n_tiles, uint32_t n_pairs,
                                          uint32_t* tile_pair_count, int lane) {
  uint2 pp;
  if (n <= 32) pp = sort_regs<1>(tk, n, lane);
  else if (n <= 64) pp = sort_regs<2>(tk, n, lane);
  else if (n <= 128) pp = sort_regs<4>(tk, n, lane);
  else pp = sort_regs<8>(tk, n, lane);
  const uint32_t p_first = pp.x, p_last = pp.y;
  if (p_first == p_last) {
    if (lane == 0 && p_first < n_pairs) tile_pair_count[(uint64_t)p_first * n_tiles + t] = n;
    return;
  }
  __syncwarp();  // the other lanes' keys are written before they are searched
  for (uint32_t p = p_first + lane; p <= p_last && p < n_pairs; p += 32) {
    const uint32_t a = lower_bound_u64(tk, n, (uint64_t)p << 48);
    const uint32_t b = lower_bound_u64(tk, n, (uint64_t)(p + 1) << 48);
    if (b > a) tile_pair_count[(uint64_t)p * n_tiles + t] = b - a;
  }
}

constexpr uint32_t kSmallTile = 256;  // keys a tile may hold to be sorted by one warp in registers

// One warp per tile.  Tiles holding more keys are appended to big[1..] (count in big[0]) for
// k_tile_sort_big.
__global__ void k_tile_sort(uint64_t* __restrict__ slots, const uint32_t* __restrict__ tile_count, uint32_t cap,
                            uint64_t n_tiles, uint32_t n_pairs, uint32_t* __restrict__ tile_pair_count,
                            uint32_t* __restrict__ big) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (t >= n_tiles) return;
  const uint32_t n = min(tile_count[t], cap);
  if (n == 0) return;
  if (n > kSmallTile) {
    if (lane == 0) big[1 + atomicAdd(big, 1u)] = (uint32_t)t;
    return;
  }
  sort_tile(slots + t * cap, n, t, n_tiles, n_pairs, tile_pair_count, lane);
}

// The listed tiles, one block of kBigSortThreads each (a tile holds at most kBigSortKeys keys): the
// keys, padded to a power of two m, are sorted by a bitonic network in shared memory, every thread
// taking m / 2 / kBigSortThreads compare-exchanges of each of its log m (log m + 1) / 2 stages.
// A fixed grid strides over the list.
constexpr int kBigSortThreads = 256;
constexpr uint32_t kBigSortKeys = 4096;
__global__ void __launch_bounds__(kBigSortThreads) k_tile_sort_big(uint64_t* __restrict__ slots,
                                                                   const uint32_t* __restrict__ tile_count,
                                                                   uint32_t cap, uint64_t n_tiles, uint32_t n_pairs,
                                                                   uint32_t* __restrict__ tile_pair_count,
                                                                   const uint32_t* __restrict__ big) {
  __shared__ uint64_t buf[kBigSortKeys];
  const uint32_t n_big = big[0];
  for (uint32_t i = blockIdx.x; i < n_big; i += gridDim.x) {
    const uint64_t t = big[1 + i];
    const uint32_t n = min(min(tile_count[t], cap), kBigSortKeys);
    uint64_t* tk = slots + t * cap;
    uint32_t m = 2;
    while (m < n) m <<= 1;
    for (uint32_t e = threadIdx.x; e < m; e += kBigSortThreads) buf[e] = e < n ? tk[e] : ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= m; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t e = threadIdx.x; e < m / 2; e += kBigSortThreads) {
          const uint32_t lo = ((e & ~(j - 1)) << 1) | (e & (j - 1)), hi = lo + j;  // lo has bit j clear
          const uint64_t x = buf[lo], y = buf[hi];
          if ((x > y) == ((lo & k) == 0)) {
            buf[lo] = y;
            buf[hi] = x;
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t e = threadIdx.x; e < n; e += kBigSortThreads) tk[e] = buf[e];
    const uint32_t p_first = (uint32_t)(buf[0] >> 48), p_last = (uint32_t)(buf[n - 1] >> 48);
    for (uint32_t p = p_first + threadIdx.x; p <= p_last && p < n_pairs; p += kBigSortThreads) {
      const uint32_t lo = lower_bound_u64(buf, n, (uint64_t)p << 48);
      const uint32_t hi = lower_bound_u64(buf, n, (uint64_t)(p + 1) << 48);
      if (hi > lo) tile_pair_count[(uint64_t)p * n_tiles + t] = hi - lo;
    }
    __syncthreads();  // the buffer is refilled for the next tile
  }
}

// one warp per tile: sorted keys -> hit records at their pair-major output positions
// tile_base (optional) gives each tile's first position; otherwise tile t starts at t * tile_groups * 32.
// Hits at output positions >= hit_cap are dropped and flagged.
__global__ void k_emit_hits(const uint64_t* __restrict__ slots, const uint32_t* __restrict__ tile_count, uint32_t cap,
                            uint64_t n_tiles, uint64_t tile_groups, const uint64_t* __restrict__ off,
                            const uint64_t* __restrict__ rec_group, uint32_t n_rec, ah_hit* __restrict__ hits,
                            const uint64_t* __restrict__ tile_base = nullptr, uint64_t hit_cap = ~0ull,
                            uint32_t* __restrict__ overflow = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t t = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (t >= n_tiles) return;
  const uint32_t n = min(tile_count[t], cap);
  if (n == 0) return;
  const uint64_t* tk = slots + t * cap;
  const uint64_t tile_pos = tile_base ? tile_base[t] : t * tile_groups * 32ull;
  // the records the tile's sites fall in, [r_lo, r_hi]: lane 0 finds the one holding the smallest
  // position, lane 1 the one holding the largest, so a site's record search spans those only
  uint64_t p_min = ~0ull, p_max = 0;
  for (uint32_t i = lane; i < n; i += 32) {
    const uint64_t x = (tk[i] >> 16) & 0xffffffffull;
    p_min = min(p_min, x);
    p_max = max(p_max, x);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    p_min = min(p_min, __shfl_xor_sync(0xffffffffu, p_min, o));
    p_max = max(p_max, __shfl_xor_sync(0xffffffffu, p_max, o));
  }
  uint32_t r = 0;
  if (lane < 2) {
    const uint64_t pos = tile_pos + (lane ? p_max : p_min);
    uint32_t lo = 0, hi = n_rec;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (rec_group[mid] * 32ull <= pos) lo = mid; else hi = mid;
    }
    r = lo;
  }
  const uint32_t r_lo = __shfl_sync(0xffffffffu, r, 0), r_hi = __shfl_sync(0xffffffffu, r, 1);
  const bool one_pair = (tk[0] >> 48) == (tk[n - 1] >> 48);  // keys are sorted by pair first
  for (uint32_t i = lane; i < n; i += 32) {
    const uint64_t key = tk[i];
    const uint32_t pair = (uint32_t)(key >> 48);
    const uint32_t first = one_pair ? 0u : lower_bound_u64(tk, n, (uint64_t)pair << 48);
    const uint64_t o = off[(uint64_t)pair * n_tiles + t] + (i - first);
    const uint64_t pos = tile_pos + ((key >> 16) & 0xffffffffull);
    uint32_t lo = r_lo, hi = r_hi + 1;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (rec_group[mid] * 32ull <= pos) lo = mid; else hi = mid;
    }
    ah_hit h;
    h.record = lo;
    h.pos = (uint32_t)(pos - rec_group[lo] * 32ull);
    h.pattern = (uint16_t)(pair * 4u + ((key >> 8) & 3u));
    h.mism = (uint8_t)(key & 0xffu);
    h.flags = 0;
    if (o < hit_cap)
      hits[o] = h;
    else if (overflow)
      atomicOr(overflow, 2u);
  }
}

__global__ void k_pair_offsets(const uint64_t* __restrict__ off, uint64_t n_tiles, uint32_t n_pairs,
                               uint64_t* __restrict__ pair_off) {
  uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p <= n_pairs) pair_off[p] = off[(uint64_t)p * n_tiles];
}

// ------------------------------------------------------------------------------------------
// Generic scan: the same bit-sliced test with the primer set read from a table (GenPattern) at run
// time, so a new primer set needs no compile.  Each position's mismatch bit is the two-variable
// boolean function x(lo, hi) = c0 ^ (lo & c1) ^ (hi & c2) ^ (lo & hi & c3) of the shifted code
// planes, with the set's coefficients as 0 / ~0 words (three LOP3); the count is a saturating
// ripple counter of `width` bits.  A warp whose windows have all failed stops the pattern early.

static_assert(sizeof(GenPattern) * kGenMaxPatterns <= 48 * 1024, "generic pattern table exceeds default shared memory");

// mismatch bits of the 32 windows at offset j of one evaluated position
__device__ __forceinline__ uint32_t gen_mismatch(const uint4& c, int j, uint2 a, uint2 b) {
  const uint32_t lo = __funnelshift_r(a.x, b.x, j), hi = __funnelshift_r(a.y, b.y, j);
  return ((lo & ((hi & c.w) ^ c.y)) ^ (hi & c.z)) ^ c.x;
}

// bits of the windows starting in group (a, b) that pass P: no clamp mismatch, fewer than k + 1
// counted mismatches
template <int W>
__device__ __forceinline__ uint32_t gen_pass(const GenPattern& P, uint2 a, uint2 b) {
  uint32_t fail = 0;
  int e = 0;
  for (; e < P.n_clamp; e += 4) {
    const uint32_t js = *reinterpret_cast<const uint32_t*>(P.j + e);
#pragma unroll
    for (int u = 0; u < 4; ++u) fail |= gen_mismatch(P.x[e + u], (js >> (8 * u)) & 31, a, b);
  }
  if (!__any_sync(__activemask(), ~fail)) return 0;
  uint32_t c[W > 0 ? W : 1] = {};
  for (; e < P.n_eval; e += 4) {
    const uint32_t js = *reinterpret_cast<const uint32_t*>(P.j + e);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t x = gen_mismatch(P.x[e + u], (js >> (8 * u)) & 31, a, b);
      if (W == 0) {
        fail |= x;
      } else {
        uint32_t carry = x;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const uint32_t nc = c[w] & carry;
          c[w] ^= carry;
          carry = nc;
        }
        fail |= carry;  // the count passed 2^W - 1 >= k
      }
    }
    if (!__any_sync(__activemask(), ~fail)) return 0;
  }
  if (W > 0) {
    // count >= k + 1 on the W counter bits (needed when k + 1 < 2^W), least significant bit first
    const uint32_t T = P.k + 1u;
    if (T < (1u << W)) {
      uint32_t ge = ~0u;
#pragma unroll
      for (int w = 0; w < W; ++w) ge = ((T >> w) & 1u) ? (c[w] & ge) : (c[w] | ge);
      fail |= ge;
    }
  }
  return ~fail;
}

// candidate windows of P: the exact re-check by set masks (a disagreement sets the status word),
// the invalid-base test (which also rejects windows leaving their record: every record ends in a
// padding base) and the slot append; the same keys as the generated kernels
__device__ __noinline__ void gen_emit(uint32_t h, const GenPattern& P, uint64_t g, uint2 a, uint2 b,
                                      const uint32_t* __restrict__ invalid, uint64_t tile_groups,
                                      uint64_t* __restrict__ slots, uint32_t* __restrict__ tile_count, uint32_t cap,
                                      uint32_t* status) {
  const uint64_t tile = g / tile_groups, tile_pos = tile * tile_groups * 32ull;
  const uint64_t lo64 = (uint64_t)a.x | ((uint64_t)b.x << 32), hi64 = (uint64_t)a.y | ((uint64_t)b.y << 32);
  const uint64_t inv64 = (uint64_t)invalid[g] | ((uint64_t)invalid[g + 1] << 32);
  const uint32_t wm = P.len == 32 ? 0xffffffffu : ((1u << P.len) - 1u);
  while (h) {
    const int i = __ffs(h) - 1;
    h &= h - 1;
    const uint32_t wl = (uint32_t)(lo64 >> i), wh = (uint32_t)(hi64 >> i);
    const uint32_t match = (~wl & ~wh & P.mset[0]) | (wl & ~wh & P.mset[1]) | (~wl & wh & P.mset[2]) |
                           (wl & wh & P.mset[3]);
    const uint32_t mis = ~match & wm;
    const int mism = __popc(mis);
    if ((mis & P.clamp_mask) || mism > P.k) {
      atomicOr(status, (uint32_t)ST_SCAN_MISMATCH);
      continue;
    }
    if ((uint32_t)(inv64 >> i) & wm) continue;
    const uint64_t pos = g * 32ull + (uint64_t)i;
    const uint64_t key =
        ((uint64_t)P.pair << 48) | ((pos - tile_pos) << 16) | ((uint64_t)P.orient << 8) | (uint64_t)mism;
    const uint32_t idx = atomicAdd(tile_count + tile, 1u);
    if (idx < cap) slots[tile * (uint64_t)cap + idx] = key;
  }
}

// one CTA per tile of blockDim.x * gpt groups (the tiles of the slot lists); the pattern table is
// staged in shared memory; every thread takes gpt groups and tests each against every pattern
__global__ void k_scan_generic(const uint2* __restrict__ planes, const uint32_t* __restrict__ invalid,
                               uint64_t group_begin, uint64_t n_groups, const GenPattern* __restrict__ pats,
                               int n_pats, int gpt, uint64_t tile_groups, uint64_t* __restrict__ slots,
                               uint32_t* __restrict__ tile_count, uint32_t cap, uint32_t* status) {
  extern __shared__ uint4 gen_sm[];
  const GenPattern* sp = reinterpret_cast<const GenPattern*>(gen_sm);
  const uint4* src = reinterpret_cast<const uint4*>(pats);
  const int words = n_pats * (int)(sizeof(GenPattern) / sizeof(uint4));
  for (int i = threadIdx.x; i < words; i += blockDim.x) gen_sm[i] = src[i];
  __syncthreads();
  const uint64_t first = (uint64_t)blockIdx.x * blockDim.x * gpt;
  for (int it = 0; it < gpt; ++it) {
    const uint64_t gl = first + (uint64_t)it * blockDim.x + threadIdx.x;
    if (gl >= n_groups) return;
    const uint64_t g = group_begin + gl;
    const uint2 a = __ldg(planes + g), b = __ldg(planes + g + 1);
    for (int q = 0; q < n_pats; ++q) {
      const GenPattern& P = sp[q];
      uint32_t h;
      switch (P.width) {
        case 0: h = gen_pass<0>(P, a, b); break;
        case 1: h = gen_pass<1>(P, a, b); break;
        case 2: h = gen_pass<2>(P, a, b); break;
        case 3: h = gen_pass<3>(P, a, b); break;
        default: h = gen_pass<4>(P, a, b);
      }
      if (h) gen_emit(h, P, g, a, b, invalid, tile_groups, slots, tile_count, cap, status);
    }
  }
}

}  // namespace

std::vector<GenPattern> gen_table(const std::vector<Pattern>& pats) {
  std::vector<GenPattern> out(pats.size());
  for (size_t q = 0; q < pats.size(); ++q) {
    const Pattern& P = pats[q];
    GenPattern& G = out[q];
    G = GenPattern{};
    G.len = P.len;
    G.k = P.k;
    G.pair = (uint16_t)(P.id / 4);
    G.orient = (uint8_t)(P.id % 4);
    G.width = 0;
    while ((1u << G.width) < P.k + 1u) G.width++;
    for (int j = 0; j < P.len; ++j) {
      for (int c = 0; c < 4; ++c)
        if ((P.set[j] >> c) & 1) G.mset[c] |= 1u << j;
      if (j >= P.clamp_lo && j < P.clamp_hi) G.clamp_mask |= 1u << j;
    }
    // evaluated positions: the clamp, then the counted ones by falling mismatch probability on
    // uniform bases (fewer bases in the set first); N never mismatches and is left out
    std::vector<int> clamp, counted;
    for (int j = 0; j < P.len; ++j) {
      if (P.set[j] == 0xF) continue;
      (j >= P.clamp_lo && j < P.clamp_hi ? clamp : counted).push_back(j);
    }
    std::stable_sort(counted.begin(), counted.end(),
                     [&](int a, int b) { return __builtin_popcount(P.set[a]) < __builtin_popcount(P.set[b]); });
    // sections padded to multiples of 4 entries (-1: padding, x = 0, j = 0)
    while (clamp.size() % 4) clamp.push_back(-1);
    while (counted.size() % 4) counted.push_back(-1);
    G.n_clamp = (uint8_t)clamp.size();
    clamp.insert(clamp.end(), counted.begin(), counted.end());
    G.n_eval = (uint8_t)clamp.size();
    for (size_t e = 0; e < clamp.size(); ++e) {
      const int j = clamp[e];
      if (j < 0) continue;
      const uint8_t S = P.set[j];
      // mismatch bit at codes A (lo 0, hi 0), C (1, 0), T (0, 1), G (1, 1) and its algebraic normal form
      const uint32_t fA = (S & 1) ? 0u : ~0u, fC = (S & 2) ? 0u : ~0u, fT = (S & 4) ? 0u : ~0u, fG = (S & 8) ? 0u : ~0u;
      G.x[e] = make_uint4(fA, fA ^ fC, fA ^ fT, fA ^ fC ^ fT ^ fG);
      G.j[e] = (uint8_t)j;
    }
  }
  return out;
}

void launch_scan_kernel(cudaStream_t s, const ScanKernel& k, const ah_batch* b, uint64_t* slots, uint32_t* tile_count,
                        uint32_t cap, uint32_t* status, unsigned long long* work, uint64_t n_tiles, int grid) {
  // whole batch, tiles of threads * groups_per_thread groups; grid > 0 selects the persistent form
  const uint64_t tg = (uint64_t)k.threads * k.groups_per_thread;
  ScanParamsHost P{b->planes, b->invalid, b->rec_group, b->rec_len, b->n_records, cap, 0, b->n_groups,
                   slots, tile_count, status, tg, work, n_tiles};
  void* args[] = {&P};
  cudaLaunchKernel((const void*)k.fn, dim3((unsigned)(grid > 0 ? grid : n_tiles)), dim3((unsigned)k.threads), args, 0, s);
}

void launch_scan_range(cudaStream_t s, const ScanKernel& k, const ah_batch* b, uint64_t* slots, uint32_t* tile_count,
                       uint32_t cap, uint32_t* status, uint64_t g0, uint64_t g1) {
  const uint64_t tg = (uint64_t)k.threads * k.groups_per_thread;
  if (g1 <= g0) return;
  ScanParamsHost P{b->planes, b->invalid, b->rec_group, b->rec_len, b->n_records, cap, g0, g1 - g0,
                   slots, tile_count, status, tg, nullptr, 0};
  void* args[] = {&P};
  cudaLaunchKernel((const void*)k.fn, dim3((unsigned)((g1 - g0 + tg - 1) / tg)), dim3((unsigned)k.threads), args, 0, s);
}

void launch_tile_max(cudaStream_t s, const uint32_t* tile_count, uint64_t n_tiles, uint32_t* out) {
  k_tile_max<<<std::max<uint64_t>(1, std::min<uint64_t>(1024, (n_tiles + 255) / 256)), 256, 0, s>>>(tile_count, n_tiles,
                                                                                                     out);
}

// sort every tile's keys and count them per pair; `big` (n_tiles + 1 words) is needed only when
// cap > kSmallTile
int launch_tile_sort(cudaStream_t s, uint64_t* slots, const uint32_t* tile_count, uint32_t cap, uint64_t n_tiles,
                     uint32_t n_pairs, uint32_t* tpc, uint32_t* big, int sm_count) {
  if (cap > kSmallTile) cudaMemsetAsync(big, 0, sizeof(uint32_t), s);
  k_tile_sort<<<(unsigned)((n_tiles + 7) / 8), 256, 0, s>>>(slots, tile_count, cap, n_tiles, n_pairs, tpc, big);
  if (cap <= kSmallTile) return 1;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, 4ull * (uint64_t)std::max(1, sm_count)));
  k_tile_sort_big<<<grid, kBigSortThreads, 0, s>>>(slots, tile_count, cap, n_tiles, n_pairs, tpc, big);
  return 2;
}

void launch_emit_hits(cudaStream_t s, const uint64_t* slots, const uint32_t* tile_count, uint32_t cap, uint64_t n_tiles,
                      uint64_t tile_groups, const uint64_t* off, const ah_batch* b, ah_hit* hits,
                      const uint64_t* tile_base, uint64_t hit_cap, uint32_t* overflow, uint64_t* pair_off,
                      uint32_t n_pairs) {
  k_emit_hits<<<(unsigned)((n_tiles + 7) / 8), 256, 0, s>>>(slots, tile_count, cap, n_tiles, tile_groups, off,
                                                            b->rec_group, b->n_records, hits, tile_base, hit_cap, overflow);
  k_pair_offsets<<<(n_pairs + 256) / 256, 256, 0, s>>>(off, n_tiles, n_pairs, pair_off);
}

namespace {

// generic-kernel chunks while a compile runs: about this many base-patterns each (a few ms), so
// the switch to the generated kernels comes soon after the compile ends
constexpr double kGenericChunkWork = 4.0e9;

// the generic kernel over tiles [t_begin, t_end), at most kGenMaxPatterns patterns per launch
ah_status enqueue_generic(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ScanConfig& cfg,
                          uint64_t tile_groups, uint64_t t_begin, uint64_t t_end, uint64_t* slots,
                          uint32_t* tile_count, uint32_t cap) {
  const size_t Q = p->pats.size();
  for (size_t q0 = 0; q0 < Q; q0 += kGenMaxPatterns) {
    const int nq = (int)std::min<size_t>(kGenMaxPatterns, Q - q0);
    for (uint64_t t0 = t_begin; t0 < t_end; t0 += 0x7fffffffull) {
      const uint64_t nt = std::min<uint64_t>(0x7fffffffull, t_end - t0);
      const uint64_t g0 = t0 * tile_groups;
      const uint64_t ng = std::min<uint64_t>(b->n_groups - std::min(b->n_groups, g0), nt * tile_groups);
      if (ng == 0) continue;
      k_scan_generic<<<(unsigned)nt, cfg.threads, nq * sizeof(GenPattern), ctx->stream>>>(
          b->planes, b->invalid, g0, ng, p->d_gen + q0, nq, cfg.groups_per_thread, tile_groups, slots, tile_count, cap,
          ctx->d_status);
      const cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) return fail(ctx, AH_ECUDA, "generic scan launch failed: %s", cudaGetErrorString(le));
      launched(ctx);
    }
  }
  return AH_OK;
}

// persistent grid: resident CTAs per SM x SMs
int persistent_grid(ah_ctx* ctx, const ScanKernel& k) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k.fn, k.threads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * ctx->sm_count;
}

// start compiling the generated kernels of `sets` on a thread of the context; returns the flag the
// compile sets (1 compiled, 2 failed: the scan that needs them then compiles again and reports)
std::shared_ptr<std::atomic<int>> start_compile(ah_ctx* ctx, const std::vector<std::vector<Pattern>>& sets,
                                                const ScanConfig& cfg) {
  auto flag = std::make_shared<std::atomic<int>>(0);
  const int device = ctx->device;
  std::lock_guard<std::mutex> lock(ctx->compile_mu);
  for (auto it = ctx->compiles.begin(); it != ctx->compiles.end();) {
    if (it->second->load() != 0) {
      it->first.join();
      it = ctx->compiles.erase(it);
    } else {
      ++it;
    }
  }
  ctx->compiles.emplace_back(
      std::thread([ctx, device, sets, cfg, flag] {
        flag->store(JitCache::global().prefetch(device, ctx, sets, cfg) ? 2 : 1);
      }),
      flag);
  return flag;
}

// the generated kernels over tiles [t_begin, t_end), one after another
ah_status enqueue_jit(ah_ctx* ctx, const ah_batch* b, const std::vector<ScanKernel>& kerns, const ScanConfig& cfg,
                      uint64_t tile_groups, uint64_t t_begin, uint64_t t_end, uint64_t* slots, uint32_t* tile_count,
                      uint32_t cap, unsigned long long* work) {
  for (const ScanKernel& kern : kerns) {
    for (uint64_t t0 = t_begin; t0 < t_end; t0 += 0x7fffffffull) {
      const uint64_t nt = std::min<uint64_t>(0x7fffffffull, t_end - t0);
      const uint64_t g0 = t0 * tile_groups;
      if (cfg.persistent) AH_CUDA(ctx, cudaMemsetAsync(work, 0, sizeof *work, ctx->stream));
      ScanParamsHost P{b->planes, b->invalid, b->rec_group, b->rec_len, b->n_records, cap, g0,
                       std::min<uint64_t>(b->n_groups - std::min(b->n_groups, g0), nt * tile_groups),
                       slots, tile_count, ctx->d_status, tile_groups, work, nt};
      void* args[] = {&P};
      const unsigned grid =
          cfg.persistent ? (unsigned)std::min<uint64_t>(nt, persistent_grid(ctx, kern)) : (unsigned)nt;
      cudaError_t le = cudaLaunchKernel((const void*)kern.fn, dim3(grid), dim3((unsigned)cfg.threads), args, 0,
                                        ctx->stream);
      if (le != cudaSuccess) return fail(ctx, AH_ECUDA, "scan kernel launch failed: %s", cudaGetErrorString(le));
      launched(ctx);
    }
  }
  return AH_OK;
}

// generic-kernel chunks over the leading tiles until *flag turns nonzero (at most two chunks in
// flight; the flag is read as each completes); returns the first tile left
ah_status generic_until(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ScanConfig& cfg,
                        uint64_t tile_groups, uint64_t n_tiles, uint64_t* slots, uint32_t* tile_count, uint32_t cap,
                        const std::atomic<int>& flag, uint64_t* t_out) {
  const double per_tile = (double)tile_groups * 32.0 * (double)std::max<size_t>(1, p->pats.size());
  const uint64_t chunk = std::max<uint64_t>(2ull * std::max(1, ctx->sm_count), (uint64_t)(kGenericChunkWork / per_tile));
  cudaEvent_t done[2] = {nullptr, nullptr};
  ah_status st = AH_OK;
  for (auto& e : done)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming | cudaEventBlockingSync) != cudaSuccess)
      st = fail(ctx, AH_ECUDA, "cudaEventCreate failed");
  uint64_t t = 0;
  int issued = 0;
  while (!st && t < n_tiles && flag.load() == 0) {
    if (issued >= 2) {
      cudaEventSynchronize(done[issued % 2]);
      if (flag.load() != 0) break;
    }
    const uint64_t nt = std::min<uint64_t>(chunk, n_tiles - t);
    if ((st = enqueue_generic(ctx, b, p, cfg, tile_groups, t, t + nt, slots, tile_count, cap))) break;
    cudaEventRecord(done[issued % 2], ctx->stream);
    issued++;
    t += nt;
  }
  for (auto& e : done)
    if (e) cudaEventDestroy(e);
  *t_out = t;
  return st;
}

// Launch the scan over the batch.  per_record: one launch per record and pair (the plain form),
// otherwise one launch over everything (grid of tiles, or persistent CTAs).
ah_status launch_scan(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ScanConfig& cfg, bool per_record,
                      uint64_t tile_groups, uint64_t n_tiles, uint64_t* slots, uint32_t* tile_count, uint32_t cap) {
  ah_status st = AH_OK;
  if (!per_record) {
    // one kernel for every pair, or (cfg.pairs_per_kernel) kernels of a few pairs each, compiled in
    // parallel and launched one after another into the same tile slot lists
    const std::vector<std::vector<Pattern>> sets = scan_groups(p->pats, cfg);
    // generic kernel: over the whole batch (mode 1), or (mode 2, generated kernels not compiled)
    // over leading tiles while a thread of the context compiles them; the scan does not wait for
    // a compile the generic kernel outlasts
    const bool generic_all = ctx->generic_scan == 1;
    std::shared_ptr<std::atomic<int>> flag;
    if (ctx->generic_scan == 2 && !ctx->jit->ready(ctx->device, sets, cfg)) flag = start_compile(ctx, sets, cfg);
    if (ctx->timing) AH_CUDA(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
    uint64_t t = 0;
    if (generic_all) {
      st = enqueue_generic(ctx, b, p, cfg, tile_groups, 0, n_tiles, slots, tile_count, cap);
      t = n_tiles;
    } else if (ctx->generic_scan == 3) {  // the hand-over at a fixed tile
      t = n_tiles / 2;
      if (t) st = enqueue_generic(ctx, b, p, cfg, tile_groups, 0, t, slots, tile_count, cap);
    } else if (flag) {
      st = generic_until(ctx, b, p, cfg, tile_groups, n_tiles, slots, tile_count, cap, *flag, &t);
    }
    if (t > 0) {
      ctx->n_generic_scans++;
      ctx->generic_bases += std::min<uint64_t>(b->n_bases, std::min<uint64_t>(b->n_groups, t * tile_groups) * 32ull);
    }
    int ops = 0;
    unsigned long long* work = nullptr;
    if (!st && t < n_tiles) {
      std::vector<ScanKernel> kerns;
      st = ctx->jit->get_many(ctx, sets, cfg, &kerns);
      if (!st && cfg.persistent) st = dalloc(ctx, &work, 1);
      if (!st) st = enqueue_jit(ctx, b, kerns, cfg, tile_groups, t, n_tiles, slots, tile_count, cap, work);
      for (const ScanKernel& kern : kerns) ops += kern.alu_ops_per_group;
    }
    if (st) {
      dfree(ctx, work);
      return st;
    }
    if (ctx->timing) AH_CUDA(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
    ctx->n_scan_launches++;          // passes over the batch
    ctx->scan_ops_per_group = ops;   // generated circuits of all patterns per 32 positions (0: generic only)
    dfree(ctx, work);
    ctx->scan_bases += b->n_bases;
    return AH_OK;
  }
  // one launch per record per pair, each with the pair's four oriented patterns
  const uint64_t blk_groups = (uint64_t)cfg.threads * cfg.groups_per_thread;
  if (ctx->timing) AH_CUDA(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
  for (uint32_t pair = 0; pair < p->n_pairs; ++pair) {
    std::vector<Pattern> pats(p->pats.begin() + 4 * pair, p->pats.begin() + 4 * pair + 4);
    ScanKernel kern;
    if ((st = ctx->jit->get(ctx, pats, cfg, &kern))) return st;
    for (uint32_t r = 0; r < b->n_records; ++r) {
      const uint64_t g0 = b->h_rec_group[r];
      const uint64_t ng = record_groups(b->h_rec_len[r]);
      ScanParamsHost P{b->planes, b->invalid, b->rec_group, b->rec_len, b->n_records, cap, g0, ng,
                       slots, tile_count, ctx->d_status, tile_groups, nullptr, 0};
      void* args[] = {&P};
      cudaError_t le = cudaLaunchKernel((const void*)kern.fn, dim3((unsigned)((ng + blk_groups - 1) / blk_groups)),
                                        dim3((unsigned)cfg.threads), args, 0, ctx->stream);
      if (le != cudaSuccess) return fail(ctx, AH_ECUDA, "scan kernel launch failed: %s", cudaGetErrorString(le));
      launched(ctx);
      ctx->n_scan_launches++;
    }
  }
  if (ctx->timing) AH_CUDA(ctx, cudaEventRecord(ctx->ev[1], ctx->stream));
  ctx->scan_bases += b->n_bases * p->n_pairs;
  return AH_OK;
}

// scan, then sort / count / place the sites; shared by the one-launch and per-record forms
ah_status scan_sites(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, bool per_record, ah_hits** out) {
  *out = nullptr;
  ScanConfig cfg = ctx->scan_cfg;
  const uint32_t n_pairs = p->n_pairs;
  ah_status st;
  uint64_t* slots = nullptr;
  uint32_t* tile_count = nullptr;
  uint32_t* d_max = nullptr;
  if ((st = dalloc(ctx, &d_max, 1))) return st;
  uint64_t n_tiles = 0, tile_groups = 0;
  uint32_t cap = (uint32_t)cfg.slot_cap;
  for (;;) {
    tile_groups = (uint64_t)cfg.threads * cfg.groups_per_thread;
    n_tiles = std::max<uint64_t>(1, (b->n_groups + tile_groups - 1) / tile_groups);
    if ((st = dalloc(ctx, &slots, n_tiles * cap))) break;
    if ((st = dalloc(ctx, &tile_count, n_tiles))) break;
    AH_CUDA(ctx, cudaMemsetAsync(tile_count, 0, n_tiles * sizeof(uint32_t), ctx->stream));
    AH_CUDA(ctx, cudaMemsetAsync(d_max, 0, sizeof(uint32_t), ctx->stream));
    if ((st = launch_scan(ctx, b, p, cfg, per_record, tile_groups, n_tiles, slots, tile_count, cap))) break;
    launch_tile_max(ctx->stream, tile_count, n_tiles, d_max);
    launched(ctx);
    AH_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, d_max, 4, cudaMemcpyDeviceToHost, ctx->stream));
    AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const uint32_t mx = *ctx->h_status;
    *ctx->h_status = 0;
    if (ctx->timing) {
      float ms = 0.f;
      AH_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
      ctx->scan_ms += ms;
    }
    if (mx <= cap) break;
    // a tile overflowed: retry with room for the fullest tile, shrinking tiles when that is large
    dfree(ctx, slots);
    dfree(ctx, tile_count);
    slots = nullptr;
    tile_count = nullptr;
    uint32_t need = 1;
    while (need < mx) need <<= 1;
    if (need <= 4096) {
      cap = need;
    } else {
      cap = 4096;
      if (cfg.groups_per_thread > 1) cfg.groups_per_thread = 1;
      else if (cfg.threads > 64) cfg.threads /= 2;
      else return fail(ctx, AH_EOVERFLOW, "scan: more than %u sites in a tile of %d groups", mx, cfg.threads);
    }
  }
  if (st) {
    dfree(ctx, slots);
    dfree(ctx, tile_count);
    dfree(ctx, d_max);
    return st;
  }
  // sort each tile, count per (pair, tile)
  uint32_t* tpc = nullptr;
  uint64_t* off = nullptr;
  const uint64_t n_cells = (uint64_t)n_pairs * n_tiles;
  if ((st = dalloc(ctx, &tpc, n_cells))) return st;
  if ((st = dalloc(ctx, &off, n_cells + 1))) return st;
  AH_CUDA(ctx, cudaMemsetAsync(tpc, 0, n_cells * sizeof(uint32_t), ctx->stream));
  uint32_t* big = nullptr;  // tiles with more than 256 keys, sorted by the large-buffer kernel
  if (cap > 256 && (st = dalloc(ctx, &big, n_tiles + 1))) return st;
  const int sorts = launch_tile_sort(ctx->stream, slots, tile_count, cap, n_tiles, n_pairs, tpc, big, ctx->sm_count);
  for (int i = 0; i < sorts; ++i) launched(ctx);
  AH_CUDA(ctx, cudaGetLastError());
  dfree(ctx, big);
  if ((st = exclusive_scan_u32(ctx, tpc, off, n_cells))) return st;
  uint64_t total = 0;
  if ((st = read_u64(ctx, off + n_cells, &total))) return st;
  ah_hits* h = new ah_hits();
  h->ctx = ctx;
  h->n = total;
  h->n_pairs = n_pairs;
  if ((st = dalloc(ctx, &h->d, total)) || (st = dalloc(ctx, &h->d_pair_off, n_pairs + 1))) {
    ah_hits_free(h);
    return st;
  }
  launch_emit_hits(ctx->stream, slots, tile_count, cap, n_tiles, tile_groups, off, b, h->d, nullptr, ~0ull, nullptr,
                   h->d_pair_off, n_pairs);
  launched(ctx, 2);
  AH_CUDA(ctx, cudaGetLastError());
  h->h_pair_off.resize(n_pairs + 1);
  AH_CUDA(ctx, cudaMemcpyAsync(h->h_pair_off.data(), h->d_pair_off, (n_pairs + 1) * sizeof(uint64_t),
                               cudaMemcpyDeviceToHost, ctx->stream));
  dfree(ctx, slots);
  dfree(ctx, tile_count);
  dfree(ctx, d_max);
  dfree(ctx, tpc);
  dfree(ctx, off);
  if ((st = check_status(ctx))) {
    ah_hits_free(h);
    return st;
  }
  *out = h;
  return AH_OK;
}

}  // namespace

ah_status scan_primers(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out) {
  return scan_sites(ctx, b, p, false, out);
}

ah_status scan_primers_per_record(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out) {
  return scan_sites(ctx, b, p, true, out);
}

}  // namespace ah
