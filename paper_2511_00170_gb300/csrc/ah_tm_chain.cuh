// Degenerate-site Tm over every concrete variant of a primer (the default reading), one thread per
// site: the parts shared by the kernel built into the library and the kernels generated per primer
// set at run time (Section "Implementations": Tm_NN in double precision; Section "Primer
// degeneracy": Tm over a primer's variants).
//
// Tm + 273.15 = N(v) / D(v) is a ratio of sums of nearest-neighbour terms, each term depending on at
// most two adjacent bases of the variant v, so the variants form a chain.  Its maximum is found
// exactly by Dinkelbach's iteration for fractional programmes, each step a Viterbi pass over the
// chain that maximises A dS - B dH in integer (or fixed-point) arithmetic over exact sums in tenths.
// A chain type C supplies the passes:
//   int weights(const TmTabs&, int32_t* W, int ws) const      -- per-site weights into W (stride ws);
//                                                                returns a bound on every variant's dS
//   template <typename S> bool pass(const TmTabs&, const int32_t* W, int ws, S A, S B, S* best,
//                                   int32_t* bsum) const      -- best score and that variant's sums
// The kernel built into the library walks any primer's chain from position masks; the generated
// ones are straight-line code for one primer set's chains.
//
// This file includes nothing and opens no namespace: the library includes it inside its own
// namespace, and the run-time compiler receives its text after definitions of the fixed-width
// integer types, uint2/uint4 (built in) and ah_hit.

// Packed sums: dH * 65536 + dS in tenths; every parameter has one decimal, so sums are exact.
constexpr int32_t kNoEdge = -2147483647 - 1;  // a transition without a parameter
// An amplicon writes this word (a NaN no Tm computation returns) into hit_tm at its two sites over
// an array cleared to zero, and the Tm kernels take only the marked sites.
constexpr unsigned long long kSiteWanted = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ int unpack_ds(int32_t p) { return (int16_t)(p & 0xffff); }
__device__ __forceinline__ int unpack_dh(int32_t p) { return (p - unpack_ds(p)) >> 16; }
__device__ __forceinline__ int32_t add_packed(int32_t p, int32_t q) {
  return (p == kNoEdge || q == kNoEdge) ? kNoEdge : p + q;
}

template <typename T>
__device__ __forceinline__ T no_score();
template <>
__device__ __forceinline__ float no_score<float>() { return -__int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double no_score<double>() { return -__longlong_as_double(0x7ff0000000000000ll); }
template <>
__device__ __forceinline__ long long no_score<long long>() { return -9223372036854775807ll - 1; }
template <>
__device__ __forceinline__ int no_score<int>() { return -2147483647 - 1; }

// Run constants computed once on the host.
struct TmRun {
  double rlnk;        // R ln(C)
  double ln_mon;      // ln of the monovalent-equivalent concentration (M)
  double corr_const;  // methods 1-4: Tm correction
  // methods 6 and 7: correction to 1/Tm, rc0 + rc1 f + rc2 / (2 (L - 1)) with f the G/C fraction
  double rc0, rc1, rc2;
  double sym_h, sym_s;  // self-complementary duplexes: the set's symmetry terms (else 0)
  double h0, s0;      // the duplex-wide initiation terms of a duplex holding G or C, plus symmetry
  // the nearest-neighbour set's initiation terms (kcal/mol, cal/(K mol)): every duplex; per
  // terminal A.T and G.C pair of the written strand; a duplex with some / no G or C; each of a 5' T
  // and a 3' A of the written strand
  double init_h, init_s, at_h, at_s, gc_h, gc_s, onegc_h, onegc_s, allat_h, allat_s, t5a_h, t5a_s;
  // the same end terms packed in tenths (dH * 65536 + dS) per variant base (A, C, T, G) at the
  // 5' end (end_l) and the 3' end (end_r)
  int32_t end_l[4], end_r[4];
  int saltcorr;
  int variants;       // 1: degenerate site Tm over the variants matching the site only
  int nn;             // the set's slot in the device tables
  int gc_split;       // 1: the set's initiation differs between duplexes with and without G or C
};

constexpr int kTmThreads = 128;
constexpr int kTmSlots = 8 * kTmThreads;  // site slots per block
constexpr int kTmBins = 256;              // primer bins of the counting sort (a multiple of 32)

// Packed parameters laid out so that for the two opposite-strand codes of an edge its 16 entries
// (the variant's two bases x, y) are one row: step[(c0 4 + c1) 16 + x 4 + y] for edge i (c0, c1 at
// i, i + 1); term_l[(c1 4 + c0) 16 + y 4 + x] for the left end read from the other strand;
// term_r[(c0 4 + c1) 16 + x 4 + y] for the right end; kNoEdge without a parameter.  row_ds[r]: the
// largest dS of step row r over its defined entries (a bound for steps read in place).
struct TmTabs {
  int32_t step[256], term_l[256], term_r[256];
  int32_t row_ds[16];
};
constexpr int kTmTabWords = (int)(sizeof(TmTabs) / 4);

// the row of edge i (codes c0 at i, c1 at i + 1 of the opposite strand, cc 2 bits per position)
__device__ __forceinline__ int row_of(uint64_t cc, int i) {
  return (int)(((cc >> (2 * i)) & 3u) * 4 + ((cc >> (2 * i + 2)) & 3u)) * 16;
}

// packed sums of edge i with variant bases x, y: the terminal-mismatch entry replaces the stack at
// either end
__device__ __forceinline__ int32_t edge_tab(const TmTabs& T, int i, int L, int x, int y, uint64_t cc) {
  const int c0 = (int)(cc >> (2 * i)) & 3, c1 = (int)(cc >> (2 * i + 2)) & 3;
  const int row = (c0 * 4 + c1) * 16;
  if (i == 0) {
    const int32_t p = T.term_l[(c1 * 4 + c0) * 16 + y * 4 + x];
    if (p != kNoEdge) return p;
  }
  if (i == L - 2) {
    const int32_t p = T.term_r[row + x * 4 + y];
    if (p != kNoEdge) return p;
  }
  return T.step[row + x * 4 + y];
}

// the primer as four position masks, one per base code (bit j: position j allows the code)
struct PrimerMasks {
  uint32_t m[4];
  __device__ __forceinline__ uint32_t ch(int j) const {
    return ((m[0] >> j) & 1u) | (((m[1] >> j) & 1u) << 1) | (((m[2] >> j) & 1u) << 2) | (((m[3] >> j) & 1u) << 3);
  }
  __device__ __forceinline__ int fixed(int j) const {  // the one code of a single-choice position
    return (int)((m[1] >> j) & 1u) + 2 * (int)((m[2] >> j) & 1u) + 3 * (int)((m[3] >> j) & 1u);
  }
  // every variant holds G or C: some position allows only those
  __device__ __forceinline__ bool some_gc(int L) const {
    const uint32_t only_gc = (m[1] | m[3]) & ~(m[0] | m[2]);
    return (L >= 32 ? only_gc : only_gc & ((1u << L) - 1u)) != 0;
  }
  // positions with at least two choices
  __device__ __forceinline__ uint32_t branching(int L) const {
    const uint32_t b = (m[0] & m[1]) | (m[0] & m[2]) | (m[0] & m[3]) | (m[1] & m[2]) | (m[1] & m[3]) | (m[2] & m[3]);
    return L >= 32 ? b : b & ((1u << L) - 1u);
  }
};

// the bits of x at the even positions of a 64-bit word (bit j to bit 2j)
__device__ __forceinline__ uint64_t spread_bits(uint32_t x) {
  uint64_t v = x;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  return (v | (v << 1)) & 0x5555555555555555ull;
}

// the site's bases over [pos, pos + L) (L <= 32 spans at most two plane words), in the primer's
// orientation, 2 bits per position (position j at bits 2j, 2j + 1; nothing past L)
__device__ __forceinline__ uint64_t site_code(const uint2* __restrict__ planes, const uint64_t* __restrict__ rec_group,
                                              const ah_hit& h, int L) {
  const uint64_t x0 = rec_group[h.record] * 32 + h.pos;
  const uint2 w0 = planes[x0 >> 5], w1 = planes[(x0 >> 5) + 1];
  const int sh0 = (int)(x0 & 31);
  uint32_t lo = (uint32_t)(((((uint64_t)w1.x << 32) | w0.x) >> sh0));
  uint32_t hi = (uint32_t)(((((uint64_t)w1.y << 32) | w0.y) >> sh0));
  const uint64_t mask = L >= 32 ? ~0ull : ((1ull << (2 * L)) - 1);
  if ((h.pattern >> 1) & 1u) {  // the reverse strand: reversed and complemented (code ^ 2)
    lo = __brev(lo) >> (32 - L);
    hi = __brev(hi) >> (32 - L);
    return ((spread_bits(lo) | (spread_bits(hi) << 1)) ^ 0xAAAAAAAAAAAAAAAAull) & mask;
  }
  return (spread_bits(lo) | (spread_bits(hi) << 1)) & mask;
}

// Tm of one site over every variant of its primer by the chain method.  Returns false when the chain
// does not apply (salt methods 6 and 7, L < 3, an entropy sum that could reach zero, a ratio beyond
// the fixed-point range): the site is then enumerated variant by variant.
//  - The chain's constant terms assume a duplex holding G or C (some_gc: a position of the primer
//    allows only C and G); where the set's initiation depends on that and the primer does not
//    guarantee it, the site is enumerated.
//  - The sign condition: every variant's entropy sum must stay negative.  The chain's bound is tried
//    first; the exact largest dS is found only when the bound leaves the sign open.
//  - The start pass scores 280 dS - 1000 dH exactly in int32 (|score| < 5e7; the proving passes
//    reach the same optimum from any start, and one below the usual site Tm needed the fewest:
//    on the dense-site workload 280 K ran faster than 300, 315 and 330 K); each proving pass scores
//    lambda dS - 1000 dH in 64-bit fixed point with lambda scaled by 2^s (s = 36 below 4000 K, less
//    beyond, so that products stay below 2^63).  A pass that finds no variant above the incumbent
//    shows it optimal; otherwise the better variant's ratio is the next lambda.
template <class C>
__device__ __forceinline__ bool chain_site_tm(const TmTabs& T, int32_t* __restrict__ W, int ws, const C& chain, int L,
                                              const TmRun& R, bool some_gc, double* tm) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (R.saltcorr >= 6 || L < 3 || (R.gc_split && !some_gc)) return false;
  const int bound = chain.weights(T, W, ws);
  const double S0 = (R.saltcorr == 5 ? 0.368 * (double)(L - 1) * R.ln_mon : 0.0) + R.rlnk;
  const double H0 = R.h0, Sc = R.s0;
  const double shift = R.saltcorr >= 1 && R.saltcorr <= 4 ? R.corr_const : 0.0;
  int32_t bp;
  if (0.1 * bound + Sc + S0 >= 0.0) {  // the bound leaves the sign open: the largest dS itself
    int sc;
    if (!chain.template pass<int>(T, W, ws, 1, 0, &sc, &bp)) {
      *tm = nan;
      return true;
    }
    if (0.1 * unpack_ds(bp) + Sc + S0 >= 0.0) return false;
  }
  {
    int sc;
    if (!chain.template pass<int>(T, W, ws, 280, 1000, &sc, &bp)) {
      *tm = nan;
      return true;
    }
  }
  auto ratio = [&](int32_t p) { return 1000.0 * (0.1 * unpack_dh(p) + H0) / (0.1 * unpack_ds(p) + Sc + S0); };
  double lam = ratio(bp);
  int32_t inc = bp;
  for (int it = 0; it < 64; ++it) {
    int s = 36;
    const double al = fabs(lam);
    if (!(al < 4000.0)) {  // beyond 4000 K fewer fraction bits, the same bound on |lambda| 2^s
      if (!(al < 1.0e12)) return false;
      int e;
      frexp(al / 4000.0, &e);
      s = 36 - e;
    }
    const double scale = ldexp(1.0, s);
    const long long Lq = llrint(lam * scale), Bq = (long long)(1000.0 * scale);
    long long sc;
    int32_t cand;
    if (!chain.template pass<long long>(T, W, ws, Lq, Bq, &sc, &cand)) break;
    if (!(sc > Lq * unpack_ds(inc) - Bq * unpack_dh(inc))) break;
    const double q = ratio(cand);
    if (!(q > lam)) break;
    lam = q, inc = cand;
  }
  *tm = lam + shift - 273.15;
  return true;
}

// The site Tm of every marked site of a launch.  Blocks of kTmThreads threads take windows of
// kTmSlots site slots.  Each thread first settles its slots where that needs no chain (not wanted,
// or a step between two single-choice positions without a parameter: every variant contains it,
// NaN); the rest are sorted by primer and taken in that order, kTmThreads at a time, so the threads
// of a warp share the chain's shape and the warps are full.  Sites the chain does not cover go to
// the list defer (count at defer[0]) for the enumerating kernel.  Shared memory: the tables, the
// window's keys and their order by primer, then each thread's weights, strided by the block size.
// D supplies fill(TmTabs&, const int32_t* image, int slot) and site(pr, T, W, ws, P, code, L, R, &tm).
// Only the sites of primers [pr_lo, pr_hi) are taken; the others are left as they are for another
// launch (a launch per primer keeps one primer's code hot in the instruction cache).
template <class D>
__device__ __forceinline__ void tm_hits_body(const ah_hit* __restrict__ hits, uint64_t n,
                                             const uint2* __restrict__ planes, const uint64_t* __restrict__ rec_group,
                                             const uint8_t* __restrict__ plen, const uint4* __restrict__ pmask,
                                             const TmRun& Rp, double* __restrict__ out, uint32_t* __restrict__ defer,
                                             const uint64_t* __restrict__ d_n, const int32_t* __restrict__ image,
                                             uint32_t pr_lo, uint32_t pr_hi) {
  // the run constants in shared memory: device functions take them by reference, and a reference
  // to a kernel parameter would make the compiler copy it to local memory for every thread
  __shared__ TmRun R_sh;
  __shared__ int n_valid;
  __shared__ uint32_t bins[kTmBins];
  if (threadIdx.x == 0) R_sh = Rp, n_valid = 0;
  const TmRun& R = R_sh;
  extern __shared__ __align__(16) uint32_t tm_smem[];
  TmTabs& T = *reinterpret_cast<TmTabs*>(tm_smem);
  uint32_t* keys = tm_smem + kTmTabWords;
  uint32_t* order = tm_smem + kTmTabWords + kTmSlots;
  int32_t* W = reinterpret_cast<int32_t*>(tm_smem + kTmTabWords + 2 * kTmSlots) + threadIdx.x;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  D::fill(T, image, Rp.nn);
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kTmSlots;
  const uint64_t n_here = d_n && *d_n < n ? *d_n : n;
  int mine = 0;
  for (int t = threadIdx.x; t < kTmSlots; t += kTmThreads) {
    const uint64_t i = base + t;
    uint32_t key = 0xFFFFFFFFu;
    if (i < n_here && (unsigned long long)__double_as_longlong(out[i]) == kSiteWanted) {
      const ah_hit h = hits[i];
      const uint32_t pr = (h.pattern >> 2) * 2 + (h.pattern & 1u);
      if (pr < pr_lo || pr >= pr_hi) {
        keys[t] = key;
        continue;
      }
      const int L = plen[h.pattern];
      const uint64_t code = site_code(planes, rec_group, h, L);
      const uint64_t cc = code ^ 0xAAAAAAAAAAAAAAAAull;
      const uint4 mk = pmask[pr];
      const PrimerMasks P{{mk.x, mk.y, mk.z, mk.w}};
      const uint32_t fixed = ~P.branching(L) & (L >= 32 ? 0xFFFFFFFFu : ((1u << L) - 1u));
      bool undefined = false;
      for (uint32_t f = fixed & (fixed >> 1); f && !undefined; f &= f - 1) {  // steps j, j + 1 both fixed
        const int j = __ffs(f) - 1;
        if (edge_tab(T, j, L, P.fixed(j), P.fixed(j + 1), cc) == kNoEdge) undefined = true;
      }
      if (undefined) {
        out[i] = nan;
      } else {
        key = (pr << 16) | (uint32_t)t;
        ++mine;
      }
    }
    keys[t] = key;
  }
  if (mine) atomicAdd(&n_valid, mine);
  __syncthreads();
  if (n_valid == 0) return;
  // group the sites by primer: a counting sort over the primers (their ids folded into kTmBins
  // bins, which can only mix shapes, never lose a site); order within a primer does not matter
  for (int k = threadIdx.x; k < kTmBins; k += kTmThreads) bins[k] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < kTmSlots; t += kTmThreads)
    if (keys[t] != 0xFFFFFFFFu) atomicAdd(&bins[(keys[t] >> 16) % kTmBins], 1u);
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the bins, kTmBins / 32 per lane
    constexpr int per = kTmBins / 32;
    uint32_t v[per], sum = 0;
    for (int k = 0; k < per; ++k) v[k] = bins[threadIdx.x * per + k], sum += v[k];
    uint32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if ((int)threadIdx.x >= o) x += y;
    }
    uint32_t run = x - sum;
    for (int k = 0; k < per; ++k) bins[threadIdx.x * per + k] = run, run += v[k];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kTmSlots; t += kTmThreads) {
    const uint32_t key = keys[t];
    if (key != 0xFFFFFFFFu) order[atomicAdd(&bins[(key >> 16) % kTmBins], 1u)] = key;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < n_valid; q += kTmThreads) {
    const uint32_t key = order[q];
    const uint32_t t = key & 0xFFFFu, pr = key >> 16;
    const uint64_t i = base + t;
    const ah_hit h = hits[i];
    const int L = plen[h.pattern];
    const uint4 mk = pmask[pr];
    const PrimerMasks P{{mk.x, mk.y, mk.z, mk.w}};
    double tm;
    if (D::site(pr, T, W, kTmThreads, P, site_code(planes, rec_group, h, L), L, R, &tm))
      out[i] = tm;
    else  // the chain does not cover it: listed for the enumerating kernel
      defer[1 + atomicAdd(defer, 1u)] = (uint32_t)i;
  }
}
