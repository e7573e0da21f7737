// Run-time specialisation of the degenerate-site Tm kernel for one primer set (Section
// "Implementations": Tm_NN; Section "Primer degeneracy": Tm over a primer's variants).
//
// The kernel built into the library walks each primer's chain from position masks, so every pass
// tests at run time which of the 16 transitions of each step exist.  With the primer known, the
// chain is fixed and its passes become straight-line code over exactly the transitions that exist.
// The generated chain also regroups the terms.  Let the branch positions (two or more choices) be
// d_0 < ... < d_(n-1).
//  - Where d_(t+1) > d_t + 1, every variant's terms between them split into one term that depends
//    on the choice at d_t, fixed terms, and one term that depends on the choice at d_(t+1).  Each
//    part is added to its branch position's node weight, so such a step costs |A| + |B| rather than
//    |A| x |B|, and the Viterbi chain falls apart into independent segments.
//  - Where d_(t+1) = d_t + 1, the step's weights are read from the parameter table's row for the
//    site's two codes, in place (at the duplex's ends, with the terminal-mismatch rule: stored).
//  - The node weights hold everything else: the ends' initiation terms and the fixed steps.
// Every variant's sums are the same as the built-in chain's, so the result is the same maximum.
// The driver (sign condition, start pass, proving passes) and the kernel body are shared with the
// built-in kernel (ah_tm_chain.cuh).
#include <algorithm>
#include <cctype>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <map>
#include <sstream>

#include "ah_internal.h"

namespace ah {
namespace {

// the text of ah_tm_chain.cuh (a raw string literal written by the build)
const char* kChainHeader =
#include "ah_tm_chain_src.inc"
    ;

const char* kPrelude = R"(
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
struct ah_hit {
  uint32_t record;
  uint32_t pos;
  uint16_t pattern;
  uint8_t mism;
  uint8_t flags;
};
static_assert(sizeof(ah_hit) == 12, "ah_hit layout");
)";

const char* kChainHelpers = R"(
static_assert(sizeof(TmRun) == TM_RUN_BYTES, "TmRun layout");
// the terminal-mismatch entry when the end step has one, else the stack
__device__ __forceinline__ int32_t pick(int32_t p, int32_t q) { return p != kNoEdge ? p : q; }
template <typename S>
__device__ __forceinline__ S score(int32_t p, S A, S B) { return A * (S)unpack_ds(p) - B * (S)unpack_dh(p); }
)";

uint8_t code_set(char ch) {  // IUPAC code to a set over the codes A=0, C=1, T=2, G=3
  switch (ch) {
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
    default: return SET_A | SET_C | SET_G | SET_T;
  }
}

std::vector<int> codes(uint8_t set) {
  std::vector<int> v;
  for (int c = 0; c < 4; ++c)
    if ((set >> c) & 1u) v.push_back(c);
  return v;
}
int only(uint8_t set) { return codes(set)[0]; }

// One primer's chain: branch positions, which steps between them are adjacent, where each node's
// weights and each stored step's weights live in W.
struct Chain {
  int L = 0;
  uint8_t set[32] = {};
  std::vector<int> D;
  std::vector<int> node_slot;  // first slot of node t (one per choice); -1: its weights are literals
  std::vector<std::vector<std::string>> node_lit;  // those weights, one per choice: "0" or an end term
  std::vector<int> edge_slot;  // adjacent steps at the duplex's ends: first slot (|A| x |B|), else -1
  int words = 0;
  bool adjacent(int t) const { return D[t + 1] == D[t] + 1; }
  bool stored(int t) const { return adjacent(t) && (D[t] == 0 || D[t] == L - 2); }
};

Chain make_chain(const std::string& primer) {
  Chain c;
  c.L = (int)primer.size();
  for (int j = 0; j < c.L; ++j) c.set[j] = code_set(primer[j]);
  for (int j = 0; j < c.L; ++j)
    if (__builtin_popcount(c.set[j]) >= 2) c.D.push_back(j);
  if (c.D.empty()) c.D.push_back(0);  // a concrete primer: one node with one choice
  const int n = (int)c.D.size();
  for (int t = 0; t < n; ++t) {
    const int d = c.D[t];
    // a node whose weight holds nothing (no step and no end term) is a literal zero
    bool steps = t == 0 || t == n - 1;
    if (t > 0 && !c.adjacent(t - 1)) steps = true;
    if (t + 1 < n && !c.adjacent(t)) steps = true;
    c.node_lit.emplace_back();
    if (steps) {
      c.node_slot.push_back(c.words);
      c.words += __builtin_popcount(c.set[d]);
      continue;
    }
    c.node_slot.push_back(-1);
    for (int a : codes(c.set[d])) {
      std::string v;
      if (d == 0) v = "R->end_l[" + std::to_string(a) + "]";
      if (d == c.L - 1) v += (v.empty() ? "" : " + ") + std::string("R->end_r[") + std::to_string(a) + "]";
      c.node_lit.back().push_back(v.empty() ? "0" : v);
    }
  }
  for (int t = 0; t + 1 < n; ++t) {
    if (c.stored(t)) {
      c.edge_slot.push_back(c.words);
      c.words += __builtin_popcount(c.set[c.D[t]]) * __builtin_popcount(c.set[c.D[t + 1]]);
    } else {
      c.edge_slot.push_back(-1);
    }
  }
  return c;
}

// packed parameters of edge i for variant bases x (at i) and y (at i + 1); rows r<i> and rl declared
std::string edge_expr(const Chain& c, int i, int x, int y) {
  const std::string st = "T.step[r" + std::to_string(i) + " + " + std::to_string(x * 4 + y) + "]";
  if (i == 0) return "pick(T.term_l[rl + " + std::to_string(y * 4 + x) + "], " + st + ")";
  if (i == c.L - 2) return "pick(T.term_r[r" + std::to_string(i) + " + " + std::to_string(x * 4 + y) + "], " + st + ")";
  return st;
}

std::string rows_decl(const Chain& c, const std::vector<int>& edges, const char* indent) {
  std::ostringstream os;
  for (int i : edges) {
    os << indent << "const int r" << i << " = row_of(cc, " << i << ");\n";
    if (i == 0) os << indent << "const int rl = ((int)((cc >> 2) & 3u) * 4 + (int)(cc & 3u)) * 16;\n";
  }
  return os.str();
}


// struct C<q> { uint64_t cc; weights(); pass<S>(); } for one primer
std::string chain_struct(const Chain& c, int q) {
  std::ostringstream os;
  const int L = c.L, n = (int)c.D.size();
  auto fixed_at = [&](int j) { return only(c.set[j]); };
  os << "struct C" << q << " {  // L = " << L << ", " << n << " branch position(s)\n  uint64_t cc;\n  const TmRun* R;\n";
  if (L < 3) {  // the driver defers these before any pass
    os << "  __device__ __forceinline__ int weights(const TmTabs&, int32_t*, int) const { return 0; }\n";
    os << "  template <typename S> __device__ __forceinline__ bool pass(const TmTabs&, const int32_t*, int, S, S, S*,"
          " int32_t*) const { return false; }\n};\n";
    return os.str();
  }
  // ---- weights
  os << "  __device__ __forceinline__ int weights(const TmTabs& T, int32_t* __restrict__ W, int ws) const {\n";
  {
    std::vector<int> all;
    for (int i = 0; i + 1 < L; ++i) all.push_back(i);
    os << rows_decl(c, all, "    ");
  }
  os << "    int bound = 0;\n";
  for (int t = 0; t < n; ++t) {
    const int d = c.D[t];
    if (c.node_slot[t] < 0) {  // weights without steps: only their part of the bound
      if (c.node_lit[t][0] == "0") continue;
      os << "    {  // node " << t << " at position " << d << " (end terms only)\n      int mx = unpack_ds("
         << c.node_lit[t][0] << ");\n";
      for (size_t k = 1; k < c.node_lit[t].size(); ++k) os << "      mx = max(mx, unpack_ds(" << c.node_lit[t][k] << "));\n";
      os << "      bound += mx;\n    }\n";
      continue;
    }
    // fixed part: ends not at a branch position, fixed steps before the first / after the last
    // branch position and between separated ones
    std::vector<std::string> fixed;
    std::string konst = "0";
    if (t == 0) {
      if (d != 0) konst += " + R->end_l[" + std::to_string(fixed_at(0)) + "]";
      for (int i = 0; i + 2 <= d; ++i) fixed.push_back(edge_expr(c, i, fixed_at(i), fixed_at(i + 1)));
    }
    if (t == n - 1) {
      if (d != L - 1) konst += " + R->end_r[" + std::to_string(fixed_at(L - 1)) + "]";
      for (int i = d + 1; i + 1 < L; ++i) fixed.push_back(edge_expr(c, i, fixed_at(i), fixed_at(i + 1)));
    }
    if (t + 1 < n && !c.adjacent(t))
      for (int i = d + 1; i + 2 <= c.D[t + 1]; ++i) fixed.push_back(edge_expr(c, i, fixed_at(i), fixed_at(i + 1)));
    os << "    {  // node " << t << " at position " << d << "\n      const int32_t f = " << konst;
    for (auto& e : fixed) os << "\n          + " << e;
    os << ";\n      int mx = -2147483647 - 1;\n";
    const std::vector<int> ch = codes(c.set[d]);
    for (size_t k = 0; k < ch.size(); ++k) {
      const int a = ch[k];
      std::string p = "f";
      if (d == 0) p += " + R->end_l[" + std::to_string(a) + "]";
      if (d == L - 1) p += " + R->end_r[" + std::to_string(a) + "]";
      if (d >= 1 && (t == 0 || !c.adjacent(t - 1))) p = "add_packed(" + edge_expr(c, d - 1, fixed_at(d - 1), a) + ", " + p + ")";
      if (d + 1 < L && (t == n - 1 || !c.adjacent(t))) p = "add_packed(" + edge_expr(c, d, a, fixed_at(d + 1)) + ", " + p + ")";
      os << "      { const int32_t p = " << p << ";\n        W[" << (c.node_slot[t] + (int)k)
         << " * ws] = p;\n        if (p != kNoEdge) mx = max(mx, unpack_ds(p)); }\n";
    }
    os << "      bound += mx == -2147483647 - 1 ? 0 : mx;\n    }\n";
  }
  for (int t = 0; t + 1 < n; ++t) {
    if (!c.adjacent(t)) continue;
    const int d = c.D[t];
    if (!c.stored(t)) {
      os << "    bound += T.row_ds[r" << d << " >> 4];  // step " << d << " read in place\n";
      continue;
    }
    os << "    {  // step " << d << " at the duplex's end\n      int mx = -2147483647 - 1;\n";
    const std::vector<int> ca = codes(c.set[d]), cb = codes(c.set[d + 1]);
    int k = c.edge_slot[t];
    for (int a : ca)
      for (int b : cb) {
        os << "      { const int32_t p = " << edge_expr(c, d, a, b) << ";\n        W[" << k++
           << " * ws] = p;\n        if (p != kNoEdge) mx = max(mx, unpack_ds(p)); }\n";
      }
    os << "      bound += mx == -2147483647 - 1 ? 0 : mx;\n    }\n";
  }
  os << "    return bound;\n  }\n";
  // ---- one pass
  os << "  template <typename S>\n  __device__ __forceinline__ bool pass(const TmTabs& T, const int32_t* __restrict__ W, "
        "int ws, S A, S B, S* best, int32_t* bsum) const {\n";
  os << "    const S none = no_score<S>();\n    S tot = 0;\n    int32_t tsum = 0;\n";
  int t = 0;
  while (t < n) {
    int t1 = t;
    while (t1 + 1 < n && c.adjacent(t1)) ++t1;
    os << "    {  // segment of nodes " << t << ".." << t1 << "\n";
    // first node's states
    {
      const std::vector<int> ch = codes(c.set[c.D[t]]);
      for (size_t k = 0; k < ch.size(); ++k) {
        const int a = ch[k];
        os << "      S c" << t << "_" << a << " = none;\n      int32_t s" << t << "_" << a << " = 0;\n";
        if (c.node_slot[t] < 0)
          os << "      c" << t << "_" << a << " = score<S>(" << c.node_lit[t][k] << ", A, B), s" << t << "_" << a
             << " = " << c.node_lit[t][k] << ";\n";
        else
          os << "      { const int32_t p = W[" << (c.node_slot[t] + (int)k) << " * ws]; if (p != kNoEdge) c" << t << "_"
             << a << " = score<S>(p, A, B), s" << t << "_" << a << " = p; }\n";
      }
    }
    for (int u = t + 1; u <= t1; ++u) {
      const int d = c.D[u - 1];
      const std::vector<int> ca = codes(c.set[d]), cb = codes(c.set[c.D[u]]);
      const bool st = c.stored(u - 1);
      if (!st) os << "      const int r" << d << " = row_of(cc, " << d << ");\n";
      for (size_t kb = 0; kb < cb.size(); ++kb) {
        const int b = cb[kb];
        os << "      S c" << u << "_" << b << " = none;\n      int32_t s" << u << "_" << b << " = 0;\n      {\n";
        os << "        S m = none;\n        int32_t ms = 0;\n";
        for (size_t ka = 0; ka < ca.size(); ++ka) {
          const int a = ca[ka];
          std::string e = st ? "W[" + std::to_string(c.edge_slot[u - 1] + (int)(ka * cb.size() + kb)) + " * ws]"
                             : "T.step[r" + std::to_string(d) + " + " + std::to_string(a * 4 + b) + "]";
          os << "        { const int32_t e = " << e << "; if (c" << (u - 1) << "_" << a
             << " != none && e != kNoEdge) { const S v = c" << (u - 1) << "_" << a << " + score<S>(e, A, B); if (v > m) m = v, ms = s"
             << (u - 1) << "_" << a << " + e; } }\n";
        }
        if (c.node_slot[u] < 0) {
          const std::string lit = c.node_lit[u][kb];
          if (lit == "0")
            os << "        if (m != none) c" << u << "_" << b << " = m, s" << u << "_" << b << " = ms;\n      }\n";
          else
            os << "        if (m != none) c" << u << "_" << b << " = m + score<S>(" << lit << ", A, B), s" << u << "_" << b
               << " = ms + " << lit << ";\n      }\n";
        } else {
          os << "        const int32_t p = W[" << (c.node_slot[u] + (int)kb) << " * ws];\n";
          os << "        if (m != none && p != kNoEdge) c" << u << "_" << b << " = m + score<S>(p, A, B), s" << u << "_" << b
             << " = ms + p;\n      }\n";
        }
      }
    }
    os << "      S sb = none;\n      int32_t ss = 0;\n";
    for (int a : codes(c.set[c.D[t1]]))
      os << "      if (c" << t1 << "_" << a << " > sb) sb = c" << t1 << "_" << a << ", ss = s" << t1 << "_" << a << ";\n";
    os << "      if (sb == none) return false;\n      tot += sb;\n      tsum += ss;\n    }\n";
    t = t1 + 1;
  }
  os << "    *best = tot;\n    *bsum = tsum;\n    return true;\n  }\n};\n";
  return os.str();
}

}  // namespace

int tm_chain_adjacent(const std::vector<std::string>& primers) {
  std::map<std::string, int> seen;
  int total = 0;
  for (const std::string& q : primers) {
    if (!seen.emplace(q, 0).second) continue;
    const Chain c = make_chain(q);
    for (int t = 0; t + 1 < (int)c.D.size(); ++t)
      if (c.adjacent(t)) total += __builtin_popcount(c.set[c.D[t]]) * __builtin_popcount(c.set[c.D[t + 1]]);
  }
  return total;
}

std::string tm_chain_source(const std::vector<std::string>& primers, int* weight_words) {
  std::ostringstream os;
  os << "// generated degenerate-site Tm kernel: " << primers.size() << " primer(s)\n";
  os << "#define TM_RUN_BYTES " << tm_run_bytes() << "\n";
  os << kPrelude << kChainHeader << kChainHelpers;
  std::map<std::string, int> distinct;
  std::vector<int> index(primers.size());
  int words = 1;
  for (size_t q = 0; q < primers.size(); ++q) {
    auto it = distinct.find(primers[q]);
    if (it == distinct.end()) {
      const int id = (int)distinct.size();
      distinct.emplace(primers[q], id);
      const Chain c = make_chain(primers[q]);
      words = std::max(words, c.words);
      os << chain_struct(c, id);
      index[q] = id;
    } else {
      index[q] = it->second;
    }
  }
  // one driver for every primer: the chain's two calls switch on the primer (warp-uniform after the
  // kernel's sort), so the driver is compiled once and only the chains per primer
  os << "struct Chains {\n  uint32_t pr;\n  uint64_t cc;\n  const TmRun* R;\n";
  os << "  __device__ __forceinline__ int weights(const TmTabs& T, int32_t* __restrict__ W, int ws) const {\n"
        "    switch (pr) {\n";
  for (size_t q = 0; q < primers.size(); ++q)
    os << "      case " << q << ": return C" << index[q] << "{cc, R}.weights(T, W, ws);\n";
  os << "      default: return 0;\n    }\n  }\n";
  os << "  template <typename S>\n  __device__ __forceinline__ bool pass(const TmTabs& T, const int32_t* __restrict__ W, "
        "int ws, S A, S B, S* best, int32_t* bsum) const {\n    switch (pr) {\n";
  for (size_t q = 0; q < primers.size(); ++q)
    os << "      case " << q << ": return C" << index[q] << "{cc, R}.template pass<S>(T, W, ws, A, B, best, bsum);\n";
  os << "      default: return false;\n    }\n  }\n};\n";
  os << "struct GenSites {\n";
  os << "  static __device__ __forceinline__ void fill(TmTabs& T, const int32_t* __restrict__ image, int) {\n";
  os << "    int32_t* d = reinterpret_cast<int32_t*>(&T);\n";
  os << "    for (int e = threadIdx.x; e < kTmTabWords; e += blockDim.x) d[e] = image[e];\n  }\n";
  os << "  static __device__ __forceinline__ bool site(uint32_t pr, const TmTabs& T, int32_t* __restrict__ W, int ws,\n"
        "                                              const PrimerMasks P, uint64_t code, int L, const TmRun& R,"
        " double* tm) {\n";
  os << "    if (pr >= " << primers.size() << "u) return false;\n";
  os << "    return chain_site_tm(T, W, ws, Chains{pr, code ^ 0xAAAAAAAAAAAAAAAAull, &R}, L, R, P.some_gc(L), tm);\n"
        "  }\n};\n";
  // blocks per SM the register allocation must allow: as many as shared memory holds (228 KB per SM,
  // 1 KB of it reserved per block), from 4 to 8; more resident warps hide the chains' latencies (the
  // 64 registers of 8 blocks cost a few dozen bytes of spills)
  os << "constexpr int kTmJitSmem = 4 * (kTmTabWords + 2 * kTmSlots + " << words
     << " * kTmThreads) + (int)sizeof(TmRun) + 4 + 4 * kTmBins + 1024;\n"
        "constexpr int kTmJitFit = 228 * 1024 / kTmJitSmem;\n"
        "constexpr int kTmJitBlocks = kTmJitFit < 4 ? 4 : kTmJitFit > 8 ? 8 : kTmJitFit;\n";
  os << "extern \"C\" __global__ void __launch_bounds__(kTmThreads, kTmJitBlocks) ah_tm_jit(\n"
        "    const ah_hit* __restrict__ hits, uint64_t n, const uint2* __restrict__ planes,\n"
        "    const uint64_t* __restrict__ rec_group, const uint8_t* __restrict__ plen, const uint4* __restrict__ pmask,\n"
        "    const TmRun Rp, double* __restrict__ out, uint32_t* __restrict__ defer, const uint64_t* __restrict__ d_n,\n"
        "    const int32_t* __restrict__ image, uint32_t pr_lo, uint32_t pr_hi) {\n"
        "  tm_hits_body<GenSites>(hits, n, planes, rec_group, plen, pmask, Rp, out, defer, d_n, image, pr_lo, pr_hi);\n}\n";
  if (weight_words) *weight_words = words;
  return os.str();
}

namespace {

struct TmEntry {
  std::mutex m;
  std::condition_variable cv;
  bool done = false, loaded = false;
  ah_status st = AH_OK;
  std::string err;
  std::vector<char> cubin;
  TmKernel k;
};

std::mutex g_mu;
std::map<std::string, std::shared_ptr<TmEntry>>* g_cache = new std::map<std::string, std::shared_ptr<TmEntry>>();

std::vector<std::string> primer_list(const ah_primers* p) {
  std::vector<std::string> v;
  for (uint32_t q = 0; q < p->n_pairs; ++q) v.push_back(p->fwd[q]), v.push_back(p->rev[q]);
  return v;
}

// compiles (once per source) and, when load_it, loads the kernel; err filled on failure
ah_status get_kernel(int device, ah_ctx* stats, const std::vector<std::string>& primers, bool load_it, TmKernel* out,
                     std::string* err) {
  int words = 0;
  const std::string src = tm_chain_source(primers, &words);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  const std::string key = std::to_string(major * 10 + minor) + "\n" + src;
  std::shared_ptr<TmEntry> e;
  bool mine = false;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache->find(key);
    if (it == g_cache->end()) {
      e = std::make_shared<TmEntry>();
      g_cache->emplace(key, e);
      mine = true;
    } else {
      e = it->second;
    }
  }
  if (mine) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<char> cubin;
    std::string cerr;
    const ah_status st = nvrtc_compile(device, src, "ah_tm_jit.cu", &cubin, &cerr);
    {
      std::lock_guard<std::mutex> lock(e->m);
      e->st = st;
      e->err = cerr;
      e->cubin.swap(cubin);
      e->k.weight_words = words;
      e->done = true;
    }
    e->cv.notify_all();
    if (st) {
      std::lock_guard<std::mutex> lock(g_mu);
      g_cache->erase(key);
    } else if (stats) {
      std::lock_guard<std::mutex> lock(stats->stats_mu);
      stats->jit_compiles++;
      stats->jit_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
  }
  std::unique_lock<std::mutex> lock(e->m);
  e->cv.wait(lock, [&] { return e->done; });
  if (e->st) {
    *err = e->err;
    return e->st;
  }
  if (!load_it) return AH_OK;
  if (!e->loaded) {
    cudaSetDevice(device);
    cudaLibrary_t lib;
    cudaError_t ce = cudaLibraryLoadData(&lib, e->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (ce == cudaSuccess) ce = cudaLibraryGetKernel(&e->k.fn, lib, "ah_tm_jit");
    if (ce != cudaSuccess) {
      *err = std::string("loading the generated Tm kernel failed: ") + cudaGetErrorString(ce);
      return AH_EJIT;
    }
    e->loaded = true;
    std::vector<char>().swap(e->cubin);
  }
  *out = e->k;
  return AH_OK;
}

enum Lookup { kAbsent, kBusy, kReady };

// the kernel if it is compiled (loading it into the process here when it was compiled elsewhere)
Lookup lookup(int device, const std::vector<std::string>& primers, TmKernel* out) {
  const std::string src = tm_chain_source(primers, nullptr);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  const std::string key = std::to_string(major * 10 + minor) + "\n" + src;
  std::shared_ptr<TmEntry> e;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache->find(key);
    if (it == g_cache->end()) return kAbsent;
    e = it->second;
  }
  {
    std::lock_guard<std::mutex> lock(e->m);
    if (!e->done || e->st) return kBusy;  // a failed compile is dropped from the cache by its thread
    if (e->loaded) {
      *out = e->k;
      return kReady;
    }
  }
  std::string err;
  return get_kernel(device, nullptr, primers, true, out, &err) ? kBusy : kReady;
}

}  // namespace

ah_status tm_kernel_for(ah_ctx* ctx, const ah_primers* p, bool wait, int slot, TmKernel* out) {
  *out = TmKernel{};
  if (ctx->tm_kernel == 1 || p->n_pairs == 0 || 2 * p->n_pairs > (uint32_t)kTmJitMaxPrimers) return AH_OK;
  const std::vector<std::string> primers = primer_list(p);
  if (tm_chain_adjacent(primers) > kTmJitMaxAdjacent) return AH_OK;
  if (ctx->tm_kernel == 2 && !wait) {  // the built-in kernel until the generated one is compiled
    const Lookup l = lookup(ctx->device, primers, out);
    if (l == kReady) {
      out->split_sites = ctx->tm_split_sites;
      return tm_tab_image(ctx, slot, &out->image);
    }
    *out = TmKernel{};
    if (l == kAbsent) {
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
      auto flag = std::make_shared<std::atomic<int>>(0);
      ctx->compiles.emplace_back(std::thread([ctx, device, primers, flag] {
                                   TmKernel k;
                                   std::string err;
                                   flag->store(get_kernel(device, ctx, primers, false, &k, &err) ? 2 : 1);
                                 }),
                                 flag);
    }
    return AH_OK;
  }
  std::string err;
  const ah_status st = get_kernel(ctx->device, ctx, primers, true, out, &err);
  if (st) {
    *out = TmKernel{};
    return fail(ctx, st, "%s", err.c_str());
  }
  out->split_sites = ctx->tm_split_sites;
  return tm_tab_image(ctx, slot, &out->image);
}

}  // namespace ah

extern "C" {

ah_status ah_tm_kernel_check(const char* const* primers, uint32_t n, int sm, char* log, uint64_t log_cap) {
  if (log && log_cap) log[0] = '\0';
  if (!primers || n == 0 || n > 64 || sm < 50) return AH_EINVAL;
  std::vector<std::string> v;
  for (uint32_t i = 0; i < n; ++i) {
    if (!primers[i]) return AH_EINVAL;
    std::string s(primers[i]);
    if (s.size() < 2 || s.size() > 32) return AH_EINVAL;
    for (char& ch : s) {
      ch = (char)toupper((unsigned char)ch);
      if (!strchr("ACGTRYSWKMBDHVN", ch)) return AH_EINVAL;
    }
    v.push_back(s);
  }
  std::vector<char> cubin;
  std::string err;
  const ah_status st = ah::nvrtc_compile_sm(sm, ah::tm_chain_source(v, nullptr), "ah_tm_jit.cu", &cubin, &err);
  if (st && log && log_cap) {
    const size_t k = std::min<size_t>(err.size(), log_cap - 1);
    memcpy(log, err.data(), k);
    log[k] = '\0';
  }
  return st;
}

}  // extern "C"
