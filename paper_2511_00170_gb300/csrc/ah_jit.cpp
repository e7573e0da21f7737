// Run-time specialisation of the scan kernel for one primer set (Supplementary, "Primer matching
// and clamp logic": per-base IUPAC masks, mismatch counting, exact 3' clamp).
//
// The kernel is bit-sliced: one 32-bit word holds one bit for each of 32 consecutive genome
// positions.  For pattern position j the genome is read through "planes" shifted by j bases
// (a funnel shift of two consecutive plane words), so word bit b answers "does the base at
// position p+j, p = 32g+b, belong to the IUPAC set of pattern position j?" for 32 positions at
// once.  The mismatch bits of the non-clamp positions are summed by a carry-save tree of full
// adders that only keeps the count up to the threshold k+1; the clamp positions are OR-ed into the
// failure word directly.  Because each IUPAC set becomes a fixed boolean function of the two code
// bits, and each adder a fixed three-input function, everything compiles to LOP3 and SHF
// instructions with constant truth tables -- which is why the source is generated per primer set.
//
// Candidate bits are rare; they go to an out-of-line routine that re-checks the window exactly
// (and flags any disagreement), rejects windows with invalid bases or past the record end, and
// appends a 64-bit key to the tile's slot list.
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <atomic>
#include <condition_variable>
#include <map>
#include <thread>
#include <sstream>

#include "ah_internal.h"

namespace ah {
namespace {

// plane kinds computed from the two code bits (lo, hi) of a group word
enum Kind { K_A = 0, K_C, K_T, K_G, K_LO, K_HI, K_XOR, K_COUNT };
const char* kKindName[K_COUNT] = {"A", "C", "T", "G", "LO", "HI", "XO"};
// plane of one kind computed from the code-bit words lo<w>, hi<w>
std::string kind_expr(int kind, int w) {
  const std::string lo = "lo" + std::to_string(w), hi = "hi" + std::to_string(w);
  switch (kind) {
    case K_A: return "~(" + lo + " | " + hi + ")";
    case K_C: return "(" + lo + " & ~" + hi + ")";
    case K_T: return "(~" + lo + " & " + hi + ")";
    case K_G: return "(" + lo + " & " + hi + ")";
    case K_LO: return lo;
    case K_HI: return hi;
    default: return "(" + lo + " ^ " + hi + ")";
  }
}

// IUPAC set (over codes A=1, C=2, T=4, G=8) -> the plane whose bit says "base in set", possibly
// complemented.  Returns false for N (always matches).
bool set_plane(uint8_t set, int* kind, bool* inverted) {
  *inverted = false;
  switch (set) {
    case SET_A: *kind = K_A; return true;
    case SET_C: *kind = K_C; return true;
    case SET_T: *kind = K_T; return true;
    case SET_G: *kind = K_G; return true;
    case SET_A | SET_G: *kind = K_XOR; *inverted = true; return true;  // R: lo == hi
    case SET_C | SET_T: *kind = K_XOR; return true;                    // Y: lo != hi
    case SET_C | SET_G: *kind = K_LO; return true;                     // S: lo set
    case SET_A | SET_T: *kind = K_LO; *inverted = true; return true;   // W: lo clear
    case SET_T | SET_G: *kind = K_HI; return true;                     // K: hi set
    case SET_A | SET_C: *kind = K_HI; *inverted = true; return true;   // M: hi clear
    case SET_C | SET_T | SET_G: *kind = K_A; *inverted = true; return true;  // B: not A
    case SET_A | SET_T | SET_G: *kind = K_C; *inverted = true; return true;  // D: not C
    case SET_A | SET_C | SET_T: *kind = K_G; *inverted = true; return true;  // H: not G
    case SET_A | SET_C | SET_G: *kind = K_T; *inverted = true; return true;  // V: not T
    default: return false;                                                   // N
  }
}

// A 32-bit value of the generated code, possibly complemented: the value is ~name when inv.
struct Val {
  std::string name;
  bool inv = false;
  bool is_const = false;  // all ones (inv=false) or all zeros (inv=true)
};

Val ones() { return Val{"", false, true}; }

struct Emitter {
  std::ostringstream os;
  int tmp = 0;
  int ops = 0;  // LOP3 instructions emitted
  // one LOP3 computing f(a, b, c) on the actual (complement-resolved) values; f works bitwise on
  // the 8-bit patterns a = 0xF0, b = 0xCC, c = 0xAA, the PTX truth-table convention
  template <class F>
  Val lop3(const Val& a, const Val& b, const Val& c, F f) {
    auto pat = [](const Val& v, unsigned base) -> unsigned {
      if (v.is_const) return v.inv ? 0x00u : 0xFFu;
      return v.inv ? (~base & 0xFFu) : base;
    };
    const unsigned lut = f(pat(a, 0xF0u), pat(b, 0xCCu), pat(c, 0xAAu)) & 0xFFu;
    auto reg = [&](const Val& v) { return v.is_const ? std::string("0u") : v.name; };
    Val out{"t" + std::to_string(tmp++), false, false};
    char buf[32];
    snprintf(buf, sizeof buf, "0x%02x", lut);
    os << "      u32 " << out.name << "; asm(\"lop3.b32 %0, %1, %2, %3, " << buf << ";\" : \"=r\"(" << out.name
       << ") : \"r\"(" << reg(a) << "), \"r\"(" << reg(b) << "), \"r\"(" << reg(c) << "));\n";
    ++ops;
    return out;
  }
  Val xor3(const Val& a, const Val& b, const Val& c) {
    return lop3(a, b, c, [](unsigned x, unsigned y, unsigned z) { return x ^ y ^ z; });
  }
  Val maj(const Val& a, const Val& b, const Val& c) {
    return lop3(a, b, c, [](unsigned x, unsigned y, unsigned z) { return (x & y) | (z & (x | y)); });
  }
  Val xor2(const Val& a, const Val& b) { return lop3(a, b, a, [](unsigned x, unsigned y, unsigned) { return x ^ y; }); }
  Val and2(const Val& a, const Val& b) { return lop3(a, b, a, [](unsigned x, unsigned y, unsigned) { return x & y; }); }
  Val or2(const Val& a, const Val& b) { return lop3(a, b, a, [](unsigned x, unsigned y, unsigned) { return x | y; }); }
  Val or3(const Val& a, const Val& b, const Val& c) {
    return lop3(a, b, c, [](unsigned x, unsigned y, unsigned z) { return x | y | z; });
  }
};

std::string plane_name(int kind, int j) { return "p" + std::string(kKindName[kind]) + "_" + std::to_string(j); }

std::string expr_of(const Val& v) {
  if (v.is_const) return v.inv ? "0u" : "0xffffffffu";
  return v.inv ? "(~" + v.name + ")" : v.name;
}

// OR-reduce with three-input ORs
Val or_reduce(Emitter& E, std::vector<Val> v) {
  if (v.empty()) return Val{"", true, true};  // all zeros
  while (v.size() > 1) {
    std::vector<Val> nv;
    size_t i = 0;
    for (; i + 2 < v.size(); i += 3) nv.push_back(E.or3(v[i], v[i + 1], v[i + 2]));
    if (i + 1 < v.size()) {
      nv.push_back(E.or2(v[i], v[i + 1]));
      i += 2;
    }
    for (; i < v.size(); ++i) nv.push_back(v[i]);
    v.swap(nv);
  }
  return v[0];
}

// carry-save reduction of the bits at each weight below wsat to at most one bit per weight; carries
// at weight wsat or above are failures (the count has reached wsat > k)
void reduce_bits(Emitter& E, std::map<int, std::vector<Val>>& bits, int wsat, std::vector<Val>& fail_terms) {
  auto carry = [&](int w, const Val& c) {
    if (w >= wsat)
      fail_terms.push_back(c);
    else
      bits[w].push_back(c);
  };
  for (int w = 1; w < wsat; w *= 2) {
    std::vector<Val> list = bits[w];
    while (list.size() >= 3) {
      std::vector<Val> nl;
      size_t i = 0;
      for (; i + 2 < list.size(); i += 3) {
        nl.push_back(E.xor3(list[i], list[i + 1], list[i + 2]));
        carry(2 * w, E.maj(list[i], list[i + 1], list[i + 2]));
      }
      for (; i < list.size(); ++i) nl.push_back(list[i]);
      list.swap(nl);
    }
    if (list.size() == 2) {
      const Val a = list[0], b = list[1];
      list = {E.xor2(a, b)};
      carry(2 * w, E.and2(a, b));
    }
    bits[w] = list;
  }
}

// count >= T over the reduced bits (weights 1 .. wsat/2, at most one bit each), or nothing when the
// count cannot reach T below wsat (T == wsat: the carries already say it)
void count_ge(Emitter& E, std::map<int, std::vector<Val>>& bits, int wsat, int T, std::vector<Val>& fail_terms) {
  if (T == wsat) return;
  Val ge = ones();
  for (int w = 1, i = 0; w < wsat; w *= 2, ++i) {
    const Val b = bits[w].empty() ? Val{"", true, true} : bits[w][0];
    const bool tbit = (T >> i) & 1;
    if (ge.is_const && !ge.inv) {
      ge = tbit ? b : ones();  // b & 1 = b ; b | 1 = 1
    } else if (b.is_const) {
      ge = tbit ? Val{"", true, true} : ge;  // 0 & ge = 0 ; 0 | ge = ge
    } else {
      ge = tbit ? E.and2(b, ge) : E.or2(b, ge);
    }
  }
  if (!(ge.is_const && ge.inv)) fail_terms.push_back(ge);
}

// Failure word of one pattern: bit set iff a clamp position mismatches or the non-clamp mismatches
// reach k+1.  Phase A (emitted with every pattern's, sharing shifted planes) covers the clamp and the
// h counted positions most likely to mismatch; phase B adds the rest to the same carry-save sums.
// The kernel runs phase B only when some window of the warp survived phase A (a warp vote): for the
// others the answer is already "fail", so the result is exact for any h.  h is the one with the
// least expected work (choose_split).
struct PatternCode {
  Val fail_a;                               // failure word after phase A (final without phase B)
  bool has_b = false;
  std::vector<std::pair<int, int>> planes_b;  // shifted planes phase B reads
  std::string code_b;                       // phase B statements
  Val fail_b;                               // final failure word, defined in code_b
  int ops_b = 0;
};

// One pattern's evaluated positions: the clamp, and the counted ones most likely to mismatch first,
// with surv[i] the probability that a window of uniform random bases passes the clamp and has fewer
// than T = k + 1 mismatches among the first i counted positions.
struct PatternIn {
  struct In {
    Val x;
    int kind, j;
    double p_mis;
  };
  std::vector<In> clamp, counted;
  int T = 1, wsat = 1;
  std::vector<double> surv;
};

PatternIn pattern_in(const Pattern& P) {
  PatternIn S;
  for (int j = 0; j < P.len; ++j) {
    int kind;
    bool inv;
    if (!set_plane(P.set[j], &kind, &inv)) continue;  // N never mismatches
    // mismatch bit: the complement of the match plane; its probability on uniform bases
    const int n_bases = __builtin_popcount(P.set[j]);
    PatternIn::In in{Val{plane_name(kind, j), !inv, false}, kind, j, (4 - n_bases) / 4.0};
    (j >= P.clamp_lo && j < P.clamp_hi ? S.clamp : S.counted).push_back(in);
  }
  S.T = P.k + 1;  // failing count
  while (S.wsat < S.T) S.wsat *= 2;
  std::stable_sort(S.counted.begin(), S.counted.end(),
                   [](const PatternIn::In& a, const PatternIn::In& b) { return a.p_mis > b.p_mis; });
  double p_clamp = 1.0;
  for (const auto& c : S.clamp) p_clamp *= 1.0 - c.p_mis;
  std::vector<double> dist(S.T + 1, 0.0);  // P(count = c) for c < T, dist[T]: count >= T
  dist[0] = 1.0;
  S.surv.push_back(p_clamp);
  for (const auto& c : S.counted) {
    std::vector<double> nd(S.T + 1, 0.0);
    for (int v = 0; v <= S.T; ++v) {
      nd[std::min(S.T, v + 1)] += dist[v] * c.p_mis;
      nd[v] += dist[v] * (1.0 - c.p_mis);
    }
    dist.swap(nd);
    S.surv.push_back(p_clamp * (1.0 - dist[S.T]));
  }
  return S;
}

// the pattern's code with phase A over the clamp and counted[0, h); used_a collects the shifted
// planes phase A reads
PatternCode emit_pattern(Emitter& EA, int* tmp, const PatternIn& S, size_t h,
                         std::map<std::pair<int, int>, bool>& used_a) {
  const auto& clamp = S.clamp;
  const auto& counted = S.counted;
  const int T = S.T, wsat = S.wsat;
  PatternCode out;
  std::vector<Val> fail_terms;
  for (const auto& c : clamp) {
    used_a[{c.kind, c.j}] = true;
    fail_terms.push_back(c.x);
  }
  std::map<int, std::vector<Val>> bits;
  for (size_t i = 0; i < h; ++i) {
    used_a[{counted[i].kind, counted[i].j}] = true;
    bits[1].push_back(counted[i].x);
  }
  if ((int)counted.size() < T) {  // the count can never fail: only the clamp decides
    out.fail_a = or_reduce(EA, fail_terms);
    return out;
  }
  if (wsat == 1) {  // k = 0: every counted mismatch fails
    for (size_t i = 0; i < h; ++i) fail_terms.push_back(counted[i].x);
  } else {
    reduce_bits(EA, bits, wsat, fail_terms);
  }
  if (h == counted.size()) {
    if (wsat > 1) count_ge(EA, bits, wsat, T, fail_terms);
    out.fail_a = or_reduce(EA, fail_terms);
    return out;
  }
  // phase A's failure word: the failures so far and the partial count reaching T
  {
    std::vector<Val> fa = fail_terms;
    if (wsat > 1) {
      std::map<int, std::vector<Val>> partial = bits;
      count_ge(EA, partial, wsat, T, fa);
    }
    out.fail_a = or_reduce(EA, fa);
  }
  // phase B: the remaining positions join the same sums.  A count that reached T in phase A only
  // grows, so phase A's failure word is part of the final one; phase B adds its own carries past
  // wsat and the final comparison.
  Emitter EB;
  EB.tmp = *tmp > EA.tmp ? *tmp : EA.tmp;
  std::map<std::pair<int, int>, bool> seen;
  std::vector<Val> fail_b{out.fail_a};
  for (size_t i = h; i < counted.size(); ++i) {
    const std::pair<int, int> pl{counted[i].kind, counted[i].j};
    if (!seen.count(pl)) out.planes_b.push_back(pl), seen[pl] = true;
    if (wsat == 1)
      fail_b.push_back(counted[i].x);
    else
      bits[1].push_back(counted[i].x);
  }
  if (wsat > 1) {
    reduce_bits(EB, bits, wsat, fail_b);
    count_ge(EB, bits, wsat, T, fail_b);
  }
  out.fail_b = or_reduce(EB, fail_b);
  out.has_b = true;
  out.code_b = EB.os.str();
  out.ops_b = EB.ops;
  EA.tmp = EB.tmp;  // temporaries stay unique across phases
  *tmp = EB.tmp;
  return out;
}

// instructions of the vote and its branch, paid by every warp whenever the pattern has a phase B
constexpr double kVoteOps = 2.0;

// Phase A's length h with the least expected ALU work per group of 32 positions: phase A's LOP3
// and the funnel shifts of planes no earlier pattern reads, plus phase B's times the probability
// that one of the `windows` windows a vote covers survives phase A (on uniform random bases; one
// vote covers 32 lanes x 32 positions, and larger values stand for genomes whose composition lets
// more windows through).  Phase B keeps at least 3 positions; h = all counted positions means a
// single phase.
size_t choose_split(const PatternIn& S, const std::map<std::pair<int, int>, bool>& used, double windows) {
  const size_t n = S.counted.size();
  if ((int)n < S.T) return n;
  auto shifts_new = [&](const std::pair<int, int>& pl, const std::map<std::pair<int, int>, bool>& have) {
    return pl.second > 0 && !have.count(pl) ? 1 : 0;
  };
  size_t best_h = n;
  double best = 0.0;
  bool have = false;
  for (size_t h = 0; h <= n; ++h) {
    if (h < n && n - h < 3) continue;
    Emitter E;
    int tmp = 0;
    std::map<std::pair<int, int>, bool> u = used;
    const PatternCode pc = emit_pattern(E, &tmp, S, h, u);
    double cost = E.ops;
    for (const auto& pl : u) cost += used.count(pl.first) ? 0 : (pl.first.second > 0);
    if (pc.has_b) {
      double b = pc.ops_b;
      for (const auto& pl : pc.planes_b) b += shifts_new(pl, u);
      const double p_any = -std::expm1(windows * std::log1p(-std::min(S.surv[h], 1.0 - 1e-12)));
      cost += kVoteOps + p_any * b;
    }
    if (!have || cost < best - 1e-9) best = cost, best_h = h, have = true;
  }
  return best_h;
}

PatternCode gen_pattern(Emitter& EA, int* tmp, const Pattern& P, std::map<std::pair<int, int>, bool>& used_a,
                        double windows) {
  const PatternIn S = pattern_in(P);
  return emit_pattern(EA, tmp, S, choose_split(S, used_a, windows), used_a);
}

const char* kPrelude = R"(
typedef unsigned int u32;
typedef unsigned long long u64;
struct ScanParams {
  const uint2* planes;
  const u32* invalid;
  const u64* rec_group;
  const u32* rec_len;
  u32 n_rec;
  u32 slot_cap;
  u64 group_begin;
  u64 n_groups;
  u64* slots;
  u32* tile_count;
  u32* status;
  u64 tile_groups;          // groups per tile of the slot lists: the tile of group g is g / tile_groups
  unsigned long long* work;
  u64 n_blocks;             // persistent kernels: blocks of NT * GPT groups in this launch
};
static __device__ __forceinline__ u32 fshr(u32 a, u32 b, u32 s) { return __funnelshift_r(a, b, s); }

// One candidate bit (window at bit i of group g, pattern q): an exact re-check by a second method
// (the window's bases against per-position set masks, mismatches counted by popcount), then the
// invalid-base test.  Every record is followed by at least one invalid padding base, so a window
// that leaves its record holds an invalid base and the one test covers record bounds too.  True
// with the window's slot key when it is a site; a disagreement with the circuit sets the status.
static __device__ __forceinline__ bool check_bit(int q, int i, u64 lo64, u64 hi64, u64 inv64, u64 g, u64 tile_pos,
                                                 const ScanParams& P, u64* key) {
  const int L = PLEN[q];
  const u32 wm = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
  const u32 wl = (u32)(lo64 >> i), wh = (u32)(hi64 >> i);  // base j of the window at bit j
  const u32 match = (~wl & ~wh & MSET[q][0]) | (wl & ~wh & MSET[q][1]) | (~wl & wh & MSET[q][2]) |
                    (wl & wh & MSET[q][3]);
  const u32 mis = ~match & wm;
  const int mism = __popc(mis);
  if ((mis & PCLAMP[q]) || mism > PK[q]) {
    atomicOr(P.status, 1u);
    return false;
  }
  if ((u32)(inv64 >> i) & wm) return false;
  const u64 pos = g * 32ull + (u64)i;
  *key = ((u64)PPAIR[q] << 48) | ((pos - tile_pos) << 16) | ((u64)PORIENT[q] << 8) | (u64)mism;
  return true;
}

// Slot append for the lanes of `mask` whose ok is set: the lanes of one tile (peers, led by
// leader) take their slots with one atomic add and write at their rank among them.
static __device__ __forceinline__ void append(u32 mask, u32 peers, u32 leader, bool ok, u64 key, u64 tile,
                                              const ScanParams& P) {
  const u32 lane = threadIdx.x & 31u;
  const u32 vb = __ballot_sync(mask, ok) & peers;
  u32 base = 0;
  if (lane == leader && vb) base = atomicAdd(P.tile_count + tile, (u32)__popc(vb));
  base = __shfl_sync(mask, base, leader);
  if (ok) {
    const u32 idx = base + __popc(vb & ((1u << lane) - 1u));
    if (idx < P.slot_cap) P.slots[tile * (u64)P.slot_cap + idx] = key;
  }
}

// Candidate words of up to four patterns q0 .. q0+3 (c[0..3], 0 where absent) handled at once by
// the lanes that reach this call together, one candidate bit per lane per round: where the words
// are found, or when a warp's candidate queue is full.  EMIT_INLINE: inlined where the words are
// found for small pattern sets (frequent sites then cost no call and no saving of the loop's
// registers), a call otherwise.
static __device__ EMIT_INLINE void emit4(u32 c0, u32 c1, u32 c2, u32 c3, int q0, u64 g, uint2 a, uint2 b,
                                         const ScanParams& P) {
  const u32 mask = __activemask();
  const u32 lane = threadIdx.x & 31u;
  const u64 tile = g / P.tile_groups, tile_pos = tile * P.tile_groups * 32ull;
  const u32 peers = __match_any_sync(mask, tile);
  const u32 leader = __ffs(peers) - 1, below = peers & ((1u << lane) - 1u);
  const u64 lo64 = (u64)a.x | ((u64)b.x << 32), hi64 = (u64)a.y | ((u64)b.y << 32);
  const u64 inv64 = (u64)P.invalid[g] | ((u64)P.invalid[g + 1] << 32);
  u32 w[4] = {c0, c1, c2, c3};
  for (;;) {
    int k = -1, i = 0;
    for (int t = 0; t < 4; ++t)
      if (k < 0 && w[t]) {
        k = t;
        i = __ffs(w[t]) - 1;
        w[t] &= w[t] - 1;
      }
    if (!__any_sync(mask, k >= 0)) break;
    bool ok = false;
    u64 key = 0;
    if (k >= 0) {  // check_bit's test written out: in this form the bench pair's loop ran 1.6 % faster
      const int q = q0 + k;
      const int L = PLEN[q];
      const u32 wm = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
      const u32 wl = (u32)(lo64 >> i), wh = (u32)(hi64 >> i);  // base j of the window at bit j
      const u32 match = (~wl & ~wh & MSET[q][0]) | (wl & ~wh & MSET[q][1]) | (~wl & wh & MSET[q][2]) |
                        (wl & wh & MSET[q][3]);
      const u32 mis = ~match & wm;
      const int mism = __popc(mis);
      if ((mis & PCLAMP[q]) || mism > PK[q]) {
        atomicOr(P.status, 1u);
      } else if (!((u32)(inv64 >> i) & wm)) {
        const u64 pos = g * 32ull + (u64)i;
        key = ((u64)PPAIR[q] << 48) | ((pos - tile_pos) << 16) | ((u64)PORIENT[q] << 8) | (u64)mism;
        ok = true;
      }
    }
    const u32 vb = __ballot_sync(mask, ok) & peers;
    u32 base = 0;
    if (lane == leader && vb) base = atomicAdd(P.tile_count + tile, (u32)__popc(vb));
    base = __shfl_sync(mask, base, leader);
    if (ok) {
      const u32 idx = base + __popc(vb & below);
      if (idx < P.slot_cap) P.slots[tile * (u64)P.slot_cap + idx] = key;
    }
  }
}

// A warp's queue of candidate words: QCAP entries of (word, pattern | group offset in the block << 16)
#define QCAP 64

// A lane's candidate words of patterns q0 .. q0+3 (group at offset off in the block) into its warp's
// queue; a full queue sends the word on at once.
static __device__ __forceinline__ void push4(u32 c0, u32 c1, u32 c2, u32 c3, int q0, u32 off, u64 g, uint2 a,
                                             uint2 b, const ScanParams& P, u32* qw, u32* qm, u32* qn) {
  const u32 c[4] = {c0, c1, c2, c3};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (!c[t]) continue;
    const u32 idx = atomicAdd(qn, 1u);
    if (idx < QCAP) {
      qw[idx] = c[t];
      qm[idx] = (off << 16) | (u32)(q0 + t);
    } else {
      emit4(t == 0 ? c[t] : 0u, t == 1 ? c[t] : 0u, t == 2 ? c[t] : 0u, t == 3 ? c[t] : 0u, q0, g, a, b, P);
    }
  }
}

// The warp's queued candidate words (n of them), 32 at a time, one word per lane, one bit per lane
// per round; every lane of the warp takes part.
static __device__ __forceinline__ void drain(const ScanParams& P, u64 first, const u32* qw, const u32* qm, u32 n) {
  const u32 lane = threadIdx.x & 31u;
  for (u32 e0 = 0; e0 < n; e0 += 32) {
    const u32 e = e0 + lane;
    u32 h = 0;
    int q = 0;
    u64 g = 0, lo64 = 0, hi64 = 0, inv64 = 0;
    if (e < n) {
      h = qw[e];
      const u32 m = qm[e];
      q = (int)(m & 0xffffu);
      g = P.group_begin + first + (m >> 16);
      const uint2 a = __ldg(P.planes + g), b = __ldg(P.planes + g + 1);
      lo64 = (u64)a.x | ((u64)b.x << 32);
      hi64 = (u64)a.y | ((u64)b.y << 32);
      inv64 = (u64)P.invalid[g] | ((u64)P.invalid[g + 1] << 32);
    }
    const u64 tile = g / P.tile_groups, tile_pos = tile * P.tile_groups * 32ull;
    const u32 peers = __match_any_sync(0xffffffffu, tile);
    const u32 leader = __ffs(peers) - 1;
    for (;;) {
      int i = -1;
      if (h) {
        i = __ffs(h) - 1;
        h &= h - 1;
      }
      if (!__any_sync(0xffffffffu, i >= 0)) break;
      u64 key = 0;
      const bool ok = i >= 0 && check_bit(q, i, lo64, hi64, inv64, g, tile_pos, P, &key);
      append(0xffffffffu, peers, leader, ok, key, tile, P);
    }
  }
}
)";

}  // namespace

std::string scan_source(const std::vector<Pattern>& pats, const ScanConfig& cfg, int* alu_ops_per_group) {
  const int Q = (int)pats.size();
  std::ostringstream os;
  os << "// generated scan kernel: " << Q << " patterns\n";
  os << "#define NT " << cfg.threads << "\n#define GPT " << cfg.groups_per_thread << "\n// shift mode "
     << cfg.shift_mode << ", persistent " << cfg.persistent << "\n";
  auto table = [&](const char* type, const char* name, auto get) {
    os << "static __device__ const " << type << " " << name << "[" << Q << "] = {";
    for (int q = 0; q < Q; ++q) os << (q ? "," : "") << (unsigned)get(pats[q]);
    os << "};\n";
  };
  table("unsigned char", "PLEN", [](const Pattern& p) { return p.len; });
  table("unsigned char", "PK", [](const Pattern& p) { return p.k; });
  table("unsigned short", "PPAIR", [](const Pattern& p) { return p.id / 4; });
  table("unsigned char", "PORIENT", [](const Pattern& p) { return p.id % 4; });
  // per pattern and code c (A, C, T, G): bit j set iff position j's set holds c; and the clamp's bits
  os << "static __device__ const unsigned int MSET[" << Q << "][4] = {";
  for (int q = 0; q < Q; ++q) {
    os << (q ? "," : "") << "{";
    for (int c = 0; c < 4; ++c) {
      uint32_t m = 0;
      for (int j = 0; j < pats[q].len; ++j)
        if ((pats[q].set[j] >> c) & 1) m |= 1u << j;
      os << (c ? "," : "") << m << "u";
    }
    os << "}";
  }
  os << "};\n";
  table("unsigned int", "PCLAMP", [](const Pattern& p) {
    uint32_t m = 0;
    for (int j = p.clamp_lo; j < p.clamp_hi; ++j) m |= 1u << j;
    return m;
  });
  // direct emission: the routine inlined at up to two call sites (8 patterns; measured on GB300 the
  // dense-site workload, 4 patterns, scanned 5 % faster inlined and the 32-pattern set 5 % slower);
  // with the queue it is only the rare fallback
  os << "#define EMIT_INLINE " << (!cfg.emit_queue && Q <= 8 ? "__forceinline__" : "__noinline__") << "\n";
  os << kPrelude;

  // body: per group of 32 positions
  Emitter E;
  std::map<std::pair<int, int>, bool> used;
  std::vector<PatternCode> pc(Q);
  int tmpc = 0;
  for (int q = 0; q < Q; ++q) pc[q] = gen_pattern(E, &tmpc, pats[q], used, std::max(1, cfg.vote_windows));
  bool kind_used[K_COUNT] = {};
  for (auto& u : used) kind_used[u.first.first] = true;
  for (auto& c : pc)
    for (auto& pl : c.planes_b) kind_used[pl.first] = true;
  if (alu_ops_per_group) {
    // the circuit's ALU instructions per group of 32 positions when every phase runs: LOP3 of the
    // trees, one funnel shift per (plane, offset), plane derivations (one per derived kind and
    // word), and the AND-reduction of failure words per block of four patterns
    int shifts = 0, derived = 0, ops_b = 0;
    for (auto& u : used) shifts += u.first.second > 0;
    for (auto& c : pc) {
      ops_b += c.ops_b;
      for (auto& pl : c.planes_b) shifts += pl.second > 0 && !used.count(pl);
    }
    for (int k = 0; k < K_COUNT; ++k) derived += kind_used[k] && k != K_LO && k != K_HI ? 2 : 0;
    *alu_ops_per_group = E.ops + ops_b + shifts + derived + 2 * ((Q + 3) / 4);
  }

  // one block of the launch: NT threads x GPT groups of 32 positions, from group_begin
  os << "static __device__ __forceinline__ void scan_block(const ScanParams& P, const u64 blk) {\n";
  if (cfg.emit_queue) {
    os << "  __shared__ u32 cand_w[NT / 32][QCAP], cand_m[NT / 32][QCAP], cand_n[NT / 32];\n";
    os << "  const u32 wp = threadIdx.x >> 5;\n";
    os << "  if ((threadIdx.x & 31u) == 0) cand_n[wp] = 0;\n  __syncwarp();\n";
  }
  os << "  const u64 first = blk * (u64)(NT * GPT);\n";
  os << "  u64 gl = first + threadIdx.x;\n";
  os << "  uint2 na = make_uint2(0u, 0u), nb = na;\n";
  os << "  if (gl < P.n_groups) { na = __ldg(P.planes + P.group_begin + gl); nb = __ldg(P.planes + P.group_begin + gl + 1); }\n";
  os << "#pragma unroll 1\n";
  os << "  for (int it = 0; it < GPT; ++it, gl += NT) {\n";
  os << "    if (gl >= P.n_groups) break;\n";
  os << "    const uint2 a = na, b = nb;\n";
  os << "    const u64 gn = gl + NT;\n";
  os << "    if (it + 1 < GPT && gn < P.n_groups) { na = __ldg(P.planes + P.group_begin + gn); nb = __ldg(P.planes + P.group_begin + gn + 1); }\n";
  os << "    const u64 g = P.group_begin + gl;\n";
  os << "    const u32 lo0 = a.x, hi0 = a.y, lo1 = b.x, hi1 = b.y;\n";
  for (int k = 0; k < K_COUNT; ++k) {
    if (!kind_used[k]) continue;
    for (int w = 0; w < 2; ++w) os << "    const u32 " << kKindName[k] << w << " = " << kind_expr(k, w) << ";\n";
  }
  int nshift = 0;
  auto emit_shift = [&](int kind, int j, const char* indent) {
    const std::string name = plane_name(kind, j), w0 = std::string(kKindName[kind]) + "0",
                      w1 = std::string(kKindName[kind]) + "1";
    if (j == 0) {
      os << indent << "const u32 " << name << " = " << w0 << ";\n";
      return;
    }
    const bool by_multiply = cfg.shift_mode == 1 || (cfg.shift_mode == 2 && (nshift++ & 1));
    if (!by_multiply) {
      os << indent << "const u32 " << name << " = fshr(" << w0 << ", " << w1 << ", " << j << "u);\n";
    } else {
      // (w0 >> j) | (w1 << (32 - j)) as hi(w0 * 2^(32-j)) + lo(w1 * 2^(32-j)): two integer
      // multiply-adds on the FMA pipe instead of one funnel shift on the ALU pipe
      const unsigned long long m = 1ull << (32 - j);
      os << indent << "u32 " << name << ";\n" << indent << "{ u32 t_; asm(\"mul.lo.u32 %0, %1, " << m
         << ";\" : \"=r\"(t_) : \"r\"(" << w1 << ")); asm(\"mad.hi.u32 %0, %1, " << m << ", %2;\" : \"=r\"(" << name
         << ") : \"r\"(" << w0 << "), \"r\"(t_)); }\n";
    }
  };
  for (auto& u : used) emit_shift(u.first.first, u.first.second, "    ");
  os << "    {\n" << E.os.str();
  // phase B of each pattern, only for warps with a window that survived phase A
  for (int q = 0; q < Q; ++q) {
    os << "      u32 f" << q << " = " << expr_of(pc[q].fail_a) << ";\n";
    if (!pc[q].has_b) continue;
    os << "      if (__any_sync(__activemask(), ~f" << q << ")) {\n";
    for (auto& pl : pc[q].planes_b)
      if (!used.count(pl)) emit_shift(pl.first, pl.second, "        ");
    os << pc[q].code_b;
    os << "        f" << q << " = " << expr_of(pc[q].fail_b) << ";\n      }\n";
  }
  // hit words and the rare emission path, in blocks of four patterns
  for (int q0 = 0; q0 < Q; q0 += 4) {
    int q1 = std::min(Q, q0 + 4);
    os << "      if (__builtin_expect((";
    for (int q = q0; q < q1; ++q) os << (q > q0 ? " & " : "") << "f" << q;
    os << ") != 0xffffffffu, 0)) " << (cfg.emit_queue ? "push4(" : "emit4(");
    for (int q = q0; q < q0 + 4; ++q) os << (q < q1 ? "~f" + std::to_string(q) : std::string("0u")) << ", ";
    if (cfg.emit_queue)
      os << q0 << ", (u32)(gl - first), g, a, b, P, cand_w[wp], cand_m[wp], &cand_n[wp]);\n";
    else
      os << q0 << ", g, a, b, P);\n";
  }
  os << "    }\n  }\n";
  // the queued candidates, by the whole warp once its groups are done
  if (cfg.emit_queue)
    os << "  __syncwarp();\n  drain(P, first, cand_w[wp], cand_m[wp], min(cand_n[wp], (u32)QCAP));\n";
  os << "}\n";
  os << "extern \"C\" __global__ void __launch_bounds__(NT" << (cfg.min_blocks > 0 ? ", " + std::to_string(cfg.min_blocks) : "")
     << ") ah_scan_jit(const ScanParams P) {\n";
  if (cfg.persistent) {
    // persistent CTAs take tiles from a counter until none are left
    os << "  __shared__ u64 s_tile;\n  for (;;) {\n";
    os << "    if (threadIdx.x == 0) s_tile = atomicAdd(P.work, 1ull);\n    __syncthreads();\n";
    os << "    const u64 t = s_tile;\n    __syncthreads();\n    if (t >= P.n_blocks) break;\n";
    os << "    scan_block(P, t);\n  }\n}\n";
  } else {
    os << "  scan_block(P, blockIdx.x);\n}\n";
  }
  return os.str();
}

// One generated kernel: compiled to a cubin (done), then loaded into the process (loaded) by the
// first caller that launches it.  Background compiles stop at the cubin, so module loading stays on
// the thread that owns the stream.
struct JitCache::Entry {
  std::mutex m;
  std::condition_variable cv;
  bool done = false;
  bool loaded = false;
  ah_status st = AH_OK;
  std::string err;
  std::vector<char> cubin;
  int ops = 0;
  ScanKernel k{};
};

ah_status nvrtc_compile(int device, const std::string& src, const char* name, std::vector<char>* cubin,
                        std::string* err) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  return nvrtc_compile_sm(major * 10 + minor, src, name, cubin, err);
}

ah_status nvrtc_compile_sm(int sm, const std::string& src, const char* name, std::vector<char>* cubin,
                           std::string* err) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), name, 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    *err = "nvrtcCreateProgram failed";
    return AH_EJIT;
  }
  std::string arch = "-arch=sm_" + std::to_string(sm) + (sm >= 90 ? "a" : "");
  const char* opts[] = {arch.c_str(), "-default-device", "-lineinfo"};
  nvrtcResult r = nvrtcCompileProgram(prog, 3, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    *err = std::string(name) + ": compilation failed: " + log.substr(0, 2000);
    return AH_EJIT;
  }
  size_t cubin_size = 0;
  nvrtcGetCUBINSize(prog, &cubin_size);
  cubin->resize(cubin_size);
  nvrtcGetCUBIN(prog, cubin->data());
  nvrtcDestroyProgram(&prog);
  return AH_OK;
}


JitCache& JitCache::global() {
  static JitCache* cache = new JitCache();  // never destroyed: kernels stay loaded until exit
  return *cache;
}

namespace {

ah_status compile(int device, const std::string& src, std::vector<char>* cubin, std::string* err) {
  return nvrtc_compile(device, src, "ah_scan_jit.cu", cubin, err);
}

// the runtime's library API (no link-time driver dependency); fills k or returns a message
ah_status load(int device, const std::vector<char>& cubin, int ops, const ScanConfig& cfg, ScanKernel* k,
               std::string* err) {
  cudaSetDevice(device);
  cudaLibrary_t lib;
  cudaError_t ce = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (ce != cudaSuccess) {
    *err = std::string("cudaLibraryLoadData failed: ") + cudaGetErrorString(ce);
    return AH_EJIT;
  }
  ce = cudaLibraryGetKernel(&k->fn, lib, "ah_scan_jit");
  if (ce != cudaSuccess) {
    *err = std::string("cudaLibraryGetKernel failed: ") + cudaGetErrorString(ce);
    return AH_EJIT;
  }
  k->threads = cfg.threads;
  k->groups_per_thread = cfg.groups_per_thread;
  k->alu_ops_per_group = ops;
  return AH_OK;
}

}  // namespace

ah_status JitCache::get(ah_ctx* ctx, const std::vector<Pattern>& pats, const ScanConfig& cfg, ScanKernel* out) {
  std::string err;
  const ah_status st = get_impl(ctx->device, ctx, pats, cfg, out, &err, true);
  return st ? fail(ctx, st, "%s", err.c_str()) : AH_OK;
}

ah_status JitCache::get_impl(int device, ah_ctx* stats, const std::vector<Pattern>& pats, const ScanConfig& cfg,
                             ScanKernel* out, std::string* err_out, bool load_it) {
  int ops = 0;
  std::string src = scan_source(pats, cfg, &ops);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  const std::string key = std::to_string(major * 10 + minor) + "\n" + src;
  std::shared_ptr<Entry> e;
  bool mine = false;
  {
    std::lock_guard<std::mutex> lock(mu_);
    auto it = cache_.find(key);
    if (it == cache_.end()) {
      e = std::make_shared<Entry>();
      cache_.emplace(key, e);
      mine = true;
    } else {
      e = it->second;
    }
  }
  if (mine) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<char> cubin;
    std::string err;
    const ah_status st = compile(device, src, &cubin, &err);
    {
      std::lock_guard<std::mutex> lock(e->m);
      e->st = st;
      e->err = err;
      e->cubin.swap(cubin);
      e->ops = ops;
      e->done = true;
    }
    e->cv.notify_all();
    if (st) {
      std::lock_guard<std::mutex> lock(mu_);
      cache_.erase(key);  // a later call may try again
    } else if (stats) {
      std::lock_guard<std::mutex> lock(stats->stats_mu);
      stats->jit_compiles++;
      stats->jit_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
  }
  std::unique_lock<std::mutex> lock(e->m);
  e->cv.wait(lock, [&] { return e->done; });
  if (e->st) {
    *err_out = e->err;
    return e->st;
  }
  if (!load_it) return AH_OK;
  if (!e->loaded) {  // the first caller that launches it loads it (under the entry's lock)
    ScanKernel k;
    const ah_status st = load(device, e->cubin, e->ops, cfg, &k, err_out);
    if (st) return st;
    e->k = k;
    e->loaded = true;
    std::vector<char>().swap(e->cubin);
  }
  *out = e->k;
  return AH_OK;
}

void JitCache::many_impl(int device, ah_ctx* stats, const std::vector<std::vector<Pattern>>& sets,
                         const ScanConfig& cfg, std::vector<ScanKernel>* out, std::vector<ah_status>* st,
                         std::vector<std::string>* err, bool load_it) {
  out->assign(sets.size(), ScanKernel{});
  st->assign(sets.size(), AH_OK);
  err->assign(sets.size(), std::string());
  if (sets.size() == 1) {
    (*st)[0] = get_impl(device, stats, sets[0], cfg, &(*out)[0], &(*err)[0], load_it);
    return;
  }
  run_parallel(sets.size(), [&](size_t i) {
    cudaSetDevice(device);
    (*st)[i] = get_impl(device, stats, sets[i], cfg, &(*out)[i], &(*err)[i], load_it);
  });
}

void JitCache::run_parallel(size_t n, const std::function<void(size_t)>& fn) {
  if (n == 0) return;
  if (n == 1) {
    fn(0);
    return;
  }
  // items are taken from a shared counter by the caller and by helper tasks on the workers; the
  // caller returns once every item is done.  A helper that starts after the last item was taken
  // finds none and leaves without touching fn.
  struct Job {
    std::function<void(size_t)> fn;
    size_t n = 0;
    std::atomic<size_t> next{0}, done{0};
    std::mutex m;
    std::condition_variable cv;
  };
  auto job = std::make_shared<Job>();
  job->fn = fn;
  job->n = n;
  auto loop = [](const std::shared_ptr<Job>& j) {
    for (size_t i = j->next++; i < j->n; i = j->next++) {
      j->fn(i);
      if (++j->done == j->n) {
        std::lock_guard<std::mutex> l(j->m);
        j->cv.notify_all();
      }
    }
  };
  {
    std::lock_guard<std::mutex> lock(pool_mu_);
    const size_t want = std::max<size_t>(1, std::min<size_t>(16, std::thread::hardware_concurrency()));
    while (workers_.size() < want)
      workers_.emplace_back([this] {
        for (;;) {
          std::function<void()> t;
          {
            std::unique_lock<std::mutex> l(pool_mu_);
            pool_cv_.wait(l, [this] { return !tasks_.empty(); });
            t = std::move(tasks_.front());
            tasks_.pop_front();
          }
          t();
        }
      });
    for (size_t h = 0; h + 1 < std::min(n, workers_.size() + 1); ++h) tasks_.emplace_back([job, loop] { loop(job); });
  }
  pool_cv_.notify_all();
  loop(job);
  std::unique_lock<std::mutex> l(job->m);
  job->cv.wait(l, [&] { return job->done.load() == job->n; });
}

ah_status JitCache::get_many(ah_ctx* ctx, const std::vector<std::vector<Pattern>>& sets, const ScanConfig& cfg,
                             std::vector<ScanKernel>* out) {
  std::vector<ah_status> st;
  std::vector<std::string> err;
  many_impl(ctx->device, ctx, sets, cfg, out, &st, &err, true);
  for (size_t i = 0; i < sets.size(); ++i)
    if (st[i]) return fail(ctx, st[i], "%s", err[i].c_str());
  return AH_OK;
}

ah_status JitCache::prefetch(int device, ah_ctx* stats, const std::vector<std::vector<Pattern>>& sets,
                             const ScanConfig& cfg) {
  cudaSetDevice(device);
  std::vector<ScanKernel> out;
  std::vector<ah_status> st;
  std::vector<std::string> err;
  many_impl(device, stats, sets, cfg, &out, &st, &err, false);
  for (ah_status s : st)
    if (s) return s;
  return AH_OK;
}

bool JitCache::ready(int device, const std::vector<std::vector<Pattern>>& sets, const ScanConfig& cfg) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  for (const auto& pats : sets) {
    int ops = 0;
    const std::string key = std::to_string(major * 10 + minor) + "\n" + scan_source(pats, cfg, &ops);
    std::shared_ptr<Entry> e;
    {
      std::lock_guard<std::mutex> lock(mu_);
      auto it = cache_.find(key);
      if (it == cache_.end()) return false;
      e = it->second;
    }
    std::lock_guard<std::mutex> lock(e->m);
    if (!e->done || e->st || !e->loaded) return false;
  }
  return true;
}

std::vector<std::vector<Pattern>> scan_groups(const std::vector<Pattern>& pats, const ScanConfig& cfg) {
  std::vector<std::vector<Pattern>> out;
  const size_t per = cfg.pairs_per_kernel > 0 ? 4 * (size_t)cfg.pairs_per_kernel : pats.size();
  for (size_t i = 0; i < pats.size(); i += per)
    out.emplace_back(pats.begin() + i, pats.begin() + std::min(pats.size(), i + per));
  if (out.empty()) out.emplace_back();
  return out;
}

}  // namespace ah
