// Melting-temperature stage (Section "Implementations": AHv2 reimplements Biopython's Tm_NN in
// double precision; Section "Primer degeneracy": Tm is evaluated for the primer's variants).
//
// Every site gets the maximum, over the concrete variants of its (degenerate) primer, of the
// nearest-neighbour Tm of the variant paired with the site; an amplicon gets the lower of its two
// site values.  All arithmetic is FP64: the Tm threshold decision needs it.  The parameter tables
// below are expanded on the host into direct lookups indexed by the four base codes of a step
// (top 5'-ab-3' over bottom 3'-xy-5'), so a step costs one constant-memory load.
#include <cmath>
#include <cstring>

#include "ah_internal.h"

namespace ah {
namespace {

struct Step {
  char a, b, x, y;  // 5'-ab-3' over 3'-xy-5'
  double dh, ds;    // kcal/mol, cal/(K mol)
};

// Watson-Crick nearest-neighbour stacks (Allawi & SantaLucia 1997, Biochemistry 36:10581).
const Step kStacks[] = {
    {'A', 'A', 'T', 'T', -7.9, -22.2}, {'A', 'T', 'T', 'A', -7.2, -20.4}, {'T', 'A', 'A', 'T', -7.2, -21.3},
    {'C', 'A', 'G', 'T', -8.5, -22.7}, {'G', 'T', 'C', 'A', -8.4, -22.4}, {'C', 'T', 'G', 'A', -7.8, -21.0},
    {'G', 'A', 'C', 'T', -8.2, -22.2}, {'C', 'G', 'G', 'C', -10.6, -27.2}, {'G', 'C', 'C', 'G', -9.8, -24.4},
    {'G', 'G', 'C', 'C', -8.0, -19.9},
};

// Internal mismatches adjacent to a Watson-Crick pair and the tandem G.T steps:
// G.T (Allawi & SantaLucia 1997), G.A (Allawi & SantaLucia 1998, Biochemistry 37:2170),
// C.T (Allawi & SantaLucia 1998, Nucleic Acids Res 26:2694), A.C (Allawi & SantaLucia 1998,
// Biochemistry 37:9435), A.A / C.C / G.G / T.T (Peyret et al. 1999, Biochemistry 38:3468).
const Step kInternal[] = {
    // G.T
    {'A', 'G', 'T', 'T', 1.0, 0.9}, {'A', 'T', 'T', 'G', -2.5, -8.3}, {'C', 'G', 'G', 'T', -4.1, -11.7},
    {'C', 'T', 'G', 'G', -2.8, -8.0}, {'G', 'G', 'C', 'T', 3.3, 10.4}, {'G', 'G', 'T', 'T', 5.8, 16.3},
    {'G', 'T', 'C', 'G', -4.4, -12.3}, {'G', 'T', 'T', 'G', 4.1, 9.5}, {'T', 'G', 'A', 'T', -0.1, -1.7},
    {'T', 'G', 'G', 'T', -1.4, -6.2}, {'T', 'T', 'A', 'G', -1.3, -5.3},
    // G.A
    {'A', 'A', 'T', 'G', -0.6, -2.3}, {'A', 'G', 'T', 'A', -0.7, -2.3}, {'C', 'A', 'G', 'G', -0.7, -2.3},
    {'C', 'G', 'G', 'A', -4.0, -13.2}, {'G', 'A', 'C', 'G', -0.6, -1.0}, {'G', 'G', 'C', 'A', 0.5, 3.2},
    {'T', 'A', 'A', 'G', 0.7, 0.7}, {'T', 'G', 'A', 'A', 3.0, 7.4},
    // C.T
    {'A', 'C', 'T', 'T', 0.7, 0.2}, {'A', 'T', 'T', 'C', -1.2, -6.2}, {'C', 'C', 'G', 'T', -0.8, -4.5},
    {'C', 'T', 'G', 'C', -1.5, -6.1}, {'G', 'C', 'C', 'T', 2.3, 5.4}, {'G', 'T', 'C', 'C', 5.2, 13.5},
    {'T', 'C', 'A', 'T', 1.2, 0.7}, {'T', 'T', 'A', 'C', 1.0, 0.7},
    // A.C
    {'A', 'A', 'T', 'C', 2.3, 4.6}, {'A', 'C', 'T', 'A', 5.3, 14.6}, {'C', 'A', 'G', 'C', 1.9, 3.7},
    {'C', 'C', 'G', 'A', 0.6, -0.6}, {'G', 'A', 'C', 'C', 5.2, 14.2}, {'G', 'C', 'C', 'A', -0.7, -3.8},
    {'T', 'A', 'A', 'C', 3.4, 8.0}, {'T', 'C', 'A', 'A', 7.6, 20.2},
    // A.A, C.C, G.G, T.T
    {'A', 'A', 'T', 'A', 1.2, 1.7}, {'C', 'A', 'G', 'A', -0.9, -4.2}, {'G', 'A', 'C', 'A', -2.9, -9.8},
    {'T', 'A', 'A', 'A', 4.7, 12.9}, {'A', 'C', 'T', 'C', 0.0, -4.4}, {'C', 'C', 'G', 'C', -1.5, -7.2},
    {'G', 'C', 'C', 'C', 3.6, 8.9}, {'T', 'C', 'A', 'C', 6.1, 16.4}, {'A', 'G', 'T', 'G', -3.1, -9.5},
    {'C', 'G', 'G', 'G', -4.9, -15.3}, {'G', 'G', 'C', 'G', -6.0, -15.8}, {'T', 'G', 'A', 'G', 1.6, 3.6},
    {'A', 'T', 'T', 'T', -2.7, -10.8}, {'C', 'T', 'G', 'T', -5.0, -15.8}, {'G', 'T', 'C', 'T', -2.2, -8.4},
    {'T', 'T', 'A', 'T', 0.2, -1.5},
};

// Terminal mismatches: 5'-ab-3'/3'-xy-5' with a.x Watson-Crick and the end pair b.y mismatched
// (SantaLucia & Peyret 2001, WO 01/94611).
const Step kTerminal[] = {
    {'A', 'A', 'T', 'A', -3.1, -7.8},  {'T', 'A', 'A', 'A', -2.5, -6.3},  {'C', 'A', 'G', 'A', -4.3, -10.7},
    {'G', 'A', 'C', 'A', -8.0, -22.5}, {'A', 'C', 'T', 'C', -0.1, 0.5},   {'T', 'C', 'A', 'C', -0.7, -1.3},
    {'C', 'C', 'G', 'C', -2.1, -5.1},  {'G', 'C', 'C', 'C', -3.9, -10.6}, {'A', 'G', 'T', 'G', -1.1, -2.1},
    {'T', 'G', 'A', 'G', -1.1, -2.7},  {'C', 'G', 'G', 'G', -3.8, -9.5},  {'G', 'G', 'C', 'G', -0.7, -19.2},
    {'A', 'T', 'T', 'T', -2.4, -6.5},  {'T', 'T', 'A', 'T', -3.2, -8.9},  {'C', 'T', 'G', 'T', -6.1, -16.9},
    {'G', 'T', 'C', 'T', -7.4, -21.2}, {'A', 'A', 'T', 'C', -1.6, -4.0},  {'A', 'C', 'T', 'A', -1.8, -3.8},
    {'C', 'A', 'G', 'C', -2.6, -5.9},  {'C', 'C', 'G', 'A', -2.7, -6.0},  {'G', 'A', 'C', 'C', -5.0, -13.8},
    {'G', 'C', 'C', 'A', -3.2, -7.1},  {'T', 'A', 'A', 'C', -2.3, -5.9},  {'T', 'C', 'A', 'A', -2.7, -7.0},
    {'A', 'C', 'T', 'T', -0.9, -1.7},  {'A', 'T', 'T', 'C', -2.3, -6.3},  {'C', 'C', 'G', 'T', -3.2, -8.0},
    {'C', 'T', 'G', 'C', -3.9, -10.6}, {'G', 'C', 'C', 'T', -4.9, -13.5}, {'G', 'T', 'C', 'C', -3.0, -7.8},
    {'T', 'C', 'A', 'T', -2.5, -6.3},  {'T', 'T', 'A', 'C', -0.7, -1.2},  {'A', 'A', 'T', 'G', -1.9, -4.4},
    {'A', 'G', 'T', 'A', -2.5, -5.9},  {'C', 'A', 'G', 'G', -3.9, -9.6},  {'C', 'G', 'G', 'A', -6.0, -15.5},
    {'G', 'A', 'C', 'G', -4.3, -11.1}, {'G', 'G', 'C', 'A', -4.6, -11.4}, {'T', 'A', 'A', 'G', -2.0, -4.7},
    {'T', 'G', 'A', 'A', -2.4, -5.8},  {'A', 'G', 'T', 'T', -3.2, -8.7},  {'A', 'T', 'T', 'G', -3.5, -9.4},
    {'C', 'G', 'G', 'T', -3.8, -9.0},  {'C', 'T', 'G', 'G', -6.6, -18.7}, {'G', 'G', 'C', 'T', -5.7, -15.9},
    {'G', 'T', 'C', 'G', -5.9, -16.1}, {'T', 'G', 'A', 'T', -3.9, -10.5}, {'T', 'T', 'A', 'G', -3.6, -9.8},
};

// Initiation terms of the same parameter set.
constexpr double kInitH = 0.0, kInitS = 0.0;
constexpr double kTermATH = 2.3, kTermATS = 4.1;
constexpr double kTermGCH = 0.1, kTermGCS = -2.8;
constexpr double kOneGCH = 0.0, kOneGCS = 0.0, kAllATH = 0.0, kAllATS = 0.0, k5TAH = 0.0, k5TAS = 0.0;
// symmetry correction of a self-complementary duplex
constexpr double kSymH = 0.0, kSymS = -1.4;

// degenerate site Tm: largest mismatch budget, and the enumeration bounds
constexpr int kMaxK = 15;
constexpr uint64_t kEnumSmall = 64, kEnumLimit = 1ull << 20;

struct NNTables {
  double step_h[256], step_s[256];  // NaN: no parameter
  double term_h[256], term_s[256];  // NaN: not a terminal-mismatch step
};
// global (not constant) memory: threads of a warp look up different steps, which the constant cache
// would serialise
__device__ NNTables c_nn;
// The same values as integers in units of 0.1 (every published value has one decimal), for the
// degenerate-site search: sums of them are exact in any arithmetic.  kNoParam marks a missing entry.
constexpr int16_t kNoParam = INT16_MIN;
struct NNTablesI {
  int16_t step_h[256], step_s[256];
  int16_t term_h[256], term_s[256];
};
__device__ NNTablesI c_nni;

int code_of(char c) {  // A=0, C=1, T=2, G=3
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'T': return 2;
    default: return 3;
  }
}
int idx4(int a, int b, int x, int y) { return a * 64 + b * 16 + x * 4 + y; }

uint8_t iupac_set(char ch) {
  switch (toupper((unsigned char)ch)) {
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

void build_tables(NNTables* t) {
  const double nan = std::nan("");
  for (int i = 0; i < 256; ++i) t->step_h[i] = t->step_s[i] = t->term_h[i] = t->term_s[i] = nan;
  // step lookup: internal-mismatch entry as written, then read from the other strand, then the
  // Watson-Crick entry as written, then read from the other strand
  auto put = [&](const Step* v, int n, bool reversed) {
    for (int i = 0; i < n; ++i) {
      const Step& s = v[i];
      int k = reversed ? idx4(code_of(s.y), code_of(s.x), code_of(s.b), code_of(s.a))
                       : idx4(code_of(s.a), code_of(s.b), code_of(s.x), code_of(s.y));
      if (std::isnan(t->step_h[k])) {
        t->step_h[k] = s.dh;
        t->step_s[k] = s.ds;
      }
    }
  };
  put(kInternal, sizeof kInternal / sizeof kInternal[0], false);
  put(kInternal, sizeof kInternal / sizeof kInternal[0], true);
  put(kStacks, sizeof kStacks / sizeof kStacks[0], false);
  put(kStacks, sizeof kStacks / sizeof kStacks[0], true);
  for (const Step& s : kTerminal) {
    int k = idx4(code_of(s.a), code_of(s.b), code_of(s.x), code_of(s.y));
    t->term_h[k] = s.dh;
    t->term_s[k] = s.ds;
  }
}

std::mutex g_tables_mu;
bool g_tables_loaded[64] = {};

ah_status load_tables(ah_ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_tables_mu);
  if (ctx->device < 64 && g_tables_loaded[ctx->device]) return AH_OK;
  static NNTables host;
  static NNTablesI host_i;
  build_tables(&host);
  auto tenths = [](double x) -> int16_t {
    if (std::isnan(x)) return kNoParam;
    const double t = std::round(x * 10.0);
    return (int16_t)t;
  };
  for (int i = 0; i < 256; ++i) {
    host_i.step_h[i] = tenths(host.step_h[i]), host_i.step_s[i] = tenths(host.step_s[i]);
    host_i.term_h[i] = tenths(host.term_h[i]), host_i.term_s[i] = tenths(host.term_s[i]);
  }
  AH_CUDA(ctx, cudaMemcpyToSymbolAsync(c_nn, &host, sizeof host, 0, cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaMemcpyToSymbolAsync(c_nni, &host_i, sizeof host_i, 0, cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->device < 64) g_tables_loaded[ctx->device] = true;
  return AH_OK;
}

// run constants computed once on the host
struct TmRun {
  double rlnk;        // R ln(C)
  double ln_mon;      // ln of the monovalent-equivalent concentration (M)
  double corr_const;  // methods 1-4: Tm correction
  // methods 6 and 7: correction to 1/Tm, rc0 + rc1 f + rc2 / (2 (L - 1)) with f the G/C fraction
  double rc0, rc1, rc2;
  double sym_h, sym_s;  // self-complementary duplexes: the symmetry terms (else 0)
  int saltcorr;
  int variants;       // 1: degenerate site Tm over the variants matching the site only
};

// Free Mg2+ (M) beside dNTPs binding it one to one, association constant 3e4 per M (Owczarzy et al.
// 2008): the positive root of Ka x^2 + (Ka (dNTP - Mg) + 1) x - Mg = 0.
double free_magnesium(double mg, double dntps) {
  if (!(dntps > 0.0)) return mg;
  const double ka = 3e4, b = ka * (dntps - mg) + 1.0;
  return (-b + std::sqrt(b * b + 4.0 * ka * mg)) / (2.0 * ka);
}

ah_status make_run(ah_ctx* ctx, const ah_tm_params* p, TmRun* r) {
  if (p->variants != 0 && p->variants != 1) return fail(ctx, AH_EINVAL, "Tm: variants must be 0 or 1");
  if (p->selfcomp != 0 && p->selfcomp != 1) return fail(ctx, AH_EINVAL, "Tm: selfcomp must be 0 or 1");
  double mon_mM = p->Na + p->K + p->Tris / 2.0;
  // Na+-equivalent of Mg2+ (von Ahsen et al. 2001) for methods 1-6; method 7 models Mg2+ itself
  if (p->saltcorr != 7 && (p->K + p->Mg + p->Tris + p->dNTPs) > 0 && p->dNTPs < p->Mg)
    mon_mM += 120.0 * std::sqrt(p->Mg - p->dNTPs);
  const double mon = mon_mM * 1e-3;
  const double mg = free_magnesium(p->Mg * 1e-3, p->dNTPs * 1e-3);
  if (p->saltcorr >= 1 && p->saltcorr <= 6 && !(mon > 0))
    return fail(ctx, AH_EINVAL, "Tm: salt correction needs a positive cation concentration");
  if (p->saltcorr == 7 && !(mon > 0) && !(mg > 0))
    return fail(ctx, AH_EINVAL, "Tm: salt method 7 needs monovalent ions or free Mg2+");
  const double conc = (p->selfcomp ? p->dnac1 : p->dnac1 - p->dnac2 / 2.0) * 1e-9;
  if (!(conc > 0)) return fail(ctx, AH_EINVAL, "Tm: strand concentrations give C <= 0");
  r->rlnk = 1.987 * std::log(conc);
  r->ln_mon = mon > 0 ? std::log(mon) : 0.0;
  r->saltcorr = p->saltcorr;
  r->variants = p->variants;
  r->sym_h = p->selfcomp ? kSymH : 0.0;
  r->sym_s = p->selfcomp ? kSymS : 0.0;
  r->corr_const = r->rc0 = r->rc1 = r->rc2 = 0.0;
  const double lm = r->ln_mon;
  switch (p->saltcorr) {
    case 1: r->corr_const = 16.6 * std::log10(mon); break;
    case 2: r->corr_const = 16.6 * std::log10(mon / (1.0 + 0.7 * mon)); break;
    case 3: r->corr_const = 12.5 * std::log10(mon); break;
    case 4: r->corr_const = 11.7 * std::log10(mon); break;
    case 6:  // Owczarzy et al. 2004
      r->rc0 = -3.95e-5 * lm + 9.40e-6 * lm * lm;
      r->rc1 = 4.29e-5 * lm;
      break;
    case 7: {  // Owczarzy et al. 2008: by the ratio sqrt([Mg2+]) / [Mon+]
      if (mon > 0 && std::sqrt(mg) / mon < 0.22) {  // monovalent ions dominate: the 2004 form
        r->rc0 = -3.95e-5 * lm + 9.40e-6 * lm * lm;
        r->rc1 = 4.29e-5 * lm;
        break;
      }
      double a = 3.92e-5, d = 1.42e-5, g = 8.31e-5;
      if (mon > 0 && std::sqrt(mg) / mon < 6.0) {  // mixed: monovalent ions modify a, d, g
        a *= 0.843 - 0.352 * std::sqrt(mon) * lm;
        d *= 1.279 - 4.03e-3 * lm - 8.03e-3 * lm * lm;
        g *= 0.486 - 0.258 * lm + 5.25e-3 * lm * lm * lm;
      }
      const double lg = std::log(mg);
      r->rc0 = a - 9.11e-6 * lg;
      r->rc1 = 6.26e-5 + d * lg;
      r->rc2 = -4.82e-4 + 5.25e-4 * lg + g * lg * lg;
      break;
    }
    default: break;
  }
  return AH_OK;
}

// Tm from the duplex sums (dH kcal/mol, dS cal/(K mol), before salt and concentration terms) and the
// variant's G/C count: symmetry terms, salt correction, Tm = 1000 dH / (dS + R ln C) - 273.15
__device__ __forceinline__ double tm_of_sums(double dh, double ds, int gc, int L, const TmRun& R) {
  dh += R.sym_h;
  ds += R.sym_s;
  if (R.saltcorr == 5) ds += 0.368 * (double)(L - 1) * R.ln_mon;
  double t = (1000.0 * dh) / (ds + R.rlnk) - 273.15;
  if (R.saltcorr >= 1 && R.saltcorr <= 4) t += R.corr_const;
  if (R.saltcorr >= 6) {
    const double corr = R.rc0 + R.rc1 * ((double)gc / (double)L) + R.rc2 / (2.0 * (double)(L - 1));
    t = 1.0 / (1.0 / (t + 273.15) + corr) - 273.15;
  }
  return t;
}

// Tm of variant v (codes, 5'->3') over c (codes of the opposite strand, 3'->5'); false if undefined
__device__ bool duplex_tm(const uint8_t* v, const uint8_t* c, int L, const TmRun& R, double* tm) {
  double dh = 0.0, ds = 0.0;
  int lo = 0, hi = L;
  {
    // left end read from the opposite strand: 5'-c1 c0-3' over 3'-v1 v0-5'
    const int k = c[1] * 64 + c[0] * 16 + v[1] * 4 + v[0];
    const double th = __ldg(&c_nn.term_h[k]);
    if (!isnan(th)) {
      dh += th;
      ds += __ldg(&c_nn.term_s[k]);
      lo = 1;
    }
  }
  if (hi - lo >= 2) {
    const int k = v[L - 2] * 64 + v[L - 1] * 16 + c[L - 2] * 4 + c[L - 1];
    const double th = __ldg(&c_nn.term_h[k]);
    if (!isnan(th)) {
      dh += th;
      ds += __ldg(&c_nn.term_s[k]);
      hi = L - 1;
    }
  }
  // initiation, from the variant's own end bases (A=0, C=1, T=2, G=3: A/T have bit 0 clear)
  dh += kInitH;
  ds += kInitS;
  int gc = 0;
  for (int j = 0; j < L; ++j) gc += v[j] & 1;
  if (gc == 0) {
    dh += kAllATH;
    ds += kAllATS;
  } else {
    dh += kOneGCH;
    ds += kOneGCS;
  }
  if (v[0] == 2) {  // 5' T
    dh += k5TAH;
    ds += k5TAS;
  }
  if (v[L - 1] == 0) {  // 3' A
    dh += k5TAH;
    ds += k5TAS;
  }
  if (v[0] & 1) { dh += kTermGCH; ds += kTermGCS; } else { dh += kTermATH; ds += kTermATS; }
  if (v[L - 1] & 1) { dh += kTermGCH; ds += kTermGCS; } else { dh += kTermATH; ds += kTermATS; }
  for (int i = lo; i + 1 < hi; ++i) {
    const int k = v[i] * 64 + v[i + 1] * 16 + c[i] * 4 + c[i + 1];
    const double sh = __ldg(&c_nn.step_h[k]);
    if (isnan(sh)) return false;
    dh += sh;
    ds += __ldg(&c_nn.step_s[k]);
  }
  *tm = tm_of_sums(dh, ds, gc, L, R);
  return true;
}

// the end-dependent initiation terms in tenths
constexpr int tenths_of(double x) { return (int)(x * 10.0 + (x >= 0 ? 0.5 : -0.5)); }
constexpr int kTermATH10 = tenths_of(kTermATH), kTermATS10 = tenths_of(kTermATS);
constexpr int kTermGCH10 = tenths_of(kTermGCH), kTermGCS10 = tenths_of(kTermGCS);
constexpr int k5TAH10 = tenths_of(k5TAH), k5TAS10 = tenths_of(k5TAS);

// nearest-neighbour sums (tenths) of edge (i, i+1) of the variant chain for bases (a, b) at
// positions i, i+1 over the opposite-strand codes c: the terminal-mismatch entry replaces the stack
// at either end; false when the step has no parameter
__device__ __forceinline__ bool edge_sums(int i, int L, uint8_t a, uint8_t b, const uint8_t* c, int* dh, int* ds) {
  if (i == 0) {
    const int k = c[1] * 64 + c[0] * 16 + b * 4 + a;  // left end read from the opposite strand
    const int th = __ldg(&c_nni.term_h[k]);
    if (th != kNoParam) {
      *dh = th;
      *ds = __ldg(&c_nni.term_s[k]);
      return true;
    }
  }
  if (i == L - 2) {
    const int k = a * 64 + b * 16 + c[L - 2] * 4 + c[L - 1];
    const int th = __ldg(&c_nni.term_h[k]);
    if (th != kNoParam) {
      *dh = th;
      *ds = __ldg(&c_nni.term_s[k]);
      return true;
    }
  }
  const int k = a * 64 + b * 16 + c[i] * 4 + c[i + 1];
  const int sh = __ldg(&c_nni.step_h[k]);
  if (sh == kNoParam) return false;
  *dh = sh;
  *ds = __ldg(&c_nni.step_s[k]);
  return true;
}

// initiation terms (tenths) that depend on the variant's end bases
__device__ __forceinline__ void end_sums(int j, int L, uint8_t v, int* dh, int* ds) {
  *dh = (v & 1) ? kTermGCH10 : kTermATH10;
  *ds = (v & 1) ? kTermGCS10 : kTermATS10;
  if (j == 0 && v == 2) *dh += k5TAH10, *ds += k5TAS10;       // 5' T
  if (j == L - 1 && v == 0) *dh += k5TAH10, *ds += k5TAS10;   // 3' A
}

// The variants that count at a site (reading R14): per position the primer's codes, only the site's
// own base inside the 3' clamp; at most k positions may differ from the site (k < 0: no limit).
struct SiteVariants {
  uint8_t s[32], c[32], ch[32][4], nch[32];
  int L, k;  // k = -1 when every combination of choices qualifies
};

// false when some position has no choice (the site breaks the clamp or a primer code)
__device__ bool site_variants(const uint8_t* sets, const uint8_t* s, int L, int k, int clamp, SiteVariants* V) {
  V->L = L;
  V->k = k >= L ? -1 : k;
  for (int j = 0; j < L; ++j) {
    V->s[j] = s[j];
    V->c[j] = s[j] ^ 2u;  // complement code
    V->nch[j] = 0;
    for (int code = 0; code < 4; ++code)
      if (((sets[j] >> code) & 1) && (j < L - clamp || code == s[j])) V->ch[j][V->nch[j]++] = (uint8_t)code;
    if (!V->nch[j]) return false;
  }
  return true;
}

// number of qualifying variants, saturating at `cap` + 1
__device__ uint64_t count_variants(const SiteVariants& V, uint64_t cap) {
  uint64_t cnt[kMaxK + 1] = {1};
  const int K = V.k < 0 ? 0 : V.k;
  for (int j = 0; j < V.L; ++j) {
    uint64_t nx[kMaxK + 1] = {0};
    for (int a = 0; a < V.nch[j]; ++a) {
      const int inc = V.k >= 0 && V.ch[j][a] != V.s[j];
      for (int m = 0; m + inc <= K; ++m) nx[m + inc] = min(cap + 1, nx[m + inc] + cnt[m]);
    }
    for (int m = 0; m <= K; ++m) cnt[m] = nx[m];
  }
  uint64_t t = 0;
  for (int m = 0; m <= K; ++m) t = min(cap + 1, t + cnt[m]);
  return t;
}

// Tm of a variant from its exact sums (tenths) and G/C count
__device__ __forceinline__ double tm_of_tenths(int dh10, int ds10, int gc, int L, const TmRun& R) {
  const double dh = 0.1 * dh10 + kInitH + (gc ? kOneGCH : kAllATH);
  const double ds = 0.1 * ds10 + kInitS + (gc ? kOneGCS : kAllATS);
  return tm_of_sums(dh, ds, gc, L, R);
}

// Maximum Tm over the qualifying variants by depth-first enumeration.  The walk adds one position's
// terms per step (the end terms at both ends, the edge to the previous base in between), so variants
// share the sums of their common prefix; a prefix whose last edge has no parameter is undefined for
// every variant below it and is cut, and so is one over the mismatch budget.  Sums are exact
// integers (tenths); each variant's Tm is one division.
__device__ bool enum_max(const SiteVariants& V, const TmRun& R, double* out) {
  int8_t idx[32];
  uint8_t mm[33], gcs[33], v[32];
  int sh[33], ss[33];  // sums of the terms of positions < j
  const int L = V.L;
  double best = -INFINITY;
  bool any = false;
  int j = 0;
  idx[0] = -1;
  mm[0] = gcs[0] = 0;
  sh[0] = ss[0] = 0;
  while (j >= 0) {
    if (++idx[j] >= V.nch[j]) {
      --j;
      continue;
    }
    const uint8_t b = V.ch[j][idx[j]];
    const int m = mm[j] + (V.k >= 0 && b != V.s[j]);
    if (V.k >= 0 && m > V.k) continue;
    int eh, es;
    if (j == 0) {
      end_sums(0, L, b, &eh, &es);
    } else if (!edge_sums(j - 1, L, v[j - 1], b, V.c, &eh, &es)) {
      continue;
    }
    const int dh = sh[j] + eh, ds = ss[j] + es;
    v[j] = b;
    const int gc = gcs[j] + (b & 1);
    if (j == L - 1) {
      end_sums(L - 1, L, b, &eh, &es);
      any = true;
      best = fmax(best, tm_of_tenths(dh + eh, ds + es, gc, L, R));
      continue;
    }
    sh[j + 1] = dh;
    ss[j + 1] = ds;
    gcs[j + 1] = (uint8_t)gc;
    mm[j + 1] = (uint8_t)m;
    ++j;
    idx[j] = -1;
  }
  *out = best;
  return any;
}

enum ChainResult { kChainOk, kChainUndefined, kChainUnbounded };

// One Viterbi pass over the chain of qualifying variants: the best score A * dS10 - B * dH10 (sums in
// tenths) in score arithmetic T over the variants, and that variant's exact sums in dh10/ds10, carried
// forward with each state (no backtracking).  T is float for the search passes and int64 (fixed
// point) for the confirming pass.  States are (position, base, mismatches so far), at most
// 4 x (k + 1) per position.
template <typename T>
__device__ __forceinline__ T no_score();
template <>
__device__ __forceinline__ float no_score<float>() { return -INFINITY; }
template <>
__device__ __forceinline__ double no_score<double>() { return -INFINITY; }
template <>
__device__ __forceinline__ long long no_score<long long>() { return LLONG_MIN; }

template <typename T>
__device__ bool chain_viterbi(const SiteVariants& V, T A, T B, T* best_score, int* dh10, int* ds10) {
  constexpr int M = kMaxK + 1;
  const int L = V.L, K = V.k < 0 ? 0 : V.k, W = K + 1;  // a base's states: mismatch counts 0..K
  auto inc = [&](int j, int a) { return (V.k >= 0 && V.ch[j][a] != V.s[j]) ? 1 : 0; };
  // state (base a, count m) at a * W + m: the best score (no_score: unreachable) and that path's
  // sums packed as dh10 * 65536 + ds10 (|sums| < 2^15 tenths, so packed sums add exactly)
  const T none = no_score<T>();
  T cur[4 * M], nxt[4 * M];
  int32_t cs[4 * M], ns[4 * M];
  for (int x = 0; x < 4 * W; ++x) cur[x] = none;
  for (int a = 0; a < V.nch[0]; ++a) {
    int dh, ds;
    end_sums(0, L, V.ch[0][a], &dh, &ds);
    const int x = a * W + inc(0, a);
    cur[x] = A * (T)ds - B * (T)dh;
    cs[x] = dh * 65536 + ds;
  }
  for (int i = 0; i + 1 < L; ++i) {
    for (int x = 0; x < 4 * W; ++x) nxt[x] = none;
    for (int b = 0; b < V.nch[i + 1]; ++b) {
      const int ib = inc(i + 1, b);
      int th = 0, ts = 0;
      if (i + 1 == L - 1) end_sums(L - 1, L, V.ch[i + 1][b], &th, &ts);
      for (int a = 0; a < V.nch[i]; ++a) {
        int dh, ds;
        if (!edge_sums(i, L, V.ch[i][a], V.ch[i + 1][b], V.c, &dh, &ds)) continue;
        dh += th, ds += ts;
        const T w = A * (T)ds - B * (T)dh;
        const int32_t pw = dh * 65536 + ds;
        for (int m = 0; m + ib <= K; ++m) {
          const T c = cur[a * W + m];
          if (c == none) continue;
          const T sc = c + w;
          const int y = b * W + m + ib;
          if (sc > nxt[y]) nxt[y] = sc, ns[y] = cs[a * W + m] + pw;
        }
      }
    }
    for (int x = 0; x < 4 * W; ++x) cur[x] = nxt[x], cs[x] = ns[x];
  }
  int arg = -1;
  for (int x = 0; x < 4 * W; ++x)
    if (cur[x] != none && (arg < 0 || cur[x] > cur[arg])) arg = x;
  if (arg < 0) return false;
  *best_score = cur[arg];
  const int32_t p = cs[arg];
  *ds10 = (int16_t)(p & 0xffff);
  *dh10 = (p - *ds10) / 65536;
  return true;
}

// Exact maximum of Tm over the qualifying variants for salt methods 0-5 and L >= 3.
// Tm + 273.15 = N(v) / D(v) with N = 1000 dH and D = dS + S0 < 0, and every term of N and D depends on
// at most two adjacent variant bases.  Dinkelbach's iteration for fractional programmes: for the
// current ratio lam, a Viterbi pass over the chain finds the variant maximising lam * D - N; its
// ratio becomes the next lam; at the optimum the maximum is 0.  Every published parameter has one
// decimal, so the passes carry exact integer sums (tenths) and each candidate's ratio is one exact
// division.  The search passes score in single precision; the optimum is confirmed by a pass in
// 64-bit fixed point (lam scaled by 2^36, products of integers exact), which continues the
// iteration should single precision have stopped short.  The sign check (the largest dS) is exact in
// single precision: its scores are integer sums far below 2^24.  kChainUnbounded when some
// qualifying variant could have D >= 0, where the iteration does not apply.
__device__ ChainResult site_tm_chain(const SiteVariants& V, const TmRun& R, double* out) {
  const int L = V.L;
    // constant part of D: salt (method 5) and R ln(C); methods 1-4 shift Tm by a constant
  const double S0 = (R.saltcorr == 5 ? 0.368 * (double)(L - 1) * R.ln_mon : 0.0) + R.rlnk;
  // all-A/T and one-G/C terms are equal here
  const double H0 = kInitH + kOneGCH + R.sym_h, Sc = kInitS + kOneGCS + R.sym_s;
  const double shift = R.saltcorr >= 1 && R.saltcorr <= 4 ? R.corr_const : 0.0;
  auto ratio = [&](int dh10, int ds10) { return 1000.0 * (0.1 * dh10 + H0) / (0.1 * ds10 + Sc + S0); };
  int dh10, ds10;
  float scf;
  // D must stay negative for every qualifying variant
  if (!chain_viterbi<float>(V, 1.f, 0.f, &scf, &dh10, &ds10)) return kChainUndefined;
  if (0.1 * ds10 + Sc + S0 >= 0.0) return kChainUnbounded;
  // start from the variant that maximises dS - dH / 300 (any defined variant works)
  if (!chain_viterbi<float>(V, 300.f, 1000.f, &scf, &dh10, &ds10)) return kChainUndefined;
  double lam = ratio(dh10, ds10);
  int best_h = dh10, best_s = ds10;
  // single-precision search: stop when a pass proposes no variant with a larger exact ratio
  for (int it = 0; it < 64; ++it) {
    if (!chain_viterbi<float>(V, (float)lam, 1000.f, &scf, &dh10, &ds10)) break;
    const double r = ratio(dh10, ds10);
    if (!(r > lam)) break;
    lam = r, best_h = dh10, best_s = ds10;
  }
  // Confirmation: no variant scores above the incumbent at lam (else continue from the better one).
  // Fixed point while |lam| < 4000 K keeps every path score below 2^62 (|sums| < 10^4 tenths);
  // beyond that, which only variants with D near 0 reach, double precision.
  constexpr double kScale = 68719476736.0;  // 2^36
  for (int it = 0; it < 64; ++it) {
    bool better;
    if (fabs(lam) < 4000.0) {
      const long long Lq = llrint(lam * kScale), Bq = (long long)(1000.0 * kScale);
      long long sc;
      if (!chain_viterbi<long long>(V, Lq, Bq, &sc, &dh10, &ds10)) break;
      better = sc > Lq * best_s - Bq * best_h;
    } else {
      double sc;
      if (!chain_viterbi<double>(V, lam, 1000.0, &sc, &dh10, &ds10)) break;
      const double inc = lam * best_s - 1000.0 * best_h;
      better = sc > inc + 1e-12 * fabs(inc);
    }
    if (!better) break;
    const double r = ratio(dh10, ds10);
    if (!(r > lam)) break;
    lam = r, best_h = dh10, best_s = ds10;
  }
  *out = lam + shift - 273.15;
  return kChainOk;
}

// Tm of a degenerate primer at a site (reading R14): the maximum over the primer's concrete variants
// with at most k mismatches to the site and none in the last `clamp` positions; NaN when none of them
// is defined.  Up to kEnumSmall qualifying variants are enumerated; more take the chain method (salt
// methods 0-5), and where that does not apply they are enumerated up to kEnumLimit.  Beyond that the
// site gets NaN and ST_TM_LIMIT is raised.
__device__ double site_tm(const uint8_t* sets, const uint8_t* s, int L, int k, int clamp, const TmRun& R,
                          uint32_t* status) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  SiteVariants V;
  if (!site_variants(sets, s, L, k, clamp, &V)) return nan;
  const uint64_t nv = count_variants(V, kEnumLimit);
  double t;
  if (nv > kEnumSmall && L >= 3 && R.saltcorr <= 5) {
    const ChainResult r = site_tm_chain(V, R, &t);
    if (r == kChainOk) return t;
    if (r == kChainUndefined) return nan;
  }
  if (nv > kEnumLimit) {
    if (status) atomicOr(status, (uint32_t)ST_TM_LIMIT);
    return nan;
  }
  return enum_max(V, R, &t) ? t : nan;
}

__device__ __forceinline__ uint8_t base_code(const uint2* planes, uint64_t group0, uint64_t x) {
  const uint2 w = planes[group0 + (x >> 5)];
  const uint32_t bit = (uint32_t)(x & 31);
  return (uint8_t)(((w.x >> bit) & 1u) | (((w.y >> bit) & 1u) << 1));
}

// Only the sites that some amplicon pairs need a Tm (an amplicon's Tm is the lower of its two
// sites'): the amplicons first write this word (a NaN no Tm computation returns) into hit_tm at
// their two sites, over an array cleared to zero, and the Tm kernel takes only the marked sites.
constexpr unsigned long long kSiteWanted = 0xFFFFFFFFFFFFFFFFull;

__global__ void k_mark_sites(const ah_amplicon* __restrict__ a, uint64_t n, double* __restrict__ hit_tm,
                             const uint64_t* __restrict__ d_n = nullptr) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (d_n ? min(n, *d_n) : n)) return;
  const uint2 hij = *reinterpret_cast<const uint2*>(&a[i]);  // hit_i, hit_j
  reinterpret_cast<unsigned long long*>(hit_tm)[hij.x] = kSiteWanted;
  reinterpret_cast<unsigned long long*>(hit_tm)[hij.y] = kSiteWanted;
}

// Sites arrive in (pair, record, pos, orient) order, so neighbouring sites alternate between the
// pair's two primers, whose chains differ in shape.  Each block first sorts its sites by primer in
// shared memory (bitonic, kTmBlock keys), so that a warp walks one primer's chain in step.
constexpr int kTmBlock = 128;

__global__ void __launch_bounds__(kTmBlock) k_tm_hits(const ah_hit* __restrict__ hits, uint64_t n,
                          const uint2* __restrict__ planes,
                          const uint64_t* __restrict__ rec_group, const uint8_t* __restrict__ plen,
                          const uint8_t* __restrict__ psets, const uint8_t* __restrict__ pk, int clamp,
                          const TmRun R, double* __restrict__ out, uint32_t* status,
                          const uint64_t* __restrict__ d_n = nullptr) {
  __shared__ uint32_t keys[kTmBlock];
  const uint64_t base = (uint64_t)blockIdx.x * kTmBlock;
  const uint64_t n_here = d_n ? min(n, *d_n) : n;
  {
    const uint64_t i = base + threadIdx.x;
    // key: primer (pair * 2 + primer, < 512), then the site's slot in the block; empty slots and
    // sites no amplicon pairs last
    const bool wanted = i < n_here && (unsigned long long)__double_as_longlong(out[i]) == kSiteWanted;
    keys[threadIdx.x] = wanted ? (((uint32_t)(hits[i].pattern >> 2) * 2u + (hits[i].pattern & 1u)) << 16) |
                                     threadIdx.x
                               : 0xFFFFFFFFu;
  }
  __syncthreads();
  for (int size = 2; size <= kTmBlock; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int t = threadIdx.x, o = t ^ stride;
      if (o > t) {
        const uint32_t x = keys[t], y = keys[o];
        const bool up = (t & size) == 0;
        if ((x > y) == up) keys[t] = y, keys[o] = x;
      }
      __syncthreads();
    }
  const uint32_t key = keys[threadIdx.x];
  if (key == 0xFFFFFFFFu) return;
  const uint64_t i = base + (key & 0xFFFFu);
  const ah_hit h = hits[i];
  const int L = plen[h.pattern];
  const uint32_t pair = h.pattern >> 2, primer = h.pattern & 1u, strand = (h.pattern >> 1) & 1u;
  const uint64_t g0 = rec_group[h.record];
  uint8_t site[32], sets[32];
  for (int j = 0; j < L; ++j) {
    // site bases in the primer's 5'->3' orientation
    site[j] = strand == 0 ? base_code(planes, g0, (uint64_t)h.pos + j)
                          : (uint8_t)(base_code(planes, g0, (uint64_t)h.pos + L - 1 - j) ^ 2u);
    sets[j] = psets[(pair * 2 + primer) * 32 + j];
  }
  out[i] = R.variants ? site_tm(sets, site, L, pk[pair], clamp, R, status) : site_tm(sets, site, L, L, 0, R, status);
}

__global__ void k_tm_amps(ah_amplicon* __restrict__ a, uint64_t n, const double* __restrict__ hit_tm, int filter,
                          double min_tm, uint32_t* __restrict__ keep, const uint64_t* __restrict__ d_n = nullptr) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (d_n && i >= *d_n) {
    if (keep) keep[i] = 0;
    return;
  }
  ah_amplicon m = a[i];
  const double ti = hit_tm[m.hit_i], tj = hit_tm[m.hit_j];
  const bool undefined = isnan(ti) || isnan(tj);
  const double t = undefined ? __longlong_as_double(0x7ff8000000000000ll) : fmin(ti, tj);
  // bit0: the threshold decision (defined and Tm >= min_tm), bit1: Tm within 1e-9 C of min_tm, so
  // that the decision rests on the last digits of a double, bit2: undefined.  Without the filter
  // the list is not compacted and the bits only annotate.
  const bool pass = !undefined && t >= min_tm;
  uint8_t flags = 0;
  if (pass) flags |= 1;
  if (!undefined && fabs(t - min_tm) <= 1e-9) flags |= 2;
  if (undefined) flags |= 4;
  m.tm = t;
  m.flags = flags;
  a[i] = m;
  if (keep) keep[i] = (!filter || pass) ? 1u : 0u;
}

__global__ void k_compact_amps(const ah_amplicon* __restrict__ in, uint64_t n, const uint32_t* __restrict__ keep,
                               const uint64_t* __restrict__ off, ah_amplicon* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && keep[i]) out[off[i]] = in[i];
}

__global__ void k_tm_duplexes(const uint8_t* __restrict__ v, const uint8_t* __restrict__ c,
                              const uint32_t* __restrict__ len, uint32_t n, const TmRun R, double* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t;
  out[i] = duplex_tm(v + 32 * (uint64_t)i, c + 32 * (uint64_t)i, (int)len[i], R, &t)
               ? t
               : __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void k_tm_sites(const uint8_t* __restrict__ sets, const uint8_t* __restrict__ site,
                           const uint32_t* __restrict__ len, const uint8_t* __restrict__ kc, uint32_t n,
                           const TmRun R, double* __restrict__ out, uint32_t* status) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = site_tm(sets + 32 * (uint64_t)i, site + 32 * (uint64_t)i, (int)len[i], kc[2 * i], kc[2 * i + 1], R,
                   status);
}

}  // namespace

ah_status tm_sites(ah_ctx* ctx, uint32_t n, const char* const* primers, const char* const* sites, const uint8_t* k,
                   const uint8_t* clamp, const ah_tm_params* params, double* out) {
  ah_status st;
  if ((st = load_tables(ctx))) return st;
  TmRun R;
  if ((st = make_run(ctx, params, &R))) return st;
  if (n == 0) return AH_OK;
  std::vector<uint8_t> sets(32 * (size_t)n, 0), sv(32 * (size_t)n, 0), kc(2 * (size_t)n);
  std::vector<uint32_t> len(n);
  for (uint32_t i = 0; i < n; ++i) {
    const size_t L = strlen(primers[i]);
    if (L < 2 || L > 32 || strlen(sites[i]) != L) return fail(ctx, AH_EINVAL, "site %u: lengths must match, 2..32", i);
    const uint32_t ki = k ? k[i] : 255u, ci = clamp ? clamp[i] : 0u;
    if (ki > (uint32_t)kMaxK && ki < L)
      return fail(ctx, AH_EINVAL, "site %u: mismatch budget %u above %d and below the length", i, ki, kMaxK);
    if (ci > L) return fail(ctx, AH_EINVAL, "site %u: clamp %u longer than the primer", i, ci);
    kc[2 * (size_t)i] = (uint8_t)std::min<uint32_t>(ki, 255u);
    kc[2 * (size_t)i + 1] = (uint8_t)ci;
    for (size_t j = 0; j < L; ++j) {
      const char x = (char)toupper((unsigned char)sites[i][j]);
      const uint8_t set = iupac_set(primers[i][j]);
      if (!set || !strchr("ACGT", x) || !x) return fail(ctx, AH_EINVAL, "site %u: bad primer code or site base", i);
      sets[32 * (size_t)i + j] = set;
      sv[32 * (size_t)i + j] = (uint8_t)code_of(x);
    }
    len[i] = (uint32_t)L;
  }
  uint8_t *ds, *dv, *dk;
  uint32_t* dl;
  double* dout;
  if ((st = dalloc(ctx, &ds, sets.size())) || (st = dalloc(ctx, &dv, sv.size())) || (st = dalloc(ctx, &dl, n)) ||
      (st = dalloc(ctx, &dk, kc.size())) || (st = dalloc(ctx, &dout, n)))
    return st;
  AH_CUDA(ctx, cudaMemcpyAsync(ds, sets.data(), sets.size(), cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(dv, sv.data(), sv.size(), cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(dl, len.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(dk, kc.data(), kc.size(), cudaMemcpyHostToDevice, ctx->stream));
  k_tm_sites<<<(n + 63) / 64, 64, 0, ctx->stream>>>(ds, dv, dl, dk, n, R, dout, ctx->d_status);
  launched(ctx);
  AH_CUDA(ctx, cudaGetLastError());
  AH_CUDA(ctx, cudaMemcpyAsync(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  dfree(ctx, ds);
  dfree(ctx, dv);
  dfree(ctx, dl);
  dfree(ctx, dk);
  dfree(ctx, dout);
  return check_status(ctx);
}

static_assert(sizeof(TmRun) <= kTmRunBytes, "Tm run constants exceed a plan's buffer");

ah_status tm_prepare(ah_ctx* ctx, const ah_tm_params* params, void* run_out, size_t run_size) {
  ah_status st;
  if ((st = load_tables(ctx))) return st;
  if (run_size < sizeof(TmRun)) return fail(ctx, AH_EINTERNAL, "tm_prepare: buffer too small");
  return make_run(ctx, params, (TmRun*)run_out);
}

void launch_tm(cudaStream_t s, const void* run, const ah_hit* hits, uint64_t hit_cap, const uint64_t* d_nhits,
               const uint8_t* pk, int clamp, uint32_t* status, const uint2* planes, const uint64_t* rec_group, const uint8_t* plen, const uint8_t* psets, double* hit_tm,
               ah_amplicon* amps, uint64_t amp_cap, const uint64_t* d_namps, int filter, double min_tm, uint32_t* keep) {
  const TmRun R = *(const TmRun*)run;
  cudaMemsetAsync(hit_tm, 0, std::max<uint64_t>(1, hit_cap) * sizeof(double), s);
  k_mark_sites<<<(unsigned)std::max<uint64_t>(1, (amp_cap + 255) / 256), 256, 0, s>>>(amps, amp_cap, hit_tm, d_namps);
  k_tm_hits<<<(unsigned)std::max<uint64_t>(1, (hit_cap + kTmBlock - 1) / kTmBlock), kTmBlock, 0, s>>>(hits, hit_cap, planes, rec_group,
                                                                                  plen, psets, pk, clamp, R, hit_tm,
                                                                                  status, d_nhits);
  k_tm_amps<<<(unsigned)std::max<uint64_t>(1, (amp_cap + 255) / 256), 256, 0, s>>>(amps, amp_cap, hit_tm, filter,
                                                                                  min_tm, keep, d_namps);
}

void launch_compact_amps(cudaStream_t s, const ah_amplicon* in, uint64_t cap, const uint32_t* keep, const uint64_t* off,
                         ah_amplicon* out) {
  k_compact_amps<<<(unsigned)std::max<uint64_t>(1, (cap + 255) / 256), 256, 0, s>>>(in, cap, keep, off, out);
}

ah_status tm_filter(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, ah_amplicons* a,
                    const ah_tm_params* params) {
  ah_status st;
  if ((st = load_tables(ctx))) return st;
  TmRun R;
  if ((st = make_run(ctx, params, &R))) return st;
  double* hit_tm = nullptr;
  uint32_t* keep = nullptr;
  if ((st = dalloc(ctx, &hit_tm, h->n))) return st;
  if (h->n && a->n) {
    AH_CUDA(ctx, cudaMemsetAsync(hit_tm, 0, h->n * sizeof(double), ctx->stream));
    k_mark_sites<<<(unsigned)((a->n + 255) / 256), 256, 0, ctx->stream>>>(a->d, a->n, hit_tm);
    launched(ctx);
  }
  if (h->n && a->n)
    k_tm_hits<<<(unsigned)((h->n + kTmBlock - 1) / kTmBlock), kTmBlock, 0, ctx->stream>>>(h->d, h->n, b->planes, b->rec_group, p->d_plen,
                                                                      p->d_psets, p->d_pk, p->clamp, R, hit_tm,
                                                                      ctx->d_status);
  if (h->n && a->n) launched(ctx);
  if (params->filter && (st = dalloc(ctx, &keep, a->n))) return st;
  if (a->n)
    k_tm_amps<<<(unsigned)((a->n + 255) / 256), 256, 0, ctx->stream>>>(a->d, a->n, hit_tm, params->filter,
                                                                      params->min_tm, keep);
  if (a->n) launched(ctx);
  AH_CUDA(ctx, cudaGetLastError());
  if (params->filter) {
    uint64_t* off;
    if ((st = dalloc(ctx, &off, a->n + 1))) return st;
    if ((st = exclusive_scan_u32(ctx, keep, off, a->n))) return st;
    uint64_t kept = 0;
    if ((st = read_u64(ctx, off + a->n, &kept))) return st;
    ah_amplicon* nd;
    if ((st = dalloc(ctx, &nd, kept))) return st;
    if (a->n)
      k_compact_amps<<<(unsigned)((a->n + 255) / 256), 256, 0, ctx->stream>>>(a->d, a->n, keep, off, nd);
    if (a->n) launched(ctx);
    AH_CUDA(ctx, cudaGetLastError());
    dfree(ctx, a->d);
    dfree(ctx, off);
    a->d = nd;
    a->n = kept;
  }
  dfree(ctx, hit_tm);
  dfree(ctx, keep);
  return check_status(ctx);
}

ah_status tm_duplexes(ah_ctx* ctx, uint32_t n, const char* const* seqs, const char* const* cseqs,
                      const ah_tm_params* params, double* out) {
  ah_status st;
  if ((st = load_tables(ctx))) return st;
  TmRun R;
  if ((st = make_run(ctx, params, &R))) return st;
  if (n == 0) return AH_OK;
  std::vector<uint8_t> v(32 * (size_t)n, 0), c(32 * (size_t)n, 0);
  std::vector<uint32_t> len(n);
  for (uint32_t i = 0; i < n; ++i) {
    size_t L = strlen(seqs[i]);
    if (L < 2 || L > 32 || strlen(cseqs[i]) != L) return fail(ctx, AH_EINVAL, "duplex %u: lengths must match, 2..32", i);
    for (size_t j = 0; j < L; ++j) {
      char a = (char)toupper((unsigned char)seqs[i][j]), x = (char)toupper((unsigned char)cseqs[i][j]);
      if (!strchr("ACGT", a) || !strchr("ACGT", x) || !a || !x)
        return fail(ctx, AH_EINVAL, "duplex %u: only A, C, G, T are allowed", i);
      v[32 * (size_t)i + j] = (uint8_t)code_of(a);
      c[32 * (size_t)i + j] = (uint8_t)code_of(x);
    }
    len[i] = (uint32_t)L;
  }
  uint8_t *dv, *dc;
  uint32_t* dl;
  double* dout;
  if ((st = dalloc(ctx, &dv, v.size())) || (st = dalloc(ctx, &dc, c.size())) || (st = dalloc(ctx, &dl, n)) ||
      (st = dalloc(ctx, &dout, n)))
    return st;
  AH_CUDA(ctx, cudaMemcpyAsync(dv, v.data(), v.size(), cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(dc, c.data(), c.size(), cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaMemcpyAsync(dl, len.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
  k_tm_duplexes<<<(n + 127) / 128, 128, 0, ctx->stream>>>(dv, dc, dl, n, R, dout);
  launched(ctx);
  AH_CUDA(ctx, cudaGetLastError());
  AH_CUDA(ctx, cudaMemcpyAsync(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  dfree(ctx, dv);
  dfree(ctx, dc);
  dfree(ctx, dl);
  dfree(ctx, dout);
  return AH_OK;
}

}  // namespace ah
