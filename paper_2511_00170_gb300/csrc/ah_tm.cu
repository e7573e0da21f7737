// Melting-temperature stage (Section "Implementations": AHv2 reimplements Biopython's Tm_NN in
// double precision; Section "Primer degeneracy": Tm is evaluated for the primer's variants).
//
// Every site gets the maximum, over the concrete variants of its (degenerate) primer, of the
// nearest-neighbour Tm of the variant paired with the site; an amplicon gets the lower of its two
// site values.  All arithmetic is FP64: the Tm threshold decision needs it.  The parameter tables
// below are expanded on the host into direct lookups indexed by the four base codes of a step
// (top 5'-ab-3' over bottom 3'-xy-5'), so a step costs one constant-memory load.
#include <climits>
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

// The other Watson-Crick sets of Tm_NN (Biopython's DNA_NN1, DNA_NN2, DNA_NN4, RNA_NN1, R_DNA_NN1).
// Breslauer et al. 1986, PNAS 83:3746.
const Step kBreslauer86[] = {
    {'A', 'A', 'T', 'T', -9.1, -24.0}, {'A', 'T', 'T', 'A', -8.6, -23.9}, {'T', 'A', 'A', 'T', -6.0, -16.9},
    {'C', 'A', 'G', 'T', -5.8, -12.9}, {'G', 'T', 'C', 'A', -6.5, -17.3}, {'C', 'T', 'G', 'A', -7.8, -20.8},
    {'G', 'A', 'C', 'T', -5.6, -13.5}, {'C', 'G', 'G', 'C', -11.9, -27.8}, {'G', 'C', 'C', 'G', -11.1, -26.7},
    {'G', 'G', 'C', 'C', -11.0, -26.6},
};
// Sugimoto et al. 1996, Nucleic Acids Res 24:4501.
const Step kSugimoto96[] = {
    {'A', 'A', 'T', 'T', -8.0, -21.9}, {'A', 'T', 'T', 'A', -5.6, -15.2}, {'T', 'A', 'A', 'T', -6.6, -18.4},
    {'C', 'A', 'G', 'T', -8.2, -21.0}, {'G', 'T', 'C', 'A', -9.4, -25.5}, {'C', 'T', 'G', 'A', -6.6, -16.4},
    {'G', 'A', 'C', 'T', -8.8, -23.5}, {'C', 'G', 'G', 'C', -11.8, -29.0}, {'G', 'C', 'C', 'G', -10.5, -26.4},
    {'G', 'G', 'C', 'C', -10.9, -28.4},
};
// SantaLucia & Hicks 2004, Annu Rev Biophys Biomol Struct 33:415.
const Step kSantaLucia04[] = {
    {'A', 'A', 'T', 'T', -7.6, -21.3}, {'A', 'T', 'T', 'A', -7.2, -20.4}, {'T', 'A', 'A', 'T', -7.2, -21.3},
    {'C', 'A', 'G', 'T', -8.5, -22.7}, {'G', 'T', 'C', 'A', -8.4, -22.4}, {'C', 'T', 'G', 'A', -7.8, -21.0},
    {'G', 'A', 'C', 'T', -8.2, -22.2}, {'C', 'G', 'G', 'C', -10.6, -27.2}, {'G', 'C', 'C', 'G', -9.8, -24.4},
    {'G', 'G', 'C', 'C', -8.0, -19.9},
};
// RNA, Freier et al. 1986, PNAS 83:9373 (U as T).
const Step kFreier86[] = {
    {'A', 'A', 'T', 'T', -6.6, -18.4}, {'A', 'T', 'T', 'A', -5.7, -15.5}, {'T', 'A', 'A', 'T', -8.1, -22.6},
    {'C', 'A', 'G', 'T', -10.5, -27.8}, {'G', 'T', 'C', 'A', -10.2, -26.2}, {'C', 'T', 'G', 'A', -7.6, -19.2},
    {'G', 'A', 'C', 'T', -13.3, -35.5}, {'C', 'G', 'G', 'C', -8.0, -19.4}, {'G', 'C', 'C', 'G', -14.2, -34.9},
    {'G', 'G', 'C', 'C', -12.2, -29.7},
};
// RNA/DNA hybrids, Sugimoto et al. 1995, Biochemistry 34:11211: the written strand is the RNA (U
// as T), every step as written.
const Step kSugimoto95[] = {
    {'A', 'A', 'T', 'T', -7.8, -21.9}, {'A', 'C', 'T', 'G', -5.9, -12.3}, {'A', 'G', 'T', 'C', -9.1, -23.5},
    {'A', 'T', 'T', 'A', -8.3, -23.9}, {'C', 'A', 'G', 'T', -9.0, -26.1}, {'C', 'C', 'G', 'G', -9.3, -23.2},
    {'C', 'G', 'G', 'C', -16.3, -47.1}, {'C', 'T', 'G', 'A', -7.0, -19.7}, {'G', 'A', 'C', 'T', -5.5, -13.5},
    {'G', 'C', 'C', 'G', -8.0, -17.1}, {'G', 'G', 'C', 'C', -12.8, -31.9}, {'G', 'T', 'C', 'A', -7.8, -21.6},
    {'T', 'A', 'A', 'T', -7.8, -23.2}, {'T', 'C', 'A', 'G', -8.6, -22.9}, {'T', 'G', 'A', 'C', -10.4, -28.4},
    {'T', 'T', 'A', 'A', -11.5, -36.4},
};

// One nearest-neighbour set: its stacks and the scalar terms of Tm_NN's tables (dH kcal/mol, dS
// cal/(K mol)): every duplex (init), per terminal A.T and G.C pair of the written strand (at, gc),
// a duplex with some / no G or C (onegc, allat), each of a 5' T and a 3' A (t5a), the symmetry
// term of a self-complementary duplex (sym).  The internal and terminal mismatch tables are shared.
struct NNSet {
  const Step* stacks;
  int n_stacks;
  double init[2], at[2], gc[2], onegc[2], allat[2], t5a[2], sym[2];
};
// slots of the sets on the device; nn_table (Biopython's numbering) -> slot, -1: not built
constexpr int kNNSlots = 6;
const NNSet kNNSets[kNNSlots] = {
    {kStacks, 10, {0, 0}, {2.3, 4.1}, {0.1, -2.8}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},  // DNA_NN3
    {kBreslauer86, 10, {0, 0}, {0, 0}, {0, 0}, {0, -16.8}, {0, -20.1}, {0, 0}, {0, -1.3}},  // DNA_NN1
    {kSugimoto96, 10, {0.6, -9.0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},  // DNA_NN2
    {kSantaLucia04, 10, {0.2, -5.7}, {2.2, 6.9}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},  // DNA_NN4
    {kFreier86, 10, {0, -10.8}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},  // RNA_NN1
    {kSugimoto95, 16, {1.9, -3.9}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},  // R_DNA_NN1
};
int nn_slot(int nn_table) {
  switch (nn_table) {
    case 0: case 3: return 0;
    case 1: return 1;
    case 2: return 2;
    case 4: return 3;
    case 5: return 4;
    case 8: return 5;
    default: return -1;
  }
}

// degenerate site Tm: largest mismatch budget, and the enumeration bounds
constexpr int kMaxK = 15;
constexpr uint64_t kEnumSmall = 64, kEnumLimit = 1ull << 20;

struct NNTables {
  double step_h[256], step_s[256];  // NaN: no parameter
  double term_h[256], term_s[256];  // NaN: not a terminal-mismatch step
};
// global (not constant) memory: threads of a warp look up different steps, which the constant cache
// would serialise
__device__ NNTables c_nn[kNNSlots];
// The same values as integers in units of 0.1 (every published value has one decimal), for the
// degenerate-site search: sums of them are exact in any arithmetic.  kNoParam marks a missing entry.
constexpr int16_t kNoParam = INT16_MIN;
struct NNTablesI {
  int16_t step_h[256], step_s[256];
  int16_t term_h[256], term_s[256];
};
__device__ NNTablesI c_nni[kNNSlots];

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

void build_tables(NNTables* t, const NNSet& set) {
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
  put(set.stacks, set.n_stacks, false);
  put(set.stacks, set.n_stacks, true);
  for (const Step& s : kTerminal) {
    int k = idx4(code_of(s.a), code_of(s.b), code_of(s.x), code_of(s.y));
    t->term_h[k] = s.dh;
    t->term_s[k] = s.ds;
  }
}

std::mutex g_tables_mu;
bool g_tables_loaded[64] = {};
NNTablesI g_host_i[kNNSlots];                   // the integer tables as uploaded
const int32_t* g_tab_image[64][kNNSlots] = {};  // per device and set: TmTabs for the generated kernels

ah_status load_tables(ah_ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_tables_mu);
  if (ctx->device < 64 && g_tables_loaded[ctx->device]) return AH_OK;
  static NNTables host[kNNSlots];
  auto tenths = [](double x) -> int16_t {
    if (std::isnan(x)) return kNoParam;
    const double t = std::round(x * 10.0);
    return (int16_t)t;
  };
  for (int k = 0; k < kNNSlots; ++k) {
    build_tables(&host[k], kNNSets[k]);
    NNTablesI& host_i = g_host_i[k];
    for (int i = 0; i < 256; ++i) {
      host_i.step_h[i] = tenths(host[k].step_h[i]), host_i.step_s[i] = tenths(host[k].step_s[i]);
      host_i.term_h[i] = tenths(host[k].term_h[i]), host_i.term_s[i] = tenths(host[k].term_s[i]);
    }
  }
  AH_CUDA(ctx, cudaMemcpyToSymbolAsync(c_nn, host, sizeof host, 0, cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaMemcpyToSymbolAsync(c_nni, g_host_i, sizeof g_host_i, 0, cudaMemcpyHostToDevice, ctx->stream));
  AH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->device < 64) g_tables_loaded[ctx->device] = true;
  return AH_OK;
}

// run constants, packed sums, table layout, site codes and the per-site chain driver shared with the
// kernels generated at run time
#include "ah_tm_chain.cuh"

// Free Mg2+ (M) beside dNTPs binding it one to one, association constant 3e4 per M (Owczarzy et al.
// 2008): the positive root of Ka x^2 + (Ka (dNTP - Mg) + 1) x - Mg = 0.
double free_magnesium(double mg, double dntps) {
  if (!(dntps > 0.0)) return mg;
  const double ka = 3e4, b = ka * (dntps - mg) + 1.0;
  return (-b + std::sqrt(b * b + 4.0 * ka * mg)) / (2.0 * ka);
}

ah_status make_run(ah_ctx* ctx, const ah_tm_params* p, TmRun* r) {
  if (p->variants != 0 && p->variants != 1) return fail(ctx, AH_EINVAL, "Tm: variants must be 0 or 1");
  const int slot = nn_slot(p->nn_table);
  if (slot < 0)
    return fail(ctx, AH_EINVAL, "Tm: nearest-neighbour table %d is not available (0-5 and 8; RNA_NN2 and RNA_NN3 "
                "are not built)", p->nn_table);
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
  const NNSet& set = kNNSets[slot];
  r->nn = slot;
  r->sym_h = p->selfcomp ? set.sym[0] : 0.0;
  r->sym_s = p->selfcomp ? set.sym[1] : 0.0;
  r->init_h = set.init[0], r->init_s = set.init[1];
  r->at_h = set.at[0], r->at_s = set.at[1];
  r->gc_h = set.gc[0], r->gc_s = set.gc[1];
  r->onegc_h = set.onegc[0], r->onegc_s = set.onegc[1];
  r->allat_h = set.allat[0], r->allat_s = set.allat[1];
  r->t5a_h = set.t5a[0], r->t5a_s = set.t5a[1];
  r->gc_split = set.onegc[0] != set.allat[0] || set.onegc[1] != set.allat[1];
  r->h0 = set.init[0] + set.onegc[0] + r->sym_h;
  r->s0 = set.init[1] + set.onegc[1] + r->sym_s;
  auto tenth = [](double x) { return (int32_t)std::lround(x * 10.0); };
  for (int v = 0; v < 4; ++v) {  // A=0, C=1, T=2, G=3
    const double* e = (v & 1) ? set.gc : set.at;
    const int32_t h = tenth(e[0]), sd = tenth(e[1]);
    r->end_l[v] = (h + (v == 2 ? tenth(set.t5a[0]) : 0)) * 65536 + sd + (v == 2 ? tenth(set.t5a[1]) : 0);  // 5' T
    r->end_r[v] = (h + (v == 0 ? tenth(set.t5a[0]) : 0)) * 65536 + sd + (v == 0 ? tenth(set.t5a[1]) : 0);  // 3' A
  }
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
    const double th = __ldg(&c_nn[R.nn].term_h[k]);
    if (!isnan(th)) {
      dh += th;
      ds += __ldg(&c_nn[R.nn].term_s[k]);
      lo = 1;
    }
  }
  if (hi - lo >= 2) {
    const int k = v[L - 2] * 64 + v[L - 1] * 16 + c[L - 2] * 4 + c[L - 1];
    const double th = __ldg(&c_nn[R.nn].term_h[k]);
    if (!isnan(th)) {
      dh += th;
      ds += __ldg(&c_nn[R.nn].term_s[k]);
      hi = L - 1;
    }
  }
  // initiation, from the variant's own end bases (A=0, C=1, T=2, G=3: A/T have bit 0 clear)
  dh += R.init_h;
  ds += R.init_s;
  int gc = 0;
  for (int j = 0; j < L; ++j) gc += v[j] & 1;
  if (gc == 0) {
    dh += R.allat_h;
    ds += R.allat_s;
  } else {
    dh += R.onegc_h;
    ds += R.onegc_s;
  }
  if (v[0] == 2) {  // 5' T
    dh += R.t5a_h;
    ds += R.t5a_s;
  }
  if (v[L - 1] == 0) {  // 3' A
    dh += R.t5a_h;
    ds += R.t5a_s;
  }
  if (v[0] & 1) { dh += R.gc_h; ds += R.gc_s; } else { dh += R.at_h; ds += R.at_s; }
  if (v[L - 1] & 1) { dh += R.gc_h; ds += R.gc_s; } else { dh += R.at_h; ds += R.at_s; }
  for (int i = lo; i + 1 < hi; ++i) {
    const int k = v[i] * 64 + v[i + 1] * 16 + c[i] * 4 + c[i + 1];
    const double sh = __ldg(&c_nn[R.nn].step_h[k]);
    if (isnan(sh)) return false;
    dh += sh;
    ds += __ldg(&c_nn[R.nn].step_s[k]);
  }
  *tm = tm_of_sums(dh, ds, gc, L, R);
  return true;
}


// nearest-neighbour sums (tenths) of edge (i, i+1) of the variant chain for bases (a, b) at
// positions i, i+1 over the opposite-strand codes c: the terminal-mismatch entry replaces the stack
// at either end; false when the step has no parameter
__device__ __forceinline__ bool edge_sums(const NNTablesI& ti, int i, int L, uint8_t a, uint8_t b, const uint8_t* c,
                                          int* dh, int* ds) {
  if (i == 0) {
    const int k = c[1] * 64 + c[0] * 16 + b * 4 + a;  // left end read from the opposite strand
    const int th = __ldg(&ti.term_h[k]);
    if (th != kNoParam) {
      *dh = th;
      *ds = __ldg(&ti.term_s[k]);
      return true;
    }
  }
  if (i == L - 2) {
    const int k = a * 64 + b * 16 + c[L - 2] * 4 + c[L - 1];
    const int th = __ldg(&ti.term_h[k]);
    if (th != kNoParam) {
      *dh = th;
      *ds = __ldg(&ti.term_s[k]);
      return true;
    }
  }
  const int k = a * 64 + b * 16 + c[i] * 4 + c[i + 1];
  const int sh = __ldg(&ti.step_h[k]);
  if (sh == kNoParam) return false;
  *dh = sh;
  *ds = __ldg(&ti.step_s[k]);
  return true;
}

// initiation terms (tenths) that depend on the variant's end bases
__device__ __forceinline__ void end_sums(const TmRun& R, int j, int L, uint8_t v, int* dh, int* ds) {
  const int32_t p = j == 0 ? R.end_l[v] : R.end_r[v];
  *dh = unpack_dh(p);
  *ds = unpack_ds(p);
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
  const double dh = 0.1 * dh10 + R.init_h + (gc ? R.onegc_h : R.allat_h);
  const double ds = 0.1 * ds10 + R.init_s + (gc ? R.onegc_s : R.allat_s);
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
      end_sums(R, 0, L, b, &eh, &es);
    } else if (!edge_sums(c_nni[R.nn], j - 1, L, v[j - 1], b, V.c, &eh, &es)) {
      continue;
    }
    const int dh = sh[j] + eh, ds = ss[j] + es;
    v[j] = b;
    const int gc = gcs[j] + (b & 1);
    if (j == L - 1) {
      end_sums(R, L - 1, L, b, &eh, &es);
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
__device__ bool chain_viterbi(const SiteVariants& V, const TmRun& R, T A, T B, T* best_score, int* dh10, int* ds10) {
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
    end_sums(R, 0, L, V.ch[0][a], &dh, &ds);
    const int x = a * W + inc(0, a);
    cur[x] = A * (T)ds - B * (T)dh;
    cs[x] = dh * 65536 + ds;
  }
  for (int i = 0; i + 1 < L; ++i) {
    for (int x = 0; x < 4 * W; ++x) nxt[x] = none;
    for (int b = 0; b < V.nch[i + 1]; ++b) {
      const int ib = inc(i + 1, b);
      int th = 0, ts = 0;
      if (i + 1 == L - 1) end_sums(R, L - 1, L, V.ch[i + 1][b], &th, &ts);
      for (int a = 0; a < V.nch[i]; ++a) {
        int dh, ds;
        if (!edge_sums(c_nni[R.nn], i, L, V.ch[i][a], V.ch[i + 1][b], V.c, &dh, &ds)) continue;
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
  // every qualifying variant holds G or C, or the set's initiation does not depend on it
  const double H0 = R.h0, Sc = R.s0;
  const double shift = R.saltcorr >= 1 && R.saltcorr <= 4 ? R.corr_const : 0.0;
  auto ratio = [&](int dh10, int ds10) { return 1000.0 * (0.1 * dh10 + H0) / (0.1 * ds10 + Sc + S0); };
  int dh10, ds10;
  float scf;
  // D must stay negative for every qualifying variant
  if (!chain_viterbi<float>(V, R, 1.f, 0.f, &scf, &dh10, &ds10)) return kChainUndefined;
  if (0.1 * ds10 + Sc + S0 >= 0.0) return kChainUnbounded;
  // start from the variant that maximises dS - dH / 300 (any defined variant works)
  if (!chain_viterbi<float>(V, R, 300.f, 1000.f, &scf, &dh10, &ds10)) return kChainUndefined;
  double lam = ratio(dh10, ds10);
  int best_h = dh10, best_s = ds10;
  // single-precision search: stop when a pass proposes no variant with a larger exact ratio
  for (int it = 0; it < 64; ++it) {
    if (!chain_viterbi<float>(V, R, (float)lam, 1000.f, &scf, &dh10, &ds10)) break;
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
      if (!chain_viterbi<long long>(V, R, Lq, Bq, &sc, &dh10, &ds10)) break;
      better = sc > Lq * best_s - Bq * best_h;
    } else {
      double sc;
      if (!chain_viterbi<double>(V, R, lam, 1000.0, &sc, &dh10, &ds10)) break;
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
__device__ __noinline__ double site_tm(const uint8_t* sets, const uint8_t* s, int L, int k, int clamp, const TmRun& R,
                          uint32_t* status) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  SiteVariants V;
  if (!site_variants(sets, s, L, k, clamp, &V)) return nan;
  const uint64_t nv = count_variants(V, kEnumLimit);
  double t;
  bool some_gc = !R.gc_split;  // the chain's constant terms assume G or C in every variant
  for (int j = 0; j < L && !some_gc; ++j) {
    bool only = V.nch[j] > 0;
    for (int a = 0; a < V.nch[j]; ++a) only = only && (V.ch[j][a] & 1);
    some_gc = only;
  }
  if (nv > kEnumSmall && L >= 3 && R.saltcorr <= 5 && some_gc) {
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

// ---------------------------------------------------------------------------------------------
// Degenerate site Tm, one group of G lanes per site (G = 4, 8, 16 or 32 lanes of one warp).
//
// The chain of the variants only branches at the primer's degenerate positions: a position with a
// single choice contributes fixed terms.  So the chain is first compressed onto the D degenerate
// positions d_0 < ... < d_{D-1}: the sums of every edge between d_t and d_{t+1} are folded into one
// weight per pair of choices (a at d_t, b at d_{t+1}), those before d_0 into a weight per choice at
// d_0 and those after d_{D-1} into one per choice at d_{D-1}.  The weights are exact integer sums
// (tenths) packed as dH * 65536 + dS, computed once per site into shared memory; the passes then
// walk D - 1 steps instead of L - 1 and read no parameter table.  A step between two single-choice
// positions lies on every variant, so one without a parameter leaves the site undefined at once.
//
// In a pass, lane r of the group holds the state (base r / W, mismatches r % W), W = k + 1 with a
// mismatch budget k (else W = 1), and takes its best predecessor from the lanes of the previous
// position by shuffles.  The group's lanes share every loop bound, so they stay converged.
//
// The iteration is site_tm_chain's with two passes saved: the sign condition (every variant's
// entropy sum D < 0) is first tried with a bound (the sum of each step's largest dS), and the pass
// that finds the largest dS runs only when the bound does not settle it; after the start pass the
// iterations run in exact arithmetic at once (64-bit fixed point, double beyond 4000 K), so the pass
// that shows the optimum is also the one that proves it.  Sites whose chain does not apply (salt
// methods 6 and 7, L < 3, an entropy sum that could reach zero, state widths above G / 4) are handed
// whole to site_tm by the group's first lane.

struct TmGroupSh {      // per site, in shared memory; followed by the (D - 1) x 16 step weights
  uint8_t set[32];      // the primer's IUPAC sets (5'->3')
  uint8_t s[32];        // the site's base codes in the primer's orientation
  uint8_t c[32];        // their complements (the opposite strand, 3'->5')
  uint8_t ch[32];       // the choices that count at each position (the clamp holds the site's base)
  uint8_t dpos[32];     // the positions where the chain branches, in order
  int32_t pre[4], suf[4];
};
constexpr int kTmGroupHeadWords = (int)(sizeof(TmGroupSh) / 4);
static_assert(sizeof(TmGroupSh) % 16 == 0, "group header keeps 16-byte alignment");

// words of shared memory per site for chains of at most dmax branch positions; the stride is 4 more
// than a multiple of 32 words, so the groups of one warp read different banks
__host__ __device__ inline int tm_group_words(int dmax) {
  const int w = kTmGroupHeadWords + 16 * (dmax > 1 ? dmax - 1 : 0);
  return (w + 31) / 32 * 32 + 4;
}

__device__ __forceinline__ int fixed_base(uint32_t ch) { return __ffs(ch) - 1; }

// packed sums (tenths) of edge i with base x at i and y at i + 1, kNoEdge without a parameter
__device__ __forceinline__ int32_t edge_packed(const TmGroupSh& sh, const TmRun& R, int L, int i, int x, int y) {
  int eh, es;
  if (!edge_sums(c_nni[R.nn], i, L, (uint8_t)x, (uint8_t)y, sh.c, &eh, &es)) return kNoEdge;
  return eh * 65536 + es;
}

// One Viterbi pass of the compressed chain: the best score A * dS10 - B * dH10 over the qualifying
// variants and that variant's exact sums, the same in every lane of the group.
template <typename T, int G>
__device__ bool group_viterbi(const TmGroupSh& sh, const int32_t* __restrict__ w, int D, int W, int K, int m0,
                              int r, unsigned gmask, T A, T B, T* best, int* dh10, int* ds10) {
  const T none = no_score<T>();
  const bool live = r < 4 * W;
  const int b = live ? r / W : 0, m = live ? r % W : 0;
  T cur = none;
  int32_t cs = 0;
  uint32_t chp = sh.ch[sh.dpos[0]];
  {
    const int d0 = sh.dpos[0];
    const int mm = m0 + ((K >= 0 && b != sh.s[d0]) ? 1 : 0);
    if (live && ((chp >> b) & 1) && mm == m && sh.pre[b] != kNoEdge) {
      cs = sh.pre[b];
      cur = A * (T)unpack_ds(cs) - B * (T)unpack_dh(cs);
    }
  }
  for (int t = 0; t + 1 < D; ++t) {
    const int dn = sh.dpos[t + 1];
    const uint32_t chn = sh.ch[dn];
    const int ib = (K >= 0 && b != sh.s[dn]) ? 1 : 0;
    const int mp = m - ib;
    const bool ok = live && ((chn >> b) & 1) && mp >= 0;
    const int32_t* wt = w + t * 16 + b;
    T nx = none;
    int32_t ns = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (!((chp >> a) & 1)) continue;  // the same in every lane of the group
      const int src = a * W + (mp >= 0 ? mp : 0);
      const T c = __shfl_sync(gmask, cur, src, G);
      const int32_t pc = __shfl_sync(gmask, cs, src, G);
      const int32_t p = wt[a * 4];
      if (ok && c != none && p != kNoEdge) {
        const T sc = c + (A * (T)unpack_ds(p) - B * (T)unpack_dh(p));
        if (sc > nx) nx = sc, ns = pc + p;
      }
    }
    cur = nx, cs = ns, chp = chn;
  }
  if (cur != none) {
    const int32_t p = sh.suf[b];
    if (p == kNoEdge) {
      cur = none;
    } else {
      cur = cur + (A * (T)unpack_ds(p) - B * (T)unpack_dh(p));
      cs += p;
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const T oc = __shfl_xor_sync(gmask, cur, o, G);
    const int32_t ocs = __shfl_xor_sync(gmask, cs, o, G);
    if (oc > cur || (oc == cur && ocs > cs)) cur = oc, cs = ocs;
  }
  if (cur == none) return false;
  *best = cur;
  *ds10 = unpack_ds(cs);
  *dh10 = unpack_dh(cs);
  return true;
}

// Tm of the site held in sh (set, s and c filled, L its length) for a primer with mismatch budget k
// (k >= L: none) and clamp: the maximum over qualifying variants, as site_tm returns it.  Called by
// all G lanes of the group (lane r, mask gmask); w: the group's weight area (room for dmax - 1 steps).
template <int G>
__device__ double group_site_tm(TmGroupSh& sh, int32_t* w, int L, int k, int clamp, const TmRun& R, uint32_t* status,
                                int r, unsigned gmask) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const int K = k >= L ? -1 : k, W = K < 0 ? 1 : K + 1;
  // choices per position, the branch positions, and the fixed positions' mismatches
  uint32_t dmask = 0, empty = 0, fixed_mm = 0;
  for (int j = r; j < L; j += G) {
    uint8_t ch = sh.set[j];
    if (j >= L - clamp) ch &= (uint8_t)(1u << sh.s[j]);
    sh.ch[j] = ch;
    const int n = __popc(ch);
    if (n == 0) empty |= 1u << j;
    if (n >= 2) dmask |= 1u << j;
    if (n == 1 && K >= 0 && ch != (1u << sh.s[j])) fixed_mm |= 1u << j;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    dmask |= __shfl_xor_sync(gmask, dmask, o, G);
    empty |= __shfl_xor_sync(gmask, empty, o, G);
    fixed_mm |= __shfl_xor_sync(gmask, fixed_mm, o, G);
  }
  if (empty) return nan;
  const int m0 = __popc(fixed_mm);
  if (K >= 0 && m0 > K) return nan;
  if (R.saltcorr >= 6 || L < 3 || W * 4 > G || R.gc_split) {
    __syncwarp(gmask);
    double t = nan;
    if (r == 0) t = site_tm(sh.set, sh.s, L, k, clamp, R, status);
    return __shfl_sync(gmask, t, 0, G);
  }
  __syncwarp(gmask);
  {  // steps between two single-choice positions are on every variant
    bool bad = false;
    for (int i = r; i + 1 < L; i += G)
      if (!((dmask >> i) & 3u) && edge_packed(sh, R, L, i, fixed_base(sh.ch[i]), fixed_base(sh.ch[i + 1])) == kNoEdge)
        bad = true;
    if (__any_sync(gmask, bad)) return nan;
  }
  if (!dmask) dmask = 1;  // a concrete primer: a chain of one node with a single choice
  const int D = __popc(dmask);
  for (int t = r; t < D; t += G) {  // the t-th set bit of dmask
    uint32_t x = dmask;
    for (int q = 0; q < t; ++q) x &= x - 1;
    sh.dpos[t] = (uint8_t)(__ffs(x) - 1);
  }
  __syncwarp(gmask);
  // weights: before d_0, after d_{D-1}, and between consecutive branch positions
  if (r < 4) {
    const int d0 = sh.dpos[0], dl = sh.dpos[D - 1];
    int32_t p = kNoEdge, q = kNoEdge;
    if ((sh.ch[d0] >> r) & 1) {
      int eh, es;
      end_sums(R, 0, L, (uint8_t)(d0 == 0 ? r : fixed_base(sh.ch[0])), &eh, &es);
      p = eh * 65536 + es;
      for (int i = 0; i < d0; ++i)
        p = add_packed(p, edge_packed(sh, R, L, i, fixed_base(sh.ch[i]), i + 1 == d0 ? r : fixed_base(sh.ch[i + 1])));
    }
    if ((sh.ch[dl] >> r) & 1) {
      int eh, es;
      end_sums(R, L - 1, L, (uint8_t)(dl == L - 1 ? r : fixed_base(sh.ch[L - 1])), &eh, &es);
      q = eh * 65536 + es;
      for (int i = dl; i + 1 < L; ++i)
        q = add_packed(q, edge_packed(sh, R, L, i, i == dl ? r : fixed_base(sh.ch[i]), fixed_base(sh.ch[i + 1])));
    }
    sh.pre[r] = p;
    sh.suf[r] = q;
  }
  for (int t = r; t + 1 < D; t += G) {
    const int lo = sh.dpos[t], hi = sh.dpos[t + 1];
    const uint32_t cha = sh.ch[lo], chb = sh.ch[hi];
    int32_t* wt = w + t * 16;
    if (hi == lo + 1) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          wt[a * 4 + b] = ((cha >> a) & 1) && ((chb >> b) & 1) ? edge_packed(sh, R, L, lo, a, b) : kNoEdge;
    } else {
      // left step (choice a, then a fixed base), the fixed steps, right step (fixed base, then b)
      int32_t mid = 0, left[4], right[4];
      for (int i = lo + 1; i + 1 < hi; ++i)
        mid += edge_packed(sh, R, L, i, fixed_base(sh.ch[i]), fixed_base(sh.ch[i + 1]));  // defined: checked above
      const int fl = fixed_base(sh.ch[lo + 1]), fr = fixed_base(sh.ch[hi - 1]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        left[a] = (cha >> a) & 1 ? edge_packed(sh, R, L, lo, a, fl) : kNoEdge;
        right[a] = (chb >> a) & 1 ? edge_packed(sh, R, L, hi - 1, fr, a) : kNoEdge;
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) wt[a * 4 + b] = add_packed(add_packed(left[a], mid), right[b]);
    }
  }
  __syncwarp(gmask);
  // a bound on every variant's dS: each step's largest (tenths)
  int bound = 0;
  for (int t = r; t + 1 < D; t += G) {
    int mx = INT_MIN;
    for (int e = 0; e < 16; ++e) {
      const int32_t p = w[t * 16 + e];
      if (p != kNoEdge) mx = max(mx, unpack_ds(p));
    }
    bound += mx == INT_MIN ? 0 : mx;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) bound += __shfl_xor_sync(gmask, bound, o, G);
  {
    int mp = INT_MIN, ms = INT_MIN;
    for (int x = 0; x < 4; ++x) {
      if (sh.pre[x] != kNoEdge) mp = max(mp, unpack_ds(sh.pre[x]));
      if (sh.suf[x] != kNoEdge) ms = max(ms, unpack_ds(sh.suf[x]));
    }
    if (mp == INT_MIN || ms == INT_MIN) return nan;  // no choice at an end has its terms
    bound += mp + ms;
  }
  const double S0 = (R.saltcorr == 5 ? 0.368 * (double)(L - 1) * R.ln_mon : 0.0) + R.rlnk;
  const double H0 = R.h0, Sc = R.s0;
  const double shift = R.saltcorr >= 1 && R.saltcorr <= 4 ? R.corr_const : 0.0;
  auto ratio = [&](int dh10, int ds10) { return 1000.0 * (0.1 * dh10 + H0) / (0.1 * ds10 + Sc + S0); };
  int dh10, ds10;
  float scf;
  if (0.1 * bound + Sc + S0 >= 0.0) {  // the bound leaves the sign open: the largest dS itself
    if (!group_viterbi<float, G>(sh, w, D, W, K, m0, r, gmask, 1.f, 0.f, &scf, &dh10, &ds10)) return nan;
    if (0.1 * ds10 + Sc + S0 >= 0.0) {  // some variant's entropy sum could reach zero: enumerate
      double t = nan;
      if (r == 0) t = site_tm(sh.set, sh.s, L, k, clamp, R, status);
      return __shfl_sync(gmask, t, 0, G);
    }
  }
  // start from the variant that maximises dS - dH / 300 (any defined variant works)
  if (!group_viterbi<float, G>(sh, w, D, W, K, m0, r, gmask, 300.f, 1000.f, &scf, &dh10, &ds10)) return nan;
  double lam = ratio(dh10, ds10);
  int best_h = dh10, best_s = ds10;
  // exact iterations: a pass that finds no variant scoring above the incumbent at lam proves it
  // optimal; otherwise the better variant's ratio is the next lam
  constexpr double kScale = 68719476736.0;  // 2^36
  for (int it = 0; it < 64; ++it) {
    bool better;
    if (fabs(lam) < 4000.0) {
      const long long Lq = llrint(lam * kScale), Bq = (long long)(1000.0 * kScale);
      long long sc;
      if (!group_viterbi<long long, G>(sh, w, D, W, K, m0, r, gmask, Lq, Bq, &sc, &dh10, &ds10)) break;
      better = sc > Lq * best_s - Bq * best_h;
    } else {
      double sc;
      if (!group_viterbi<double, G>(sh, w, D, W, K, m0, r, gmask, lam, 1000.0, &sc, &dh10, &ds10)) break;
      const double inc = lam * best_s - 1000.0 * best_h;
      better = sc > inc + 1e-12 * fabs(inc);
    }
    if (!better) break;
    const double q = ratio(dh10, ds10);
    if (!(q > lam)) break;
    lam = q, best_h = dh10, best_s = ds10;
  }
  return lam + shift - 273.15;
}

// Only the sites that some amplicon pairs need a Tm (an amplicon's Tm is the lower of its two
// sites'): the amplicons first write kSiteWanted into hit_tm at their two sites, over an array
// cleared to zero, and the Tm kernels take only the marked sites.

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
                          const TmRun Rp, double* __restrict__ out, uint32_t* status,
                          const uint64_t* __restrict__ d_n = nullptr) {
  // the run constants in shared memory: device functions take them by reference, and a reference
  // to a kernel parameter would make the compiler copy it to local memory for every thread
  __shared__ TmRun R_sh;
  if (threadIdx.x == 0) R_sh = Rp;
  __syncthreads();
  const TmRun& R = R_sh;

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

// Whether edge i of a variant with bases x at i and y at i + 1 has a parameter, over the opposite
// strand cc (2-bit codes of position j at bits 2j); the lookups of edge_sums.
__device__ __forceinline__ bool edge_defined(const NNTablesI& ti, int i, int L, int x, int y, uint64_t cc) {
  const int c0 = (int)(cc >> (2 * i)) & 3, c1 = (int)(cc >> (2 * i + 2)) & 3;
  if (i == 0 && __ldg(&ti.term_h[c1 * 64 + c0 * 16 + y * 4 + x]) != kNoParam) return true;
  if (i == L - 2 && __ldg(&ti.term_h[x * 64 + y * 16 + c0 * 4 + c1]) != kNoParam) return true;
  return __ldg(&ti.step_h[x * 64 + y * 16 + c0 * 4 + c1]) != kNoParam;
}

// The group-per-site form of k_tm_hits.  A block takes a window of kTmWindow site slots, one per
// thread.  Each thread first settles its slot where that needs no chain: not wanted (no amplicon
// pairs it), or undefined (a site base outside the clamp's choice, too many fixed mismatches, or a
// step between single-choice positions without a parameter; the group repeats these checks).  The
// remaining sites are sorted by primer (so neighbouring groups walk chains of one shape) and taken
// by the block's S groups of G lanes in rounds.
// Shared memory: the window's keys and packed site codes, then S site areas of tm_group_words(dmax).
constexpr int kTmWindow = 128;

template <int G>
__global__ void __launch_bounds__(kTmWindow) k_tm_hits_g(const ah_hit* __restrict__ hits, uint64_t n,
                                                         const uint2* __restrict__ planes,
                                                         const uint64_t* __restrict__ rec_group,
                                                         const uint8_t* __restrict__ plen,
                                                         const uint8_t* __restrict__ psets,
                                                         const uint8_t* __restrict__ pk, int clamp, const TmRun Rp,
                                                         double* __restrict__ out, uint32_t* status, int dmax,
                                                         int n_groups, const uint64_t* __restrict__ d_n) {
  // the run constants in shared memory: device functions take them by reference, and a reference
  // to a kernel parameter would make the compiler copy it to local memory for every thread
  __shared__ TmRun R_sh;
  if (threadIdx.x == 0) R_sh = Rp;
  __syncthreads();
  const TmRun& R = R_sh;

  extern __shared__ __align__(16) uint32_t tm_smem[];
  uint32_t* keys = tm_smem;                                         // kTmWindow
  uint64_t* codes = reinterpret_cast<uint64_t*>(tm_smem + kTmWindow);  // kTmWindow
  uint32_t* areas = tm_smem + 3 * kTmWindow;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const uint64_t base = (uint64_t)blockIdx.x * kTmWindow;
  const uint64_t n_here = d_n ? min(n, *d_n) : n;
  {
    const int t = threadIdx.x;
    const uint64_t i = base + t;
    uint32_t key = 0xFFFFFFFFu;
    if (i < n_here && (unsigned long long)__double_as_longlong(out[i]) == kSiteWanted) {
      const ah_hit h = hits[i];
      const int L = plen[h.pattern];
      const uint32_t pair = h.pattern >> 2, primer = h.pattern & 1u, strand = (h.pattern >> 1) & 1u;
      // the site's bases over [pos, pos + L) (L <= 32 spans at most two plane words), in the primer's
      // orientation, 2 bits per position
      const uint64_t x0 = rec_group[h.record] * 32 + h.pos;
      const uint2 w0 = planes[x0 >> 5], w1 = planes[(x0 >> 5) + 1];
      const int sh0 = (int)(x0 & 31);
      const uint64_t lo = (((uint64_t)w1.x << 32) | w0.x) >> sh0, hi = (((uint64_t)w1.y << 32) | w0.y) >> sh0;
      uint64_t code = 0;
      for (int j = 0; j < L; ++j) {
        const int q = strand == 0 ? j : L - 1 - j;
        const uint64_t b = ((lo >> q) & 1u) | (((hi >> q) & 1u) << 1);
        code |= (strand == 0 ? b : b ^ 2u) << (2 * j);
      }
      const uint64_t cc = code ^ 0xAAAAAAAAAAAAAAAAull;  // complements: code ^ 2 per position
      const uint8_t* ps = psets + (pair * 2 + primer) * 32;
      const int kk = R.variants ? (int)pk[pair] : L, cl = R.variants ? clamp : 0;
      bool undefined = false;
      int mism = 0, prev = -1;  // prev: the fixed base of position j - 1 (-1: a choice)
      for (int j = 0; j < L && !undefined; ++j) {
        const int sj = (int)(code >> (2 * j)) & 3;
        uint32_t ch = ps[j];
        if (j >= L - cl) ch &= 1u << sj;
        if (!ch) undefined = true;
        const int cur = __popc(ch) == 1 ? fixed_base(ch) : -1;
        if (cur >= 0 && cur != sj) ++mism;
        if (j > 0 && cur >= 0 && prev >= 0 && !edge_defined(c_nni[R.nn], j - 1, L, prev, cur, cc)) undefined = true;
        prev = cur;
      }
      if (kk < L && mism > kk) undefined = true;
      if (undefined) {
        out[i] = nan;
      } else {
        key = ((pair * 2 + primer) << 16) | (uint32_t)t;
        codes[t] = code;
      }
    }
    keys[t] = key;
  }
  const int n_valid = __syncthreads_count(keys[threadIdx.x] != 0xFFFFFFFFu);
  if (n_valid == 0) return;
  for (int size = 2; size <= kTmWindow; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int t = threadIdx.x, o = t ^ stride;
      if (o > t) {
        const uint32_t x = keys[t], y = keys[o];
        const bool up = (t & size) == 0;
        if ((x > y) == up) keys[t] = y, keys[o] = x;
      }
      __syncthreads();
    }
  const int g = threadIdx.x / G, r = threadIdx.x % G;
  if (g >= n_groups) return;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  TmGroupSh& sh = *reinterpret_cast<TmGroupSh*>(areas + g * tm_group_words(dmax));
  int32_t* w = reinterpret_cast<int32_t*>(&sh + 1);
  for (int q = g; q < n_valid; q += n_groups) {
    const uint32_t t = keys[q] & 0xFFFFu;
    const uint64_t i = base + t;
    const ah_hit h = hits[i];
    const int L = plen[h.pattern];
    const uint32_t pair = h.pattern >> 2, primer = h.pattern & 1u;
    const uint64_t code = codes[t];
    __syncwarp(gmask);  // the previous round's reads of the area are done
    for (int j = r; j < L; j += G) {
      const uint8_t sj = (uint8_t)((code >> (2 * j)) & 3u);
      sh.s[j] = sj;
      sh.c[j] = sj ^ 2u;
      sh.set[j] = psets[(pair * 2 + primer) * 32 + j];
    }
    __syncwarp(gmask);
    const double tm = R.variants ? group_site_tm<G>(sh, w, L, pk[pair], clamp, R, status, r, gmask)
                                 : group_site_tm<G>(sh, w, L, L, 0, R, status, r, gmask);
    if (r == 0) out[i] = tm;
  }
}

// ---------------------------------------------------------------------------------------------
// Degenerate site Tm over every concrete variant (the default reading), one thread per site.
//
// With no mismatch budget the chain's states are the 4 bases, so a thread keeps them in registers
// and takes each step's transitions itself, a fraction of the instructions that lane groups spend
// on shuffles.  Sites come from the same pre-pass and sort by primer as in k_tm_hits_g, so the
// threads of a warp share the chain's shape (their loops have the same bounds) and warps are full.
// The compressed chain's step weights are stored per thread in shared memory, only for pairs of
// allowed choices and strided by the block size (a warp's accesses fall in different banks); the
// parameter tables are copied to shared memory; the passes score in integers: the start pass with
// the exact int32 score 280 dS - 1000 dH, the proving passes in 64-bit fixed point
// (chain_site_tm).  Sites the chain does not cover (salt methods 6 and 7, L < 3, an entropy sum
// that could reach zero) are enumerated by k_tm_deferred.  The kernels generated per primer set
// (ah_tm_jit.cpp) share the driver and the kernel body and replace only the chain's passes.

// table entry e = a * 64 + b * 16 + c * 4 + d (the step 5'-ab-3' over 3'-cd-5') into its TmTabs places
__host__ __device__ __forceinline__ void put_tab_entry(TmTabs& T, const NNTablesI& ti, int e) {
  const int a = e >> 6, b = (e >> 4) & 3, c = (e >> 2) & 3, d = e & 3;
  const int sh = ti.step_h[e], th = ti.term_h[e];
  const int32_t sp = sh == kNoParam ? kNoEdge : sh * 65536 + ti.step_s[e];
  const int32_t tp = th == kNoParam ? kNoEdge : th * 65536 + ti.term_s[e];
  T.step[(c * 4 + d) * 16 + a * 4 + b] = sp;
  T.term_r[(c * 4 + d) * 16 + a * 4 + b] = tp;
  // read from the other strand: 5'-ab-3' = 5'-c1 c0-3' over 3'-y x-5' with row (c1, c0) = (a, b)
  T.term_l[(a * 4 + b) * 16 + c * 4 + d] = tp;
}

// TmTabs from the parameter tables (row_ds is not filled: only the generated chains read it)
__device__ __forceinline__ void fill_tabs(TmTabs& T, int slot) {
  for (int e = threadIdx.x; e < 256; e += blockDim.x) put_tab_entry(T, c_nni[slot], e);
}

__device__ __forceinline__ int32_t end_packed(const TmRun& R, int j, int L, int v) {
  return j == 0 ? R.end_l[v] : R.end_r[v];
}

__device__ __forceinline__ int rank_of(uint32_t ch, int a) { return __popc(ch & ((1u << a) - 1u)); }

// One pass over the compressed chain in score arithmetic S: the best A * dS10 - B * dH10 and that
// variant's exact packed sums.  W: this thread's weights (stride `ws` words); dmask: branch
// positions (never empty).
// A step between adjacent branch positions lo, lo + 1 that are not the duplex's end edges is one
// parameter lookup per pair of bases: its weights are the step table's row for the site's two
// opposite-strand codes there, read in place rather than copied per site.
__device__ __forceinline__ bool direct_step(int lo, int hi, int L) { return hi == lo + 1 && lo != 0 && lo != L - 2; }

template <typename S>
__device__ __forceinline__ bool thread_pass(const TmTabs& T, const int32_t* __restrict__ W, int ws, const PrimerMasks P,
                                            uint32_t dmask, uint64_t cc, int L, S A, S B, S* best, int32_t* bsum) {
  const S none = no_score<S>();
  S cur[4];
  int32_t cs[4];
  int lo = __ffs(dmask) - 1;
  uint32_t rest = dmask & (dmask - 1);
  uint32_t cha = P.ch(lo);
  int off = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    cur[a] = none;
    cs[a] = 0;
    if ((cha >> a) & 1u) {
      const int32_t p = W[(off + rank_of(cha, a)) * ws];
      if (p != kNoEdge) cur[a] = A * (S)unpack_ds(p) - B * (S)unpack_dh(p), cs[a] = p;
    }
  }
  off += __popc(cha);
  while (rest) {
    const int hi = __ffs(rest) - 1;
    rest &= rest - 1;
    const uint32_t chb = P.ch(hi);
    const int nb = __popc(chb);
    const bool direct = direct_step(lo, hi, L);
    const int32_t* trow = T.step + row_of(cc, lo);
    S nx[4];
    int32_t ns[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) nx[b] = none, ns[b] = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (!((cha >> a) & 1u) || cur[a] == none) continue;
      const int row = off + rank_of(cha, a) * nb;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (!((chb >> b) & 1u)) continue;
        const int32_t p = direct ? trow[a * 4 + b] : W[(row + rank_of(chb, b)) * ws];
        if (p == kNoEdge) continue;
        const S sc = cur[a] + (A * (S)unpack_ds(p) - B * (S)unpack_dh(p));
        if (sc > nx[b]) nx[b] = sc, ns[b] = cs[a] + p;
      }
    }
    if (!direct) off += __popc(cha) * nb;
#pragma unroll
    for (int b = 0; b < 4; ++b) cur[b] = nx[b], cs[b] = ns[b];
    cha = chb;
    lo = hi;
  }
  S bs = none;
  int32_t bp = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (!((cha >> a) & 1u) || cur[a] == none) continue;
    const int32_t p = W[(off + rank_of(cha, a)) * ws];
    if (p == kNoEdge) continue;
    const S sc = cur[a] + (A * (S)unpack_ds(p) - B * (S)unpack_dh(p));
    if (sc > bs) bs = sc, bp = cs[a] + p;
  }
  if (bs == none) return false;
  *best = bs;
  *bsum = bp;
  return true;
}

// The weights of one site's compressed chain into W (stride ws): one per choice at the first branch
// position (with everything before it), one per pair of choices at consecutive ones (with the fixed
// steps between them), one per choice at the last (with everything after it).  Returns a bound on
// every variant's dS (tenths): the sum of each block's largest.
__device__ __forceinline__ int thread_weights(const TmRun& R, const TmTabs& T, int32_t* __restrict__ W, int ws,
                                              const PrimerMasks P,
                                              uint32_t dmask, uint64_t cc, int L) {
  int bound = 0, off = 0;
  {
    const int d0 = __ffs(dmask) - 1;
    const uint32_t ch0 = P.ch(d0);
    int mx = INT_MIN;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (!((ch0 >> a) & 1u)) continue;
      int32_t p = end_packed(R, 0, L, d0 == 0 ? a : P.fixed(0));
      for (int i = 0; i < d0; ++i)
        p = add_packed(p, edge_tab(T, i, L, P.fixed(i), i + 1 == d0 ? a : P.fixed(i + 1), cc));
      W[(off + rank_of(ch0, a)) * ws] = p;
      if (p != kNoEdge) mx = max(mx, unpack_ds(p));
    }
    off += __popc(ch0);
    bound += mx == INT_MIN ? 0 : mx;
  }
  int lo = __ffs(dmask) - 1;
  for (uint32_t rest = dmask & (dmask - 1); rest; rest &= rest - 1) {
    const int hi = __ffs(rest) - 1;
    const uint32_t cha = P.ch(lo), chb = P.ch(hi);
    const int nb = __popc(chb);
    if (direct_step(lo, hi, L)) {  // read in place by the passes: only its part of the bound
      const int32_t* trow = T.step + row_of(cc, lo);
      int mx = INT_MIN;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int32_t p = trow[a * 4 + b];
          if (((cha >> a) & 1u) && ((chb >> b) & 1u) && p != kNoEdge) mx = max(mx, unpack_ds(p));
        }
      bound += mx == INT_MIN ? 0 : mx;
      lo = hi;
      continue;
    }
    int32_t mid = 0, left[4], right[4];
    const bool adjacent = hi == lo + 1;
    if (!adjacent) {
      for (int i = lo + 1; i + 1 < hi; ++i) mid += edge_tab(T, i, L, P.fixed(i), P.fixed(i + 1), cc);
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        left[x] = (cha >> x) & 1u ? edge_tab(T, lo, L, x, P.fixed(lo + 1), cc) : kNoEdge;
        right[x] = (chb >> x) & 1u ? edge_tab(T, hi - 1, L, P.fixed(hi - 1), x, cc) : kNoEdge;
      }
    }
    int mx = INT_MIN;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (!((cha >> a) & 1u)) continue;
      const int row = off + rank_of(cha, a) * nb;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (!((chb >> b) & 1u)) continue;
        const int32_t p = adjacent ? edge_tab(T, lo, L, a, b, cc) : add_packed(add_packed(left[a], mid), right[b]);
        W[(row + rank_of(chb, b)) * ws] = p;
        if (p != kNoEdge) mx = max(mx, unpack_ds(p));
      }
    }
    off += __popc(cha) * nb;
    bound += mx == INT_MIN ? 0 : mx;
    lo = hi;
  }
  {
    const uint32_t chl = P.ch(lo);
    int mx = INT_MIN;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (!((chl >> b) & 1u)) continue;
      int32_t p = end_packed(R, L - 1, L, lo == L - 1 ? b : P.fixed(L - 1));
      for (int i = lo; i + 1 < L; ++i)
        p = add_packed(p, edge_tab(T, i, L, i == lo ? b : P.fixed(i), P.fixed(i + 1), cc));
      W[(off + rank_of(chl, b)) * ws] = p;
      if (p != kNoEdge) mx = max(mx, unpack_ds(p));
    }
    bound += mx == INT_MIN ? 0 : mx;
  }
  return bound;
}

// the branch positions of a primer of length L (a concrete primer: its first position)
__device__ __forceinline__ uint32_t chain_nodes(const PrimerMasks P, int L) {
  const uint32_t d = P.branching(L);
  return d ? d : 1u;
}

// Any primer's compressed chain, walked from its position masks (the chain type of chain_site_tm).
struct GenericChain {
  PrimerMasks P;
  uint32_t dmask;  // branch positions
  uint64_t cc;     // the site's opposite-strand codes
  int L;
  const TmRun* R;  // the run constants (shared memory)
  __device__ __forceinline__ int weights(const TmTabs& T, int32_t* __restrict__ W, int ws) const {
    return thread_weights(*R, T, W, ws, P, dmask, cc, L);
  }
  template <typename S>
  __device__ __forceinline__ bool pass(const TmTabs& T, const int32_t* __restrict__ W, int ws, S A, S B, S* best,
                                       int32_t* bsum) const {
    return thread_pass<S>(T, W, ws, P, dmask, cc, L, A, B, best, bsum);
  }
};

// the built-in kernel's sites: tables from the parameter arrays, every primer by GenericChain
struct GenericSites {
  static __device__ __forceinline__ void fill(TmTabs& T, const int32_t*, int slot) { fill_tabs(T, slot); }
  static __device__ __forceinline__ bool site(uint32_t, const TmTabs& T, int32_t* __restrict__ W, int ws,
                                              const PrimerMasks P, uint64_t code, int L, const TmRun& R, double* tm) {
    const GenericChain c{P, chain_nodes(P, L), code ^ 0xAAAAAAAAAAAAAAAAull, L, &R};
    return chain_site_tm(T, W, ws, c, L, R, P.some_gc(L), tm);
  }
};

// the d-th allowed code of a choice set
__device__ __forceinline__ int nth_code(uint32_t ch, uint32_t d) {
  for (uint32_t k = 0; k < d; ++k) ch &= ch - 1;
  return __ffs(ch) - 1;
}

// Every variant of a site's primer (every concrete variant counting), enumerated by the 32 lanes of
// a warp from the compressed chain's weights in each lane's W: the maximum Tm, each variant's as
// enum_max computes it (exact integer sums, one FP64 evaluation).  A first sweep evaluates every
// variant in single precision; the second evaluates in FP64 those within a margin of the largest
// single-precision value (the margin covers its rounding: 1 K plus 2e-4 of the absolute
// temperature) and those whose entropy sum is within 2 cal/(K mol) of zero, where single precision
// says little.  More than 2^20 variants: NaN and ST_TM_LIMIT.
//
// A variant is a number in mixed radix, digit q the choice at the q-th branch position counted from
// the 3' end.  Its sums are suffix(d_0) + sum over q of step_q(d_(q+1), d_q) + prefix(d_(m-1)).  Each
// lane walks a contiguous block of variants like an odometer and keeps U[q], the sum of the terms
// of digits q and above: a variant then costs the terms of digit 0, and a carry recomputes U only
// up to the highest digit that changed.
constexpr int kEnumMaxBranch = 32;
__device__ __noinline__ double warp_enumerate(const TmTabs& T, const int32_t* __restrict__ W, int ws, const PrimerMasks P,
                                              uint64_t cc, int L, const TmRun& R, uint32_t* status, int lane) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const uint32_t dmask = chain_nodes(P, L);
  const uint32_t lmask = L >= 32 ? 0xFFFFFFFFu : ((1u << L) - 1u);
  const int gc_fixed = __popc((P.m[1] | P.m[3]) & ~dmask & lmask);  // C and G at single-choice positions
  // branch positions from the 3' end: position, choices, and where the weights of the step to the
  // next one (toward 5') start in W (-1: read in place from the table)
  uint8_t pos[kEnumMaxBranch], ch[kEnumMaxBranch], rad[kEnumMaxBranch];
  int16_t offq[kEnumMaxBranch];
  int m = 0;
  int off_suf = 0;
  uint64_t count = 1;
  {
    int prev_n = 0, prev_pos = -1;
    for (uint32_t x = dmask; x; x &= x - 1) {  // 5' to 3': the offsets of the blocks
      const int p = __ffs(x) - 1;
      const int n = __popc(P.ch(p));
      if (prev_pos < 0) off_suf += n;
      else if (!direct_step(prev_pos, p, L)) off_suf += prev_n * n;
      prev_n = n, prev_pos = p;
      count = min(count * (uint64_t)n, kEnumLimit + 1);
    }
    if (count > kEnumLimit) {
      if (lane == 0) atomicOr(status, (uint32_t)ST_TM_LIMIT);
      return nan;
    }
    int off = off_suf;
    for (uint32_t x = dmask; x; ++m) {  // 3' to 5'
      const int p = 31 - __clz(x);
      x &= ~(1u << p);
      pos[m] = (uint8_t)p;
      ch[m] = (uint8_t)P.ch(p);
      rad[m] = (uint8_t)__popc(ch[m]);
      offq[m] = -1;
      if (m > 0) {
        if (!direct_step(p, pos[m - 1], L)) {
          off -= rad[m] * rad[m - 1];
          offq[m - 1] = (int16_t)off;
        }
      }
    }
  }
  // the step between digit q + 1 (toward 5') and digit q, for digits dq1, dq
  auto step_w = [&](int q, uint32_t dq1, uint32_t dq) -> int32_t {
    if (offq[q] < 0) return T.step[row_of(cc, pos[q + 1]) + nth_code(ch[q + 1], dq1) * 4 + nth_code(ch[q], dq)];
    return W[(offq[q] + dq1 * rad[q] + dq) * ws];
  };
  // constant parts of dH and dS (a variant with and without G or C), and the Tm from the sums, in
  // single precision
  const double S1 = (R.saltcorr == 5 ? 0.368 * (double)(L - 1) * R.ln_mon : 0.0) + R.rlnk;
  const float Hg = (float)R.h0, Sg = (float)(R.s0 + S1);
  const float Ha = (float)(R.init_h + R.allat_h + R.sym_h), Sa = (float)(R.init_s + R.allat_s + R.sym_s + S1);
  const float shiftf = R.saltcorr >= 1 && R.saltcorr <= 4 ? (float)R.corr_const : 0.f;
  auto tm_float = [&](int32_t p, int gc, bool* near_zero) {
    const float dh = 0.1f * (float)unpack_dh(p) + (gc ? Hg : Ha), ds = 0.1f * (float)unpack_ds(p) + (gc ? Sg : Sa);
    *near_zero = fabsf(ds) < 2.f;
    float t = 1000.f * dh / ds - 273.15f + shiftf;
    if (R.saltcorr >= 6) {
      const float corr = (float)(R.rc0 + R.rc1 * ((double)gc / (double)L) + R.rc2 / (2.0 * (double)(L - 1)));
      t = 1.f / (1.f / (t + 273.15f) + corr) - 273.15f;
    }
    return t;
  };
  // this lane's block of variants
  const uint64_t per = (count + 31) / 32;
  const uint64_t v_begin = min(count, (uint64_t)lane * per), v_end = min(count, v_begin + per);
  // one sweep over the block: fn(packed sums, G/C count) for every defined variant
  auto sweep = [&](auto&& fn) {
    if (v_begin >= v_end) return;
    uint8_t d[kEnumMaxBranch];
    int32_t U[kEnumMaxBranch];
    int G[kEnumMaxBranch];
    {
      uint64_t v = v_begin;
      for (int q = 0; q < m; ++q) d[q] = (uint8_t)(v % rad[q]), v /= rad[q];
    }
    int top = m - 1;  // U[q] and G[q] are stale for q <= top
    for (uint64_t v = v_begin; v < v_end;) {
      for (int q = top; q >= 1; --q) {
        if (q == m - 1) {
          U[q] = W[d[q] * ws];
          G[q] = gc_fixed + (nth_code(ch[q], d[q]) & 1);
        } else {
          U[q] = add_packed(U[q + 1], step_w(q, d[q + 1], d[q]));
          G[q] = G[q + 1] + (nth_code(ch[q], d[q]) & 1);
        }
      }
      // digit 0 runs through its choices with the rest fixed
      for (uint32_t d0 = d[0]; d0 < rad[0] && v < v_end; ++d0, ++v) {
        int32_t p;
        int gc;
        const int c0 = nth_code(ch[0], d0);
        if (m == 1) {
          p = add_packed(W[d0 * ws], W[(off_suf + d0) * ws]);
          gc = gc_fixed + (c0 & 1);
        } else {
          p = add_packed(add_packed(U[1], step_w(0, d[1], d0)), W[(off_suf + d0) * ws]);
          gc = G[1] + (c0 & 1);
        }
        if (p != kNoEdge) fn(p, gc);
      }
      // carry
      d[0] = 0;
      top = 0;
      for (int q = 1; q < m; ++q) {
        top = q;
        if (++d[q] < rad[q]) break;
        d[q] = 0;
      }
    }
  };
  float best_f = -INFINITY;
  double best = -INFINITY;
  sweep([&](int32_t p, int gc) {
    bool nz;
    const float t = tm_float(p, gc, &nz);
    if (nz) best = fmax(best, tm_of_tenths(unpack_dh(p), unpack_ds(p), gc, L, R));
    else if (t > best_f) best_f = t;
  });
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best_f = fmaxf(best_f, __shfl_xor_sync(0xffffffffu, best_f, o));
  if (best_f > -INFINITY) {
    const float floor_f = best_f - (1.f + 2e-4f * fabsf(best_f + 273.15f));
    sweep([&](int32_t p, int gc) {
      bool nz;
      const float t = tm_float(p, gc, &nz);
      if (!nz && t >= floor_f) best = fmax(best, tm_of_tenths(unpack_dh(p), unpack_ds(p), gc, L, R));
    });
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  return best > -INFINITY ? best : nan;
}

// The site Tm of every marked site, every concrete variant counting (params variants = 0): the
// shared kernel body (tm_hits_body) over GenericChain.  Weights: thread_weight_words per thread.
__global__ void __launch_bounds__(kTmThreads, 4) k_tm_hits_t(const ah_hit* __restrict__ hits, uint64_t n,
                                                             const uint2* __restrict__ planes,
                                                             const uint64_t* __restrict__ rec_group,
                                                             const uint8_t* __restrict__ plen,
                                                             const uint4* __restrict__ pmask, const TmRun Rp,
                                                             double* __restrict__ out, uint32_t* __restrict__ defer,
                                                             const uint64_t* __restrict__ d_n) {
  tm_hits_body<GenericSites>(hits, n, planes, rec_group, plen, pmask, Rp, out, defer, d_n, nullptr, 0u, ~0u);
}

// The sites k_tm_hits_t listed (defer[0] of them at defer[1..]): one warp per site, every lane
// computing the site's weights in its own area and enumerating a share of its variants.  A grid of
// a few blocks per SM strides over the list, so sites that cluster (repeats) spread over the GPU.
__global__ void __launch_bounds__(kTmThreads) k_tm_deferred(const ah_hit* __restrict__ hits,
                                                           const uint2* __restrict__ planes,
                                                           const uint64_t* __restrict__ rec_group,
                                                           const uint8_t* __restrict__ plen,
                                                           const uint4* __restrict__ pmask, const TmRun Rp,
                                                           double* __restrict__ out, uint32_t* status,
                                                           const uint32_t* __restrict__ defer) {
  __shared__ TmRun R_sh;
  if (threadIdx.x == 0) R_sh = Rp;
  const TmRun& R = R_sh;
  extern __shared__ __align__(16) uint32_t tm_smem[];
  TmTabs& T = *reinterpret_cast<TmTabs*>(tm_smem);
  int32_t* W = reinterpret_cast<int32_t*>(tm_smem + kTmTabWords) + threadIdx.x;
  const uint32_t n_def = defer[0];
  if (blockIdx.x * (kTmThreads / 32) >= n_def) return;  // the whole block has nothing to do
  fill_tabs(T, Rp.nn);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (kTmThreads / 32);
  for (uint32_t q = blockIdx.x * (kTmThreads / 32) + (threadIdx.x >> 5); q < n_def; q += warps) {
    const uint64_t i = defer[1 + q];
    const ah_hit h = hits[i];
    const int L = plen[h.pattern];
    const uint32_t pr = (h.pattern >> 2) * 2 + (h.pattern & 1u);
    const uint4 mk = pmask[pr];
    const PrimerMasks P{{mk.x, mk.y, mk.z, mk.w}};
    const uint64_t code = site_code(planes, rec_group, h, L);
    thread_weights(R, T, W, kTmThreads, P, chain_nodes(P, L), code ^ 0xAAAAAAAAAAAAAAAAull, L);
    const double tm = warp_enumerate(T, W, kTmThreads, P, code ^ 0xAAAAAAAAAAAAAAAAull, L, R, status, lane);
    if (lane == 0) out[i] = tm;
  }
}

// ah_tm_sites in the group form: sites given as IUPAC sets and base codes, n_groups per block of
// kTmWindow threads
template <int G>
__global__ void __launch_bounds__(kTmWindow) k_tm_sites_g(const uint8_t* __restrict__ sets,
                                                          const uint8_t* __restrict__ site,
                                                          const uint32_t* __restrict__ len,
                                                          const uint8_t* __restrict__ kc, uint32_t n, const TmRun Rp,
                                                          double* __restrict__ out, uint32_t* status, int dmax,
                                                          int n_groups) {
  // the run constants in shared memory: device functions take them by reference, and a reference
  // to a kernel parameter would make the compiler copy it to local memory for every thread
  __shared__ TmRun R_sh;
  if (threadIdx.x == 0) R_sh = Rp;
  __syncthreads();
  const TmRun& R = R_sh;

  extern __shared__ __align__(16) uint32_t tm_smem[];
  const int g = threadIdx.x / G, r = threadIdx.x % G;
  if (g >= n_groups) return;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const uint64_t i = (uint64_t)blockIdx.x * n_groups + g;
  if (i >= n) return;
  TmGroupSh& sh = *reinterpret_cast<TmGroupSh*>(tm_smem + 3 * kTmWindow + g * tm_group_words(dmax));
  int32_t* w = reinterpret_cast<int32_t*>(&sh + 1);
  const int L = (int)len[i];
  for (int j = r; j < L; j += G) {
    const uint8_t sj = site[32 * i + j];
    sh.s[j] = sj;
    sh.c[j] = sj ^ 2u;
    sh.set[j] = sets[32 * i + j];
  }
  __syncwarp(gmask);
  const double t = group_site_tm<G>(sh, w, L, kc[2 * i], kc[2 * i + 1], R, status, r, gmask);
  if (r == 0) out[i] = t;
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
                              const uint32_t* __restrict__ len, uint32_t n, const TmRun Rp, double* __restrict__ out) {
  // the run constants in shared memory: device functions take them by reference, and a reference
  // to a kernel parameter would make the compiler copy it to local memory for every thread
  __shared__ TmRun R_sh;
  if (threadIdx.x == 0) R_sh = Rp;
  __syncthreads();
  const TmRun& R = R_sh;

  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t;
  out[i] = duplex_tm(v + 32 * (uint64_t)i, c + 32 * (uint64_t)i, (int)len[i], R, &t)
               ? t
               : __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void k_tm_sites(const uint8_t* __restrict__ sets, const uint8_t* __restrict__ site,
                           const uint32_t* __restrict__ len, const uint8_t* __restrict__ kc, uint32_t n,
                           const TmRun Rp, double* __restrict__ out, uint32_t* status) {
  // the run constants in shared memory: device functions take them by reference, and a reference
  // to a kernel parameter would make the compiler copy it to local memory for every thread
  __shared__ TmRun R_sh;
  if (threadIdx.x == 0) R_sh = Rp;
  __syncthreads();
  const TmRun& R = R_sh;

  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = site_tm(sets + 32 * (uint64_t)i, site + 32 * (uint64_t)i, (int)len[i], kc[2 * i], kc[2 * i + 1], R,
                   status);
}

// Launch shape of the group kernels: G lanes per site from the largest state width W (= k + 1 with a
// mismatch budget, else 1) the launch can meet, and S sites per block within 48 KB of shared memory
// for chains of at most dmax branch positions.  G = 0: widths above 8, left to the per-thread kernels.
struct TmShape {
  int G = 0, S = 0, dmax = 1;
  size_t smem = 0;
};

TmShape tm_shape(int wmax, int dmax) {
  TmShape t;
  t.dmax = std::max(1, dmax);
  t.G = wmax <= 1 ? 4 : wmax <= 2 ? 8 : wmax <= 4 ? 16 : wmax <= 8 ? 32 : 0;
  if (!t.G) return t;
  const size_t words = (size_t)tm_group_words(t.dmax);
  t.S = kTmWindow / t.G;
  while (t.S > 1 && 4 * (3 * kTmWindow + t.S * words) > 48 * 1024) --t.S;
  t.smem = 4 * (3 * kTmWindow + t.S * words);
  return t;
}

// positions of a primer with more than one IUPAC choice
int degenerate_positions(const std::string& primer) {
  int d = 0;
  for (char ch : primer) d += __builtin_popcount(iupac_set(ch)) >= 2;
  return d;
}

TmShape hits_shape(const ah_primers* p, int variants) {
  int wmax = 1, dmax = 1;
  for (uint32_t q = 0; q < p->n_pairs; ++q) {
    const size_t lmin = std::min(p->fwd[q].size(), p->rev[q].size());
    if (variants && p->k[q] < lmin) wmax = std::max(wmax, (int)p->k[q] + 1);
    dmax = std::max({dmax, degenerate_positions(p->fwd[q]), degenerate_positions(p->rev[q])});
  }
  return tm_shape(wmax, dmax);
}

// weights one thread of k_tm_hits_t stores for a primer: one per choice at the first and last branch
// positions, one per pair of choices at consecutive ones (a primer without a branch position: its
// first position, one choice)
int thread_weight_words(const std::string& primer) {
  const int L = (int)primer.size();
  std::vector<int> n, pos;
  for (int j = 0; j < L; ++j)
    if (__builtin_popcount(iupac_set(primer[j])) >= 2) n.push_back(__builtin_popcount(iupac_set(primer[j]))), pos.push_back(j);
  if (n.empty()) n.push_back(1), pos.push_back(0);
  int w = n.front() + n.back();
  for (size_t t = 0; t + 1 < n.size(); ++t) {
    const bool direct = pos[t + 1] == pos[t] + 1 && pos[t] != 0 && pos[t] != L - 2;  // see direct_step
    if (!direct) w += n[t] * n[t + 1];
  }
  return w;
}

constexpr int kTmThreadFixedWords = kTmTabWords + 2 * kTmSlots;  // tables, keys and their order
constexpr size_t kTmSmemCap = 46 * 1024;  // dynamic shared memory, beside the kernels' static arrays
// the most launches of the generated Tm kernel, each for a group of primers (TmKernel::split_sites)
constexpr uint32_t kTmPrimerLaunches = 4;

// the Tm of every marked site (hit_tm holds kSiteWanted there): one thread per site for the default
// reading when its weights fit, else the group kernel where the state width allows, else k_tm_hits
// one-thread-per-site kernel's shared memory for this primer set (0: the weights do not fit)
size_t thread_kernel_smem(const ah_primers* p, int variants) {
  if (variants) return 0;
  int ww = 1;
  for (uint32_t q = 0; q < p->n_pairs; ++q)
    ww = std::max({ww, thread_weight_words(p->fwd[q]), thread_weight_words(p->rev[q])});
  const size_t smem = 4 * ((size_t)kTmThreadFixedWords + (size_t)ww * kTmThreads);
  return smem <= kTmSmemCap ? smem : 0;
}

// defer: cap + 1 words of device scratch for the sites the chain does not cover (the thread kernel
// lists them there for k_tm_deferred).  Returns the kernels launched.
int launch_tm_hits(cudaStream_t s, const TmRun& R, const ah_primers* p, const ah_hit* hits, uint64_t cap,
                    const uint64_t* d_n, const uint2* planes, const uint64_t* rec_group, double* hit_tm,
                    uint32_t* status, uint32_t* defer, int sm_count, const TmKernel& tk, bool* generated) {
  if (generated) *generated = false;
  int n_launched = 0;
  if (const size_t smem = thread_kernel_smem(p, R.variants)) {
    cudaMemsetAsync(defer, 0, sizeof(uint32_t), s);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, (cap + kTmSlots - 1) / kTmSlots);
    const size_t smem_j = 4 * ((size_t)kTmThreadFixedWords + (size_t)tk.weight_words * kTmThreads);
    if (tk.fn && tk.image && smem_j <= kTmSmemCap) {  // the kernel generated for this primer set
      const uint8_t* plen = p->d_plen;
      const uint4* pmask = p->d_pmask;
      // many sites: one launch per group of primers (at most kTmPrimerLaunches), so that each
      // launch runs fewer primers' straight-line chains and they stay in the instruction cache
      const uint32_t n_pr = 2 * p->n_pairs;
      const uint32_t parts = cap >= tk.split_sites ? std::min<uint32_t>(n_pr, kTmPrimerLaunches) : 1;
      for (uint32_t k = 0; k < parts; ++k) {
        uint32_t pr_lo = parts > 1 ? n_pr * k / parts : 0u, pr_hi = parts > 1 ? n_pr * (k + 1) / parts : ~0u;
        void* args[] = {(void*)&hits, (void*)&cap,    (void*)&planes, (void*)&rec_group, (void*)&plen, (void*)&pmask,
                        (void*)&R,    (void*)&hit_tm, (void*)&defer,  (void*)&d_n,       (void*)&tk.image,
                        (void*)&pr_lo, (void*)&pr_hi};
        cudaLaunchKernel((const void*)tk.fn, dim3(grid), dim3(kTmThreads), args, smem_j, s);
      }
      if (generated) *generated = true;
      n_launched += parts;
    } else {
      k_tm_hits_t<<<grid, kTmThreads, smem, s>>>(hits, cap, planes, rec_group, p->d_plen, p->d_pmask, R, hit_tm, defer,
                                                 d_n);
      ++n_launched;
    }
    const size_t smem_d = smem - 4 * (size_t)(2 * kTmSlots);  // tables and weights only
    // the list's length is known on the device only: a grid of 4 to 64 blocks per SM by the site
    // capacity (the dense workload's 28 M sites: 13.07 -> 12.85 ms per step from 4 to 64 per SM;
    // warps finish their strides at different times, and more of them even that out)
    const uint64_t sms = (uint64_t)std::max(1, sm_count);
    const unsigned grid_d = (unsigned)std::min(64 * sms, std::max(4 * sms, cap >> 12));
    k_tm_deferred<<<grid_d, kTmThreads, smem_d, s>>>(hits, planes, rec_group, p->d_plen, p->d_pmask, R, hit_tm, status,
                                                     defer);
    return n_launched + 1;
  }
  const TmShape t = hits_shape(p, R.variants);
  if (!t.G) {
    k_tm_hits<<<(unsigned)std::max<uint64_t>(1, (cap + kTmBlock - 1) / kTmBlock), kTmBlock, 0, s>>>(
        hits, cap, planes, rec_group, p->d_plen, p->d_psets, p->d_pk, p->clamp, R, hit_tm, status, d_n);
    return 1;
  }
  const unsigned grid = (unsigned)std::max<uint64_t>(1, (cap + kTmWindow - 1) / kTmWindow);
#define AH_TM_HITS_G(GG)                                                                                        \
  k_tm_hits_g<GG><<<grid, kTmWindow, t.smem, s>>>(hits, cap, planes, rec_group, p->d_plen, p->d_psets, p->d_pk, \
                                                  p->clamp, R, hit_tm, status, t.dmax, t.S, d_n)
  switch (t.G) {
    case 4: AH_TM_HITS_G(4); break;
    case 8: AH_TM_HITS_G(8); break;
    case 16: AH_TM_HITS_G(16); break;
    default: AH_TM_HITS_G(32); break;
  }
#undef AH_TM_HITS_G
  return 1;
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
  int wmax = 1, dmax = 1;
  for (uint32_t i = 0; i < n; ++i) {
    if (kc[2 * (size_t)i] < len[i]) wmax = std::max(wmax, kc[2 * (size_t)i] + 1);
    dmax = std::max(dmax, degenerate_positions(primers[i]));
  }
  const TmShape t = tm_shape(wmax, dmax);
  if (!t.G) {
    k_tm_sites<<<(n + 63) / 64, 64, 0, ctx->stream>>>(ds, dv, dl, dk, n, R, dout, ctx->d_status);
  } else {
    const unsigned grid = (unsigned)((n + t.S - 1) / t.S);
#define AH_TM_SITES_G(GG)                                                                       \
  k_tm_sites_g<GG><<<grid, kTmWindow, t.smem, ctx->stream>>>(ds, dv, dl, dk, n, R, dout, ctx->d_status, \
                                                             t.dmax, t.S)
    switch (t.G) {
      case 4: AH_TM_SITES_G(4); break;
      case 8: AH_TM_SITES_G(8); break;
      case 16: AH_TM_SITES_G(16); break;
      default: AH_TM_SITES_G(32); break;
    }
#undef AH_TM_SITES_G
  }
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

size_t tm_run_bytes() { return sizeof(TmRun); }

int tm_run_slot(const void* run) { return ((const TmRun*)run)->nn; }

ah_status tm_tab_image(ah_ctx* ctx, int slot, const int32_t** out) {
  *out = nullptr;
  ah_status st;
  if ((st = load_tables(ctx))) return st;
  std::lock_guard<std::mutex> lock(g_tables_mu);
  if (ctx->device >= 64 || slot < 0 || slot >= kNNSlots) return fail(ctx, AH_EINTERNAL, "tm_tab_image: bad device or set");
  if (!g_tab_image[ctx->device][slot]) {
    TmTabs T;
    for (int e = 0; e < 256; ++e) put_tab_entry(T, g_host_i[slot], e);
    for (int r = 0; r < 16; ++r) {  // the largest dS of each step row over its defined entries
      int mx = 0;
      bool any = false;
      for (int k = 0; k < 16; ++k) {
        const int32_t p = T.step[r * 16 + k];
        if (p == kNoEdge) continue;
        const int ds = (int16_t)(p & 0xffff);
        mx = any ? std::max(mx, ds) : ds;
        any = true;
      }
      T.row_ds[r] = mx;
    }
    int32_t* d = nullptr;
    AH_CUDA(ctx, cudaMalloc(&d, sizeof T));  // kept for the life of the process, like the tables
    AH_CUDA(ctx, cudaMemcpy(d, &T, sizeof T, cudaMemcpyHostToDevice));
    g_tab_image[ctx->device][slot] = d;
  }
  *out = g_tab_image[ctx->device][slot];
  return AH_OK;
}

ah_status tm_prepare(ah_ctx* ctx, const ah_tm_params* params, void* run_out, size_t run_size) {
  ah_status st;
  if ((st = load_tables(ctx))) return st;
  if (run_size < sizeof(TmRun)) return fail(ctx, AH_EINTERNAL, "tm_prepare: buffer too small");
  return make_run(ctx, params, (TmRun*)run_out);
}

void launch_tm(cudaStream_t s, const void* run, const ah_hit* hits, uint64_t hit_cap, const uint64_t* d_nhits,
               const ah_primers* p, uint32_t* status, const uint2* planes, const uint64_t* rec_group, double* hit_tm,
               ah_amplicon* amps, uint64_t amp_cap, const uint64_t* d_namps, int filter, double min_tm, uint32_t* keep,
               uint32_t* defer, int sm_count, const TmKernel& tk) {
  const TmRun R = *(const TmRun*)run;
  cudaMemsetAsync(hit_tm, 0, std::max<uint64_t>(1, hit_cap) * sizeof(double), s);
  k_mark_sites<<<(unsigned)std::max<uint64_t>(1, (amp_cap + 255) / 256), 256, 0, s>>>(amps, amp_cap, hit_tm, d_namps);
  launch_tm_hits(s, R, p, hits, hit_cap, d_nhits, planes, rec_group, hit_tm, status, defer, sm_count, tk, nullptr);
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
  uint32_t* defer = nullptr;
  if (h->n && a->n) {
    if ((st = dalloc(ctx, &defer, h->n + 1))) return st;
    TmKernel tk;
    if (!R.variants && (st = tm_kernel_for(ctx, p, false, R.nn, &tk))) return st;
    bool generated = false;
    launched(ctx, launch_tm_hits(ctx->stream, R, p, h->d, h->n, nullptr, b->planes, b->rec_group, hit_tm,
                                 ctx->d_status, defer, ctx->sm_count, tk, &generated));
    (generated ? ctx->n_tm_generated : ctx->n_tm_builtin)++;
  }
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
  dfree(ctx, defer);
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
