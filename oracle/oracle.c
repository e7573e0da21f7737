/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of the in-silico PCR path of AmpliconHunter2
 * (Howard-Stone & Mandoiu, arXiv 2511.00170).  Only the tests, the smoke check and the bench's CPU
 * baseline may load it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes, step by step, with the passage each step follows:
 *   scan    -- Supplementary "Primer matching and clamp logic": every primer and its reverse
 *              complement is matched per base against IUPAC sets, mismatches are counted, and the
 *              3' clamp must match exactly (also Abstract: "user-specified mismatches and 3' clamp").
 *   sort    -- Supplementary "Amplicon calling and orientation": candidate sites are sorted.
 *   pair    -- same passage: opposite-sense sites are paired inside [min,max]; a same-sense site
 *              stops the walk; orientation FR/RF/FF/RR; RF is reverse-complemented.
 *   extract -- Supplementary "Primer trimming and barcode extraction" and "Headers and outputs".
 *   Tm      -- Section "Implementations" (AHv2): the nearest-neighbour Tm of Biopython's Tm_NN,
 *              in double precision; Section "Primer degeneracy": Tm is evaluated over the
 *              concrete variants of a degenerate primer.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1 a window holding any non-ACGT genome base is not a hit; lower-case acgt are bases.
 *   R2 primer code N matches any base; a code matches a base iff the base is in its IUPAC set.
 *   R3 the clamp is the last c primer positions (3' end) and must match set-wise.
 *   R4 on the reverse strand the primer's 3' end is the left end of rc(primer) on the top strand.
 *   R5 "same sense" = any + strand site of the same primer pair.
 *   R6 an anchor pairs with every antisense site before the first same-sense site or the first
 *      site whose amplicon would exceed max_len.
 *   R7 ties at one position: + before -, F before R.
 *   R8 amplicon length = end of the antisense site - start of the anchor, inclusive window.
 *   R9 orientations are filtered after pairing.
 *   R10 FF and RR amplicons are written on the top strand, barcodes as for FR.
 *   R11 a trimmed amplicon whose sites overlap is empty (the amplicon is still reported).
 *   R12 barcodes are clipped at record ends; non-ACGT bases are written as N.
 *   R13 the amplicon Tm is the lower of its two site Tms.
 *   R14 the Tm of a degenerate primer at a site is the maximum over every concrete variant of
 *       the primer, variants that mismatch the site included.  Option (variants = 1): only the
 *       variants that themselves match the site under the scan's rule count (at most k
 *       mismatching positions, an exact 3' clamp); the variant that agrees with the site wherever
 *       the primer allows it always qualifies.
 *   R15 a variant whose duplex needs a parameter the tables do not have (e.g. two adjacent
 *       mismatches other than the tandem G.T steps) has no Tm; a site with no defined variant
 *       has an undefined Tm, and an amplicon with an undefined Tm is dropped by the filter.
 *   R16 filtering compares unrounded doubles.
 *
 * The thermodynamic values are transcriptions of the published parameter sets named at each
 * table.  They could not be checked here against the publications or against Biopython, so the
 * parity of the tables themselves is unpinned; the arithmetic around them is pinned by tests.
 */
#include <ctype.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* IUPAC nomenclature (Cornish-Bowden 1985, NC-IUB): code -> set of bases, complement of codes   */

static unsigned code_set(char c) {
  switch (toupper((unsigned char)c)) {
    case 'A': return 1;  /* {A} */
    case 'C': return 2;  /* {C} */
    case 'G': return 4;  /* {G} */
    case 'T': return 8;  /* {T} */
    case 'R': return 1 | 4;
    case 'Y': return 2 | 8;
    case 'S': return 2 | 4;
    case 'W': return 1 | 8;
    case 'K': return 4 | 8;
    case 'M': return 1 | 2;
    case 'B': return 2 | 4 | 8;
    case 'D': return 1 | 4 | 8;
    case 'H': return 1 | 2 | 8;
    case 'V': return 1 | 2 | 4;
    case 'N': return 1 | 2 | 4 | 8;
    default: return 0;
  }
}

static char code_complement(char c) {
  switch (toupper((unsigned char)c)) {
    case 'A': return 'T';
    case 'T': return 'A';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'R': return 'Y';
    case 'Y': return 'R';
    case 'K': return 'M';
    case 'M': return 'K';
    case 'B': return 'V';
    case 'V': return 'B';
    case 'D': return 'H';
    case 'H': return 'D';
    case 'S': return 'S';
    case 'W': return 'W';
    case 'N': return 'N';
    default: return '?';
  }
}

/* genome character -> set bit of its base, 0 when it is not one of ACGT (reading R1) */
static unsigned genome_base(uint8_t c) {
  switch (c) {
    case 'A': case 'a': return 1;
    case 'C': case 'c': return 2;
    case 'G': case 'g': return 4;
    case 'T': case 't': return 8;
    default: return 0;
  }
}

static char genome_letter(uint8_t c) {
  switch (genome_base(c)) {
    case 1: return 'A';
    case 2: return 'C';
    case 4: return 'G';
    case 8: return 'T';
    default: return 'N';
  }
}

static char base_complement(char b) {
  switch (b) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'T': return 'A';
    default: return 'N';
  }
}

/* reverse complement of a primer written in IUPAC codes */
static void primer_revcomp(const char* p, int L, char* out) {
  for (int i = 0; i < L; ++i) out[i] = code_complement(p[L - 1 - i]);
  out[L] = 0;
}

/* 0 = ok; 1 = bad code; 2 = length outside [1,32]; 3 = clamp > length; 4 = k > length */
int or_check_primer(const char* p, int clamp, int k) {
  int L = (int)strlen(p);
  if (L < 1 || L > 32) return 2;
  for (int i = 0; i < L; ++i)
    if (code_set(p[i]) == 0) return 1;
  if (clamp < 0 || clamp > L) return 3;
  if (k < 0 || k > L) return 4;
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* scan                                                                                         */

typedef struct {
  uint32_t record;
  uint32_t pos;
  uint16_t pair;
  uint8_t primer; /* 0 = forward primer, 1 = reverse primer */
  uint8_t strand; /* 0 = primer as written binds the top strand (+), 1 = its reverse complement (-) */
  uint8_t mism;
  uint8_t pad[3];
} or_hit;

typedef struct {
  const uint8_t* seq;
  const int64_t* offsets;
  uint32_t n_pairs;
  const char* const* fwd;
  const char* const* rev;
  const uint8_t* k;
  int clamp;
} scan_job;

typedef struct {
  or_hit* v;
  int64_t n, cap;
} hit_vec;

static void push_hit(hit_vec* hv, or_hit h) {
  if (hv->n == hv->cap) {
    hv->cap = hv->cap ? hv->cap * 2 : 1024;
    hv->v = (or_hit*)realloc(hv->v, (size_t)hv->cap * sizeof(or_hit));
  }
  hv->v[hv->n++] = h;
}

/* hits of one record, in (pair, pos, strand, primer) order after the final sort */
static void scan_record(const scan_job* J, uint32_t r, hit_vec* out) {
  const uint8_t* g = J->seq + J->offsets[r];
  int64_t len = J->offsets[r + 1] - J->offsets[r];
  /* invalid[i] = number of non-ACGT bases in g[0, i) */
  uint32_t* invalid = (uint32_t*)malloc((size_t)(len + 1) * sizeof(uint32_t));
  invalid[0] = 0;
  for (int64_t i = 0; i < len; ++i) invalid[i + 1] = invalid[i] + (genome_base(g[i]) == 0);
  for (uint32_t pr = 0; pr < J->n_pairs; ++pr) {
    for (int primer = 0; primer < 2; ++primer) {
      const char* P = primer == 0 ? J->fwd[pr] : J->rev[pr];
      int L = (int)strlen(P);
      char rc[40];
      primer_revcomp(P, L, rc);
      for (int strand = 0; strand < 2; ++strand) {
        const char* pat = strand == 0 ? P : rc;
        unsigned sets[40];
        int is_clamp[40];
        for (int j = 0; j < L; ++j) {
          sets[j] = code_set(pat[j]);
          /* the 3' end of the primer: right end as written, left end of its reverse complement */
          is_clamp[j] = strand == 0 ? (j >= L - J->clamp) : (j < J->clamp);
        }
        for (int64_t p = 0; p + L <= len; ++p) {
          if (invalid[p + L] - invalid[p] != 0) continue;
          int mism = 0, clamp_ok = 1;
          for (int j = 0; j < L; ++j) {
            if ((sets[j] & genome_base(g[p + j])) == 0) {
              ++mism;
              if (is_clamp[j]) clamp_ok = 0;
            }
          }
          if (clamp_ok && mism <= J->k[pr]) {
            or_hit h;
            memset(&h, 0, sizeof h);
            h.record = r;
            h.pos = (uint32_t)p;
            h.pair = (uint16_t)pr;
            h.primer = (uint8_t)primer;
            h.strand = (uint8_t)strand;
            h.mism = (uint8_t)mism;
            push_hit(out, h);
          }
        }
      }
    }
  }
  free(invalid);
}

static int hit_cmp(const void* a, const void* b) {
  const or_hit* x = (const or_hit*)a;
  const or_hit* y = (const or_hit*)b;
  if (x->record != y->record) return x->record < y->record ? -1 : 1;
  if (x->pair != y->pair) return x->pair < y->pair ? -1 : 1;
  if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
  if (x->strand != y->strand) return x->strand < y->strand ? -1 : 1;
  if (x->primer != y->primer) return x->primer < y->primer ? -1 : 1;
  return 0;
}

typedef struct {
  const scan_job* J;
  uint32_t lo, hi;
  hit_vec hv;
} scan_part;

static void* scan_worker(void* arg) {
  scan_part* P = (scan_part*)arg;
  for (uint32_t r = P->lo; r < P->hi; ++r) scan_record(P->J, r, &P->hv);
  return NULL;
}

/* All hits, sorted by (record, pair, pos, strand, primer).  Returns the count; *out is malloc'd. */
int64_t or_scan(const uint8_t* seq, const int64_t* offsets, uint32_t n_rec, uint32_t n_pairs,
                const char* const* fwd, const char* const* rev, const uint8_t* k, int clamp,
                int n_threads, or_hit** out) {
  scan_job J = {seq, offsets, n_pairs, fwd, rev, k, clamp};
  if (n_threads < 1) n_threads = 1;
  if ((uint32_t)n_threads > n_rec) n_threads = n_rec ? (int)n_rec : 1;
  scan_part* parts = (scan_part*)calloc((size_t)n_threads, sizeof(scan_part));
  pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
  /* records are dealt out in contiguous ranges balanced by base count */
  int64_t total = offsets[n_rec] - offsets[0];
  uint32_t r = 0;
  for (int t = 0; t < n_threads; ++t) {
    parts[t].J = &J;
    parts[t].lo = r;
    int64_t target = offsets[0] + (total * (t + 1)) / n_threads;
    while (r < n_rec && (offsets[r + 1] <= target || t == n_threads - 1)) ++r;
    parts[t].hi = r;
  }
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, scan_worker, &parts[t]);
  int64_t n = 0;
  for (int t = 0; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    n += parts[t].hv.n;
  }
  or_hit* all = (or_hit*)malloc((size_t)(n ? n : 1) * sizeof(or_hit));
  int64_t w = 0;
  for (int t = 0; t < n_threads; ++t) {
    if (parts[t].hv.n) memcpy(all + w, parts[t].hv.v, (size_t)parts[t].hv.n * sizeof(or_hit));
    w += parts[t].hv.n;
    free(parts[t].hv.v);
  }
  qsort(all, (size_t)n, sizeof(or_hit), hit_cmp);
  free(parts);
  free(th);
  *out = all;
  return n;
}

/* ------------------------------------------------------------------------------------------ */
/* pairing                                                                                      */

typedef struct {
  uint32_t record;
  uint32_t pair;
  uint32_t start, end;  /* [start, end) on the top strand */
  uint32_t hit_i, hit_j;
  uint8_t orient;       /* 0 FR, 1 RF, 2 FF, 3 RR */
  uint8_t pad[3];
} or_amp;

/* orientation of an anchor (+ site, primer pi) paired with an antisense site of primer pj */
static int orientation(int pi, int pj) {
  if (pi == 0 && pj == 1) return 0; /* FR */
  if (pi == 1 && pj == 0) return 1; /* RF */
  if (pi == 0 && pj == 0) return 2; /* FF */
  return 3;                          /* RR */
}

int64_t or_pair(const or_hit* hits, int64_t n_hits, const uint32_t* lenF, const uint32_t* lenR,
                uint32_t min_len, uint32_t max_len, uint32_t orient_mask, or_amp** out) {
  int64_t cap = 1024, n = 0;
  or_amp* v = (or_amp*)malloc((size_t)cap * sizeof(or_amp));
  for (int64_t i = 0; i < n_hits; ++i) {
    const or_hit* a = &hits[i];
    if (a->strand != 0) continue; /* anchors are sense (+) sites */
    for (int64_t j = i + 1; j < n_hits; ++j) {
      const or_hit* b = &hits[j];
      if (b->record != a->record || b->pair != a->pair) break;
      if (b->strand == 0) break; /* a same-sense site stops the walk */
      uint32_t Lb = b->primer == 0 ? lenF[b->pair] : lenR[b->pair];
      uint64_t end = (uint64_t)b->pos + Lb;
      uint64_t length = end - a->pos;
      if (length > max_len) break;
      if (length < min_len) continue;
      int o = orientation(a->primer, b->primer);
      if (!((orient_mask >> o) & 1)) continue;
      if (n == cap) {
        cap *= 2;
        v = (or_amp*)realloc(v, (size_t)cap * sizeof(or_amp));
      }
      or_amp m;
      memset(&m, 0, sizeof m);
      m.record = a->record;
      m.pair = a->pair;
      m.start = a->pos;
      m.end = (uint32_t)end;
      m.hit_i = (uint32_t)i;
      m.hit_j = (uint32_t)j;
      m.orient = (uint8_t)o;
      v[n++] = m;
    }
  }
  *out = v;
  return n;
}

/* ------------------------------------------------------------------------------------------ */
/* nearest-neighbour melting temperature                                                        */
/*
 * Duplex notation: "XY/ZW" is the step 5'-XY-3' on the written strand over 3'-ZW-5' on the
 * opposite strand.  dH in kcal/mol, dS in cal/(K mol).
 */
typedef struct {
  const char* key;
  double dh, ds;
} nn_param;

/* Watson-Crick stacks: Allawi & SantaLucia (1997) Biochemistry 36:10581; identical to the
 * unified set of SantaLucia (1998) PNAS 95:1460.  The default set (nn_table 0 or 3). */
static const nn_param WC_STACK[] = {
    {"AA/TT", -7.9, -22.2}, {"AT/TA", -7.2, -20.4}, {"TA/AT", -7.2, -21.3}, {"CA/GT", -8.5, -22.7},
    {"GT/CA", -8.4, -22.4}, {"CT/GA", -7.8, -21.0}, {"GA/CT", -8.2, -22.2}, {"CG/GC", -10.6, -27.2},
    {"GC/CG", -9.8, -24.4}, {"GG/CC", -8.0, -19.9},
};
/* Breslauer et al. (1986) PNAS 83:3746 (nn_table 1). */
static const nn_param WC_BRESLAUER86[] = {
    {"AA/TT", -9.1, -24.0}, {"AT/TA", -8.6, -23.9}, {"TA/AT", -6.0, -16.9}, {"CA/GT", -5.8, -12.9},
    {"GT/CA", -6.5, -17.3}, {"CT/GA", -7.8, -20.8}, {"GA/CT", -5.6, -13.5}, {"CG/GC", -11.9, -27.8},
    {"GC/CG", -11.1, -26.7}, {"GG/CC", -11.0, -26.6},
};
/* Sugimoto et al. (1996) Nucleic Acids Res 24:4501 (nn_table 2). */
static const nn_param WC_SUGIMOTO96[] = {
    {"AA/TT", -8.0, -21.9}, {"AT/TA", -5.6, -15.2}, {"TA/AT", -6.6, -18.4}, {"CA/GT", -8.2, -21.0},
    {"GT/CA", -9.4, -25.5}, {"CT/GA", -6.6, -16.4}, {"GA/CT", -8.8, -23.5}, {"CG/GC", -11.8, -29.0},
    {"GC/CG", -10.5, -26.4}, {"GG/CC", -10.9, -28.4},
};
/* SantaLucia & Hicks (2004) Annu Rev Biophys Biomol Struct 33:415 (nn_table 4). */
static const nn_param WC_SANTALUCIA04[] = {
    {"AA/TT", -7.6, -21.3}, {"AT/TA", -7.2, -20.4}, {"TA/AT", -7.2, -21.3}, {"CA/GT", -8.5, -22.7},
    {"GT/CA", -8.4, -22.4}, {"CT/GA", -7.8, -21.0}, {"GA/CT", -8.2, -22.2}, {"CG/GC", -10.6, -27.2},
    {"GC/CG", -9.8, -24.4}, {"GG/CC", -8.0, -19.9},
};
/* RNA, Freier et al. (1986) PNAS 83:9373 (nn_table 5); U written as T. */
static const nn_param WC_FREIER86[] = {
    {"AA/TT", -6.6, -18.4}, {"AT/TA", -5.7, -15.5}, {"TA/AT", -8.1, -22.6}, {"CA/GT", -10.5, -27.8},
    {"GT/CA", -10.2, -26.2}, {"CT/GA", -7.6, -19.2}, {"GA/CT", -13.3, -35.5}, {"CG/GC", -8.0, -19.4},
    {"GC/CG", -14.2, -34.9}, {"GG/CC", -12.2, -29.7},
};
/* RNA/DNA hybrids, Sugimoto et al. (1995) Biochemistry 34:11211 (nn_table 8): the written strand
 * is the RNA, so all 16 steps are listed as written (U written as T). */
static const nn_param WC_SUGIMOTO95[] = {
    {"AA/TT", -7.8, -21.9}, {"AC/TG", -5.9, -12.3}, {"AG/TC", -9.1, -23.5}, {"AT/TA", -8.3, -23.9},
    {"CA/GT", -9.0, -26.1}, {"CC/GG", -9.3, -23.2}, {"CG/GC", -16.3, -47.1}, {"CT/GA", -7.0, -19.7},
    {"GA/CT", -5.5, -13.5}, {"GC/CG", -8.0, -17.1}, {"GG/CC", -12.8, -31.9}, {"GT/CA", -7.8, -21.6},
    {"TA/AT", -7.8, -23.2}, {"TC/AG", -8.6, -22.9}, {"TG/AC", -10.4, -28.4}, {"TT/AA", -11.5, -36.4},
};

#define NELEM(a) ((int)(sizeof(a) / sizeof((a)[0])))

/* One nearest-neighbour set: its stacks and the scalar terms of Biopython's Tm_NN tables, as
 * dH/dS pairs: "init" (every duplex), "init_A/T" and "init_G/C" (per terminal pair of that kind on
 * the written strand), "init_oneG/C" / "init_allA/T" (the duplex holds some / no G or C),
 * "init_5T/A" (each of a 5' T and a 3' A of the written strand), "sym" (self-complementary). */
typedef struct {
  const nn_param* wc;
  int n_wc;
  double init[2], at[2], gc[2], onegc[2], allat[2], t5a[2], sym[2];
} nn_set;

static const nn_set NN_SETS[] = {
    /* 0 and 3: Allawi & SantaLucia 1997 */
    {WC_STACK, NELEM(WC_STACK), {0, 0}, {2.3, 4.1}, {0.1, -2.8}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},
    {WC_BRESLAUER86, NELEM(WC_BRESLAUER86), {0, 0}, {0, 0}, {0, 0}, {0, -16.8}, {0, -20.1}, {0, 0}, {0, -1.3}},
    {WC_SUGIMOTO96, NELEM(WC_SUGIMOTO96), {0.6, -9.0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},
    {WC_STACK, NELEM(WC_STACK), {0, 0}, {2.3, 4.1}, {0.1, -2.8}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},
    {WC_SANTALUCIA04, NELEM(WC_SANTALUCIA04), {0.2, -5.7}, {2.2, 6.9}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},
    {WC_FREIER86, NELEM(WC_FREIER86), {0, -10.8}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1.4}},
    {NULL, 0, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}}, /* 6: not built */
    {NULL, 0, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}}, /* 7: not built */
    {WC_SUGIMOTO95, NELEM(WC_SUGIMOTO95), {1.9, -3.9}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}},
};

/* the set of nn_table t, NULL when there is none */
static const nn_set* nn_set_of(int t) {
  if (t < 0 || t >= NELEM(NN_SETS) || !NN_SETS[t].wc) return NULL;
  return &NN_SETS[t];
}

/* Internal single mismatches next to a Watson-Crick pair, plus the tandem G.T steps.
 * G.T: Allawi & SantaLucia (1997) Biochemistry 36:10581.  G.A: Allawi & SantaLucia (1998)
 * Biochemistry 37:2170.  C.T: Allawi & SantaLucia (1998) NAR 26:2694.  A.C: Allawi &
 * SantaLucia (1998) Biochemistry 37:9435.  A.A, C.C, G.G, T.T: Peyret et al. (1999)
 * Biochemistry 38:3468. */
static const nn_param INTERNAL_MM[] = {
    /* G.T */
    {"AG/TT", 1.0, 0.9}, {"AT/TG", -2.5, -8.3}, {"CG/GT", -4.1, -11.7}, {"CT/GG", -2.8, -8.0},
    {"GG/CT", 3.3, 10.4}, {"GG/TT", 5.8, 16.3}, {"GT/CG", -4.4, -12.3}, {"GT/TG", 4.1, 9.5},
    {"TG/AT", -0.1, -1.7}, {"TG/GT", -1.4, -6.2}, {"TT/AG", -1.3, -5.3},
    /* G.A */
    {"AA/TG", -0.6, -2.3}, {"AG/TA", -0.7, -2.3}, {"CA/GG", -0.7, -2.3}, {"CG/GA", -4.0, -13.2},
    {"GA/CG", -0.6, -1.0}, {"GG/CA", 0.5, 3.2}, {"TA/AG", 0.7, 0.7}, {"TG/AA", 3.0, 7.4},
    /* C.T */
    {"AC/TT", 0.7, 0.2}, {"AT/TC", -1.2, -6.2}, {"CC/GT", -0.8, -4.5}, {"CT/GC", -1.5, -6.1},
    {"GC/CT", 2.3, 5.4}, {"GT/CC", 5.2, 13.5}, {"TC/AT", 1.2, 0.7}, {"TT/AC", 1.0, 0.7},
    /* A.C */
    {"AA/TC", 2.3, 4.6}, {"AC/TA", 5.3, 14.6}, {"CA/GC", 1.9, 3.7}, {"CC/GA", 0.6, -0.6},
    {"GA/CC", 5.2, 14.2}, {"GC/CA", -0.7, -3.8}, {"TA/AC", 3.4, 8.0}, {"TC/AA", 7.6, 20.2},
    /* A.A, C.C, G.G, T.T */
    {"AA/TA", 1.2, 1.7}, {"CA/GA", -0.9, -4.2}, {"GA/CA", -2.9, -9.8}, {"TA/AA", 4.7, 12.9},
    {"AC/TC", 0.0, -4.4}, {"CC/GC", -1.5, -7.2}, {"GC/CC", 3.6, 8.9}, {"TC/AC", 6.1, 16.4},
    {"AG/TG", -3.1, -9.5}, {"CG/GG", -4.9, -15.3}, {"GG/CG", -6.0, -15.8}, {"TG/AG", 1.6, 3.6},
    {"AT/TT", -2.7, -10.8}, {"CT/GT", -5.0, -15.8}, {"GT/CT", -2.2, -8.4}, {"TT/AT", 0.2, -1.5},
};

/* Terminal mismatches: 5'-XY-3'/3'-X'Y'-5' with X.X' Watson-Crick and the duplex-terminal pair
 * Y.Y' mismatched.  SantaLucia & Peyret (2001) patent application WO 01/94611. */
static const nn_param TERMINAL_MM[] = {
    {"AA/TA", -3.1, -7.8}, {"TA/AA", -2.5, -6.3}, {"CA/GA", -4.3, -10.7}, {"GA/CA", -8.0, -22.5},
    {"AC/TC", -0.1, 0.5},  {"TC/AC", -0.7, -1.3}, {"CC/GC", -2.1, -5.1},  {"GC/CC", -3.9, -10.6},
    {"AG/TG", -1.1, -2.1}, {"TG/AG", -1.1, -2.7}, {"CG/GG", -3.8, -9.5},  {"GG/CG", -0.7, -19.2},
    {"AT/TT", -2.4, -6.5}, {"TT/AT", -3.2, -8.9}, {"CT/GT", -6.1, -16.9}, {"GT/CT", -7.4, -21.2},
    {"AA/TC", -1.6, -4.0}, {"AC/TA", -1.8, -3.8}, {"CA/GC", -2.6, -5.9},  {"CC/GA", -2.7, -6.0},
    {"GA/CC", -5.0, -13.8}, {"GC/CA", -3.2, -7.1}, {"TA/AC", -2.3, -5.9}, {"TC/AA", -2.7, -7.0},
    {"AC/TT", -0.9, -1.7}, {"AT/TC", -2.3, -6.3}, {"CC/GT", -3.2, -8.0},  {"CT/GC", -3.9, -10.6},
    {"GC/CT", -4.9, -13.5}, {"GT/CC", -3.0, -7.8}, {"TC/AT", -2.5, -6.3}, {"TT/AC", -0.7, -1.2},
    {"AA/TG", -1.9, -4.4}, {"AG/TA", -2.5, -5.9}, {"CA/GG", -3.9, -9.6},  {"CG/GA", -6.0, -15.5},
    {"GA/CG", -4.3, -11.1}, {"GG/CA", -4.6, -11.4}, {"TA/AG", -2.0, -4.7}, {"TG/AA", -2.4, -5.8},
    {"AG/TT", -3.2, -8.7}, {"AT/TG", -3.5, -9.4}, {"CG/GT", -3.8, -9.0},  {"CT/GG", -6.6, -18.7},
    {"GG/CT", -5.7, -15.9}, {"GT/CG", -5.9, -16.1}, {"TG/AT", -3.9, -10.5}, {"TT/AG", -3.6, -9.8},
};


static int find_param(const nn_param* t, int n, const char* key, double* dh, double* ds) {
  for (int i = 0; i < n; ++i)
    if (strcmp(t[i].key, key) == 0) {
      *dh += t[i].dh;
      *ds += t[i].ds;
      return 1;
    }
  return 0;
}

/* Read access to one parameter entry, exactly as stored (no lookup rules, no arithmetic), so that
 * tests can hold the tables against published values: table 0 the Watson-Crick stacks of set
 * `set` (nn_table numbering), 1 the internal mismatches, 2 the terminal mismatches, 3 the set's
 * scalar terms ("init", "init_A/T", "init_G/C", "init_oneG/C", "init_allA/T", "init_5T/A",
 * "sym").  Returns 1 if the key exists. */
int or_nn_entry_set(int set, int table, const char* key, double* dh, double* ds) {
  *dh = *ds = 0.0;
  const nn_set* S = nn_set_of(set);
  if (!S) return 0;
  switch (table) {
    case 0: return find_param(S->wc, S->n_wc, key, dh, ds);
    case 1: return find_param(INTERNAL_MM, NELEM(INTERNAL_MM), key, dh, ds);
    case 2: return find_param(TERMINAL_MM, NELEM(TERMINAL_MM), key, dh, ds);
    default: break;
  }
  const struct { const char* key; const double* v; } scalars[] = {
      {"init", S->init},   {"init_A/T", S->at},       {"init_G/C", S->gc}, {"init_oneG/C", S->onegc},
      {"init_allA/T", S->allat}, {"init_5T/A", S->t5a}, {"sym", S->sym},
  };
  for (int i = 0; i < NELEM(scalars); ++i)
    if (strcmp(scalars[i].key, key) == 0) {
      *dh = scalars[i].v[0];
      *ds = scalars[i].v[1];
      return 1;
    }
  return 0;
}

/* the same for the default set */
int or_nn_entry(int table, const char* key, double* dh, double* ds) { return or_nn_entry_set(0, table, key, dh, ds); }

typedef struct {
  double Na, K, Tris, Mg, dNTPs; /* mM */
  double dnac1, dnac2;           /* nM */
  int saltcorr;                  /* 0 none, 1..7 */
  int selfcomp;
  int variants;                  /* 0: every concrete variant (R14); 1: only those matching the site */
  int nn_table;                  /* nearest-neighbour set, Biopython's numbering: 0 or 3 DNA_NN3 (the
                                    default), 1 DNA_NN1, 2 DNA_NN2, 4 DNA_NN4, 5 RNA_NN1, 8 R_DNA_NN1 */
} or_tm_params;

static double gc_fraction(const char* s, int L) {
  int gc = 0, n = 0;
  for (int i = 0; i < L; ++i) {
    char c = (char)toupper((unsigned char)s[i]);
    if (c == 'G' || c == 'C' || c == 'S') ++gc;
    if (code_set(c)) ++n;
  }
  return n ? (double)gc / n : 0.0;
}

/* Free Mg2+ (mM) when dNTPs bind Mg2+ one to one with association constant Ka = 3e4 per M
 * (Owczarzy et al. 2008): with x the free Mg2+, the bound amount Mg - x and the free dNTP
 * dNTP - (Mg - x) satisfy Ka x (dNTP - Mg + x) = Mg - x, whose positive root is taken (in M). */
double or_free_mg(double mg_mM, double dntps_mM) {
  const double ka = 3e4, mg = mg_mM * 1e-3, dn = dntps_mM * 1e-3;
  if (dn <= 0.0) return mg_mM;
  const double b = ka * (dn - mg) + 1.0;
  return 1e3 * (-b + sqrt(b * b + 4.0 * ka * mg)) / (2.0 * ka);
}

/* Salt method 7 (Owczarzy et al. 2008, Mg2+ with monovalent ions): a correction to 1/Tm.  [Mon+]
 * = Na + K + Tris/2 (no Na-equivalent for Mg2+), [Mg2+] free of dNTPs, both in M, f the G/C
 * fraction, N the duplex length:
 *   [Mon+] > 0 and sqrt([Mg2+]) / [Mon+] < 0.22: monovalent ions dominate and the correction is
 *     Owczarzy et al. 2004's (method 6) at [Mon+];
 *   otherwise a + b ln[Mg2+] + f (c + d ln[Mg2+]) + (e + f' ln[Mg2+] + g ln^2[Mg2+]) / (2 (N - 1))
 *     with a = 3.92e-5, b = -9.11e-6, c = 6.26e-5, d = 1.42e-5, e = -4.82e-4, f' = 5.25e-4,
 *     g = 8.31e-5, where for a ratio below 6 the monovalent ions modify three of them:
 *     a *= 0.843 - 0.352 sqrt([Mon+]) ln[Mon+], d *= 1.279 - 4.03e-3 ln[Mon+] - 8.03e-3 ln^2[Mon+],
 *     g *= 0.486 - 0.258 ln[Mon+] + 5.25e-3 ln^3[Mon+].
 * Undefined (*ok = 0) without any cation. */
static double salt_owczarzy2008(const or_tm_params* p, const char* seq, int L, int* ok) {
  const double mon = (p->Na + p->K + p->Tris / 2.0) * 1e-3;
  const double mg = or_free_mg(p->Mg, p->dNTPs) * 1e-3;
  const double f = gc_fraction(seq, L);
  double a = 3.92e-5, b = -9.11e-6, c = 6.26e-5, d = 1.42e-5, e = -4.82e-4, f2 = 5.25e-4, g = 8.31e-5;
  if (mon > 0.0) {
    const double ratio = sqrt(mg) / mon, lm = log(mon);
    if (ratio < 0.22) return (4.29 * f - 3.95) * 1e-5 * lm + 9.40e-6 * lm * lm;
    if (ratio < 6.0) {
      a *= 0.843 - 0.352 * sqrt(mon) * lm;
      d *= 1.279 - 4.03e-3 * lm - 8.03e-3 * lm * lm;
      g *= 0.486 - 0.258 * lm + 5.25e-3 * lm * lm * lm;
    }
  }
  if (!(mg > 0.0)) {
    *ok = 0;
    return 0.0;
  }
  const double lg = log(mg);
  return a + b * lg + f * (c + d * lg) + (e + f2 * lg + g * lg * lg) / (2.0 * (L - 1));
}

/* Salt correction (von Ahsen et al. 2001 Na-equivalent for Mg/dNTPs; methods: 1 Schildkraut &
 * Lifson 1965, 2 Wetmur 1991, 3 SantaLucia et al. 1996, 4 and 5 SantaLucia 1998, 6 Owczarzy et
 * al. 2004, 7 Owczarzy et al. 2008).  Returns 0 with *ok = 0 when the method is not covered. */
static double salt_correction(const or_tm_params* p, const char* seq, int L, int* ok) {
  *ok = 1;
  if (p->saltcorr == 0) return 0.0;
  if (p->saltcorr == 7) return salt_owczarzy2008(p, seq, L, ok);
  double Mon = p->Na + p->K + p->Tris / 2.0;
  if ((p->K + p->Mg + p->Tris + p->dNTPs) > 0 && p->dNTPs < p->Mg) Mon += 120.0 * sqrt(p->Mg - p->dNTPs);
  double mon = Mon * 1e-3;
  if (mon <= 0) {
    *ok = 0;
    return 0.0;
  }
  switch (p->saltcorr) {
    case 1: return 16.6 * log10(mon);
    case 2: return 16.6 * log10(mon / (1.0 + 0.7 * mon));
    case 3: return 12.5 * log10(mon);
    case 4: return 11.7 * log10(mon);
    case 5: return 0.368 * (L - 1) * log(mon);
    case 6: return (4.29 * gc_fraction(seq, L) - 3.95) * 1e-5 * log(mon) + 9.40e-6 * log(mon) * log(mon);
    default: *ok = 0; return 0.0;
  }
}

/*
 * Nearest-neighbour sums of the duplex of `seq` (5'->3', A/C/G/T) with `cseq`, the opposite strand
 * written 3'->5' under it, same length L >= 2.  Returns 0 when a step has no parameter (reading
 * R15).  Order of the model:
 *   1. a mismatched pair at either end next to a Watson-Crick pair is scored from the terminal
 *      mismatch table and leaves the stack;
 *   2. initiation from the written strand's own end bases;
 *   3. the remaining nearest-neighbour steps, each from the internal mismatch table or the
 *      Watson-Crick table, read in either direction.
 * Salt and strand concentration are applied by or_tm_duplex.
 */
int or_duplex_sums_set(int set, const char* seq, const char* cseq, int L, double* dh_out, double* ds_out) {
  double dh = 0.0, ds = 0.0;
  const nn_set* S = nn_set_of(set);
  if (!S) return 0;
  int lo = 0, hi = L; /* active pairs [lo, hi) */
  char key[6];
  if (L < 2) return 0;
  /* 1. terminal mismatches, the left end read from the opposite strand */
  key[0] = cseq[1];
  key[1] = cseq[0];
  key[2] = '/';
  key[3] = seq[1];
  key[4] = seq[0];
  key[5] = 0;
  if (find_param(TERMINAL_MM, NELEM(TERMINAL_MM), key, &dh, &ds)) lo = 1;
  if (hi - lo >= 2) {
    key[0] = seq[hi - 2];
    key[1] = seq[hi - 1];
    key[2] = '/';
    key[3] = cseq[hi - 2];
    key[4] = cseq[hi - 1];
    if (find_param(TERMINAL_MM, NELEM(TERMINAL_MM), key, &dh, &ds)) hi -= 1;
  }
  /* 2. initiation */
  dh += S->init[0];
  ds += S->init[1];
  if (gc_fraction(seq, L) == 0.0) {
    dh += S->allat[0];
    ds += S->allat[1];
  } else {
    dh += S->onegc[0];
    ds += S->onegc[1];
  }
  if (seq[0] == 'T') {
    dh += S->t5a[0];
    ds += S->t5a[1];
  }
  if (seq[L - 1] == 'A') {
    dh += S->t5a[0];
    ds += S->t5a[1];
  }
  for (int e = 0; e < 2; ++e) {
    char c = e == 0 ? seq[0] : seq[L - 1];
    if (c == 'A' || c == 'T') {
      dh += S->at[0];
      ds += S->at[1];
    } else if (c == 'G' || c == 'C') {
      dh += S->gc[0];
      ds += S->gc[1];
    }
  }
  /* 3. stacks */
  for (int i = lo; i + 1 < hi; ++i) {
    char rev[6];
    key[0] = seq[i];
    key[1] = seq[i + 1];
    key[2] = '/';
    key[3] = cseq[i];
    key[4] = cseq[i + 1];
    key[5] = 0;
    for (int c = 0; c < 5; ++c) rev[c] = key[4 - c];
    rev[5] = 0;
    if (find_param(INTERNAL_MM, NELEM(INTERNAL_MM), key, &dh, &ds)) continue;
    if (find_param(INTERNAL_MM, NELEM(INTERNAL_MM), rev, &dh, &ds)) continue;
    if (find_param(S->wc, S->n_wc, key, &dh, &ds)) continue;
    if (find_param(S->wc, S->n_wc, rev, &dh, &ds)) continue;
    return 0;
  }
  *dh_out = dh;
  *ds_out = ds;
  return 1;
}

/* the same with the default set */
int or_duplex_sums(const char* seq, const char* cseq, int L, double* dh_out, double* ds_out) {
  return or_duplex_sums_set(0, seq, cseq, L, dh_out, ds_out);
}

/* Melting temperature (degrees C): salt correction, then Tm = 1000 dH / (dS + R ln(C)) - 273.15
 * with R = 1.987 cal/(K mol) and C = (c1 - c2/2) nM (c1 alone, plus the symmetry term, for a
 * self-complementary duplex).  *defined = 0 when the sums or the salt method are undefined. */
double or_tm_duplex(const char* seq, const char* cseq, int L, const or_tm_params* p, int* defined) {
  double dh = 0.0, ds = 0.0;
  *defined = or_duplex_sums_set(p->nn_table, seq, cseq, L, &dh, &ds);
  if (!*defined) return NAN;
  double k = (p->dnac1 - p->dnac2 / 2.0) * 1e-9;
  if (p->selfcomp) {
    const nn_set* S = nn_set_of(p->nn_table);
    k = p->dnac1 * 1e-9;
    dh += S->sym[0];
    ds += S->sym[1];
  }
  int ok = 1;
  double corr = salt_correction(p, seq, L, &ok);
  if (!ok) {
    *defined = 0;
    return NAN;
  }
  const double R = 1.987;
  if (p->saltcorr == 5) ds += corr;
  double tm = (1000.0 * dh) / (ds + R * log(k)) - 273.15;
  if (p->saltcorr >= 1 && p->saltcorr <= 4) tm += corr;
  if (p->saltcorr == 6 || p->saltcorr == 7) tm = 1.0 / (1.0 / (tm + 273.15) + corr) - 273.15;
  return tm;
}

/*
 * Tm of a (possibly degenerate) primer at a site (reading R14): the maximum over every concrete
 * variant of the primer that has at most k positions differing from the site and none in the
 * last `clamp` positions (k = L, clamp = 0: every variant).  `site` holds the genome bases in the primer's own 5'->3' orientation;
 * the opposite strand under the primer is their complement.  *status: 0 ok, 1 undefined (no
 * qualifying variant, or none whose duplex is defined).
 */
double or_tm_site(const char* primer, const char* site, int L, int k, int clamp, const or_tm_params* p,
                  int* status) {
  char cseq[40], var[40];
  char choices[40][4];
  int nchoice[40], idx[40];
  for (int i = 0; i < L; ++i) {
    cseq[i] = base_complement(site[i]);
    unsigned s = code_set(primer[i]);
    nchoice[i] = 0;
    if (s & 1) choices[i][nchoice[i]++] = 'A';
    if (s & 2) choices[i][nchoice[i]++] = 'C';
    if (s & 4) choices[i][nchoice[i]++] = 'G';
    if (s & 8) choices[i][nchoice[i]++] = 'T';
    idx[i] = 0;
  }
  cseq[L] = 0;
  var[L] = 0;
  double best = -INFINITY;
  int any = 0;
  for (;;) {
    int mism = 0, clamp_ok = 1;
    for (int i = 0; i < L; ++i) {
      var[i] = choices[i][idx[i]];
      if (var[i] != toupper((unsigned char)site[i])) {
        ++mism;
        if (i >= L - clamp) clamp_ok = 0;
      }
    }
    if (clamp_ok && mism <= k) {
      int defined = 0;
      double t = or_tm_duplex(var, cseq, L, p, &defined);
      if (defined) {
        any = 1;
        if (t > best) best = t;
      }
    }
    /* next variant (odometer over the degenerate positions) */
    int i = L - 1;
    while (i >= 0) {
      if (++idx[i] < nchoice[i]) break;
      idx[i] = 0;
      --i;
    }
    if (i < 0) break;
  }
  *status = any ? 0 : 1;
  return any ? best : NAN;
}

/* site bases of a hit, in its primer's 5'->3' orientation */
static void hit_site(const uint8_t* g, const or_hit* h, int L, char* out) {
  if (h->strand == 0) {
    for (int i = 0; i < L; ++i) out[i] = genome_letter(g[h->pos + i]);
  } else {
    for (int i = 0; i < L; ++i) out[i] = base_complement(genome_letter(g[h->pos + L - 1 - i]));
  }
  out[L] = 0;
}

/* Tm of every hit (NaN + status 1 when undefined); k and clamp matter only with variants = 1. */
void or_tm_hits(const uint8_t* seq, const int64_t* offsets, const or_hit* hits, int64_t n_hits,
                const char* const* fwd, const char* const* rev, const uint8_t* k, int clamp,
                const or_tm_params* p, double* tm, uint8_t* status) {
  for (int64_t i = 0; i < n_hits; ++i) {
    const or_hit* h = &hits[i];
    const char* P = h->primer == 0 ? fwd[h->pair] : rev[h->pair];
    int L = (int)strlen(P);
    char site[40];
    hit_site(seq + offsets[h->record], h, L, site);
    int st = 0;
    tm[i] = p->variants ? or_tm_site(P, site, L, k[h->pair], clamp, p, &st) : or_tm_site(P, site, L, L, 0, p, &st);
    status[i] = (uint8_t)st;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* sequences, trimming, barcodes, primer snippets                                               */

static void put_top(const uint8_t* g, int64_t a, int64_t b, char* out) {
  for (int64_t i = a; i < b; ++i) out[i - a] = genome_letter(g[i]);
}

static void put_rc(const uint8_t* g, int64_t a, int64_t b, char* out) {
  for (int64_t i = a; i < b; ++i) out[b - 1 - i] = base_complement(genome_letter(g[i]));
}

static int64_t clip(int64_t x, int64_t len) { return x < 0 ? 0 : (x > len ? len : x); }

/*
 * For amplicon m, five strings: the amplicon (or its trimmed interior), the forward barcode, the
 * reverse barcode, and the bases under each of its two sites in primer orientation (site i, then
 * site j).  Writes field ranges into off[5 * m .. 5 * m + 5] (begin offsets; end = next begin).
 * Two passes: arena == NULL returns the total length.
 */
int64_t or_extract(const uint8_t* seq, const int64_t* offsets, const or_hit* hits, const or_amp* amps,
                   int64_t n_amps, const uint32_t* lenF, const uint32_t* lenR, int trim, int fb, int rb,
                   char* arena, int64_t* off) {
  int64_t w = 0;
  for (int64_t m = 0; m < n_amps; ++m) {
    const or_amp* A = &amps[m];
    const or_hit* hi = &hits[A->hit_i];
    const or_hit* hj = &hits[A->hit_j];
    const uint8_t* g = seq + offsets[A->record];
    int64_t len = offsets[A->record + 1] - offsets[A->record];
    int64_t Li = hi->primer == 0 ? lenF[hi->pair] : lenR[hi->pair];
    int64_t Lj = hj->primer == 0 ? lenF[hj->pair] : lenR[hj->pair];
    int64_t s_i = hi->pos, e_i = hi->pos + Li, s_j = hj->pos, e_j = hj->pos + Lj;
    int rc = A->orient == 1; /* RF is written reverse-complemented */
    /* field 0: amplicon */
    int64_t a = s_i, b = e_j;
    if (trim) {
      a = e_i;
      b = s_j;
      if (b < a) b = a; /* overlapping sites: empty (R11) */
    }
    if (off) off[5 * m + 0] = w;
    if (arena) (rc ? put_rc : put_top)(g, a, b, arena + w);
    w += b - a;
    /* fields 1, 2: barcodes */
    int64_t fa, fbnd, ra, rbnd;
    if (!rc) {
      fa = clip(s_i - fb, len), fbnd = clip(s_i, len);
      ra = clip(e_j, len), rbnd = clip(e_j + rb, len);
    } else {
      fa = clip(e_j, len), fbnd = clip(e_j + fb, len);
      ra = clip(s_i - rb, len), rbnd = clip(s_i, len);
    }
    if (off) off[5 * m + 1] = w;
    if (arena) (rc ? put_rc : put_top)(g, fa, fbnd, arena + w);
    w += fbnd - fa;
    if (off) off[5 * m + 2] = w;
    if (arena) (rc ? put_rc : put_top)(g, ra, rbnd, arena + w);
    w += rbnd - ra;
    /* fields 3, 4: sites in primer orientation */
    if (off) off[5 * m + 3] = w;
    if (arena) (hi->strand == 0 ? put_top : put_rc)(g, s_i, e_i, arena + w);
    w += Li;
    if (off) off[5 * m + 4] = w;
    if (arena) (hj->strand == 0 ? put_top : put_rc)(g, s_j, e_j, arena + w);
    w += Lj;
  }
  if (off) off[5 * n_amps] = w;
  return w;
}

void or_free(void* p) { free(p); }
