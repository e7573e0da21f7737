/*
 * Seeded synthetic-input generator: bulk base filling for genome records.
 *
 * This module only draws random inputs (bases, runs of N, tandem repeats). It holds none of the
 * in-silico PCR arithmetic and is shared by the oracle tests, the CUDA-path tests and the bench.
 *
 * Randomness is counter based: value(key, i) = mix64(key + (i + 1) * GOLDEN), where mix64 is the
 * SplitMix64 output function (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014).  Every draw is a pure function of (seed-derived key, counter), so the
 * host and any other implementation produce identical genomes.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>
#include <stdlib.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }

/* uniform double in [0,1) from the top 53 bits */
static inline double unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

uint64_t synth_mix64(uint64_t z) { return mix64(z); }
uint64_t synth_draw(uint64_t key, uint64_t i) { return draw(key, i); }

/* iid bases with P(G)=P(C)=gc/2, P(A)=P(T)=(1-gc)/2, position i uses counter first + i */
void synth_fill_bases(uint8_t* out, uint64_t n, uint64_t key, double gc, uint64_t first) {
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t r = draw(key, first + i);
    double u = unit(r);
    if (u < gc)
      out[i] = (r & 1) ? 'G' : 'C';
    else
      out[i] = (r & 1) ? 'A' : 'T';
  }
}

/*
 * Runs of 'N': gaps between runs are exponential with mean chosen so that the expected fraction
 * of N positions is `frac`; run lengths are uniform on {1..run_max}.  Sequential in the record.
 * synth_nrun_list writes up to `cap` runs (start, length) and returns how many there are;
 * synth_fill_nruns writes them into a record and returns the number of N positions.
 */
uint64_t synth_nrun_list(uint64_t n, uint64_t key, double frac, uint32_t run_max, uint64_t* starts, uint32_t* lens,
                         uint64_t cap) {
  if (frac <= 0.0 || run_max == 0 || n == 0) return 0;
  double mean_run = 0.5 * (1.0 + (double)run_max);
  double mean_gap = mean_run * (1.0 - frac) / frac;
  uint64_t c = 0, pos = 0, runs = 0;
  pos = (uint64_t)floor(-log(1.0 - unit(draw(key, c++))) * mean_gap);
  while (pos < n) {
    uint64_t len = 1 + draw(key, c++) % run_max;
    if (pos + len > n) len = n - pos;
    if (runs < cap) {
      starts[runs] = pos;
      lens[runs] = (uint32_t)len;
    }
    ++runs;
    pos += len;
    pos += 1 + (uint64_t)floor(-log(1.0 - unit(draw(key, c++))) * mean_gap);
  }
  return runs;
}

uint64_t synth_fill_nruns(uint8_t* out, uint64_t n, uint64_t key, double frac, uint32_t run_max) {
  if (frac <= 0.0 || run_max == 0 || n == 0) return 0;
  uint64_t cnt = synth_nrun_list(n, key, frac, run_max, NULL, NULL, 0);
  uint64_t* st = (uint64_t*)malloc((cnt ? cnt : 1) * sizeof(uint64_t));
  uint32_t* ln = (uint32_t*)malloc((cnt ? cnt : 1) * sizeof(uint32_t));
  synth_nrun_list(n, key, frac, run_max, st, ln, cnt);
  uint64_t total = 0;
  for (uint64_t r = 0; r < cnt; ++r) {
    memset(out + st[r], 'N', ln[r]);
    total += ln[r];
  }
  free(st);
  free(ln);
  return total;
}

/* tandem repeat: a random unit of `period` bases copied over [0, n) */
void synth_fill_tandem(uint8_t* out, uint64_t n, uint64_t key, uint32_t period) {
  static const char acgt[4] = {'A', 'C', 'G', 'T'};
  uint8_t unit_bases[64];
  if (period == 0 || period > 64) return;
  for (uint32_t j = 0; j < period; ++j) unit_bases[j] = (uint8_t)acgt[draw(key, j) & 3];
  for (uint64_t i = 0; i < n; ++i) out[i] = unit_bases[i % period];
}
