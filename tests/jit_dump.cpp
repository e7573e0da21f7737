// Test helper: print the scan kernel source the engine generates for a primer set, or (first
// argument "gen") the pattern table of the generic scan kernel, one pattern per block:
//   len k n_eval n_clamp width clamp_mask mset0 mset1 mset2 mset3
//   then n_eval lines "j c0 c1 c2 c3" (coefficients as 0 / 4294967295)
// usage: jit_dump [gen] [compile] [shift=N] [windows=N] [queue=N] [persistent=N] [min_blocks=N]
//                 k clamp primer [primer ...]
// (each primer gives its + and - strand patterns; shift=N sets the scan source's shift mode, 0 by
// default; windows=N the windows per warp vote its phase split is drawn for, 1024 by default;
// queue=1 the candidate queue; persistent=1 the persistent form; min_blocks=N the register bound.
// "compile" compiles the source for sm_103a with NVRTC, no device needed, and prints
// "compiled <cubin bytes>" or the compiler's log; "ops" prints the circuit's LOP3/SHF count per 32
// positions with every phase run.  A primer may carry its own mismatch budget as "PRIMER:k".)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../paper_2511_00170_gb300/csrc/ah_internal.h"

static uint8_t set_of(char c) {
  switch (c) {
    case 'A': return 1; case 'C': return 2; case 'T': return 4; case 'G': return 8;
    case 'R': return 9; case 'Y': return 6; case 'S': return 10; case 'W': return 5; case 'K': return 12;
    case 'M': return 3; case 'B': return 14; case 'D': return 13; case 'H': return 7; case 'V': return 11;
    default: return 15;
  }
}
static uint8_t comp(uint8_t s) { return (uint8_t)(((s & 1) << 2) | ((s & 4) >> 2) | ((s & 2) << 2) | ((s & 8) >> 2)); }

int main(int argc, char** argv) {
  const bool gen = argc > 1 && !strcmp(argv[1], "gen");
  if (gen) ++argv, --argc;
  const bool compile = argc > 1 && !strcmp(argv[1], "compile");
  if (compile) ++argv, --argc;
  const bool ops_only = argc > 1 && !strcmp(argv[1], "ops");
  if (ops_only) ++argv, --argc;
  int shift_mode = 0, windows = 1024, queue = 0, persistent = 0, min_blocks = 0;
  if (argc > 1 && !strncmp(argv[1], "shift=", 6)) shift_mode = atoi(argv[1] + 6), ++argv, --argc;
  if (argc > 1 && !strncmp(argv[1], "windows=", 8)) windows = atoi(argv[1] + 8), ++argv, --argc;
  if (argc > 1 && !strncmp(argv[1], "queue=", 6)) queue = atoi(argv[1] + 6), ++argv, --argc;
  if (argc > 1 && !strncmp(argv[1], "persistent=", 11)) persistent = atoi(argv[1] + 11), ++argv, --argc;
  if (argc > 1 && !strncmp(argv[1], "min_blocks=", 11)) min_blocks = atoi(argv[1] + 11), ++argv, --argc;
  const int k = atoi(argv[1]), clamp = atoi(argv[2]);
  std::vector<ah::Pattern> pats;
  for (int a = 3; a < argc; ++a)
    for (int strand = 0; strand < 2; ++strand) {
      ah::Pattern P;
      memset(&P, 0, sizeof P);
      const char* pr = argv[a];
      const char* colon = strchr(pr, ':');
      const int L = colon ? (int)(colon - pr) : (int)strlen(pr);
      P.len = (uint8_t)L;
      P.k = (uint8_t)(colon ? atoi(colon + 1) : k);
      P.id = (uint16_t)pats.size();
      for (int j = 0; j < L; ++j) P.set[j] = strand == 0 ? set_of(pr[j]) : comp(set_of(pr[L - 1 - j]));
      P.clamp_lo = (uint8_t)(strand == 0 ? L - clamp : 0);
      P.clamp_hi = (uint8_t)(strand == 0 ? L : clamp);
      pats.push_back(P);
    }
  if (gen) {
    for (const ah::GenPattern& G : ah::gen_table(pats)) {
      printf("%d %d %d %d %d %u %u %u %u %u\n", G.len, G.k, G.n_eval, G.n_clamp, G.width, G.clamp_mask, G.mset[0],
             G.mset[1], G.mset[2], G.mset[3]);
      for (int e = 0; e < G.n_eval; ++e) printf("%d %u %u %u %u\n", G.j[e], G.x[e].x, G.x[e].y, G.x[e].z, G.x[e].w);
    }
    return 0;
  }
  ah::ScanConfig cfg;
  cfg.shift_mode = shift_mode;
  cfg.vote_windows = windows;
  cfg.emit_queue = queue;
  cfg.persistent = persistent;
  cfg.min_blocks = min_blocks;
  int ops = 0;
  const std::string src = ah::scan_source(pats, cfg, &ops);
  if (ops_only) {
    printf("%d\n", ops);
    return 0;
  }
  if (!compile) {
    puts(src.c_str());
    return 0;
  }
  std::vector<char> cubin;
  std::string err;
  if (ah::nvrtc_compile_sm(103, src, "ah_scan_jit.cu", &cubin, &err) != AH_OK) {
    printf("error: %s\n", err.c_str());
    return 1;
  }
  printf("compiled %zu\n", cubin.size());
  return 0;
}
