// Internal declarations shared by the engine's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <atomic>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <functional>
#include <thread>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ah.h"

namespace ah {

// Base codes of the packed layout: A=0, C=1, T=2, G=3 (bit 0 = ASCII bit 1, bit 1 = ASCII bit 2).
// An IUPAC code is held as a 4-bit set over these codes: bit c set iff code c is allowed.
enum : uint8_t { SET_A = 1, SET_C = 2, SET_T = 4, SET_G = 8 };

// Geometry shared by kernels and host code.
constexpr int kGroupBases = 32;            // bases per plane word
constexpr int kTailGroups = 64;            // zero groups after the last record
// host->device streaming chunk: 256 Mi bases (64 MB packed).  Measured on GB300 from page-locked memory,
// the staged pack reaches 72, 192 and 199 GB/s with 16, 64 and 256 Mi-base chunks (a plain copy: 211).
constexpr uint64_t kChunkBases = 256ull << 20;

// Groups of a record of len bases: whole 64-base blocks (records start 16-byte aligned) with at
// least one padding base after the record, so a window that leaves its record meets an invalid base.
__host__ __device__ inline uint64_t record_groups(uint64_t len) { return (len / 64 + 1) * 2; }

// Device status word bits (set by kernels, read by synchronising calls).
enum : uint32_t {
  ST_SCAN_MISMATCH = 1u << 0,   // bit-sliced matcher and exact re-check disagree
  ST_PAIR_OVERFLOW = 1u << 1,
  ST_BAD_INPUT = 1u << 2,
  ST_TM_LIMIT = 1u << 3,        // a degenerate site Tm needed more than its enumeration bound
};

struct Pattern {
  uint8_t set[32];     // IUPAC set per position, 5'->3' of the oriented pattern on the top strand
  uint8_t len;
  uint8_t clamp_lo;    // clamp positions [clamp_lo, clamp_hi) must match
  uint8_t clamp_hi;
  uint8_t k;
  uint16_t id;         // 4 * pair + orient
};

// One oriented pattern as the generic (compile-free) scan kernel reads it.  The evaluated positions
// (N excluded) come clamp first, then the counted ones most likely to mismatch first; entry e has
// offset j[e] in the window and mismatch bit c0 ^ (lo & c1) ^ (hi & c2) ^ (lo & hi & c3) of the
// base's code bits, x[e] = (c0, c1, c2, c3), each 0 or ~0.  Both sections are padded to multiples
// of 4 entries with x = 0 (never a mismatch): entries [0, n_clamp) are the clamp's, [n_clamp,
// n_eval) the counted positions'.
struct alignas(16) GenPattern {
  uint4 x[40];
  uint8_t j[40];
  uint32_t mset[4];     // bit j of mset[c]: position j's set holds code c (A, C, T, G)
  uint32_t clamp_mask;  // bits of the clamp positions
  uint8_t len, k, n_eval, n_clamp;
  uint16_t pair;
  uint8_t orient;
  uint8_t width;        // counter bits: the least w with 2^w >= k + 1
};
std::vector<GenPattern> gen_table(const std::vector<Pattern>& pats);
constexpr int kGenMaxPatterns = 64;  // patterns per generic launch (the table sits in shared memory)

struct ScanConfig {
  int threads = 128;        // threads per CTA (128 x 8 was fastest for a single pair in a sweep on GB300)
  int groups_per_thread = 8;
  int slot_cap = 256;       // hit slots per tile before overflow
  int shift_mode = 0;       // pattern-position alignment: 0 funnel shifts (ALU pipe), 1 multiply pairs
                            // (FMA pipe), 2 alternate the two
  int persistent = 0;       // 1: CTAs loop over tiles taken from a device counter
  int min_blocks = 0;       // generated kernels: blocks per SM the register allocation must allow
                            // (0: no bound); large circuits run more warps with a few spills
  int pairs_per_kernel = 0; // regular scans: kernels of at most this many pairs, compiled in parallel
                            // and launched one after another (0: one kernel for every pair)
  int emit_queue = 0;       // generated kernels: 0 candidates emitted where found, 1 queued per warp and
                            // emitted by the whole warp after its block (dense sites)
  int vote_windows = 1024;  // generated kernels: windows the phase-split cost model takes one warp vote
                            // to cover (1024 = 32 lanes x 32 positions on uniform random bases; larger
                            // values weigh phase two as if windows survived phase one more often)
};

// default of ah_ctx::tm_split_sites: each launch re-reads the window's site marks, which pays once
// the chains of fewer primers per launch keep the instruction cache warm
constexpr uint64_t kTmSplitSitesDefault = 4ull << 20;

class JitCache;

}  // namespace ah

struct ah_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  cudaMemPool_t pool = nullptr;      // the context's stream-ordered memory pool
  uint8_t* bounce[2] = {nullptr, nullptr};       // page-locked buffers for copies into pageable memory
  cudaEvent_t bounce_ev[2] = {nullptr, nullptr};
  uint32_t* d_status = nullptr;      // device status word
  uint32_t* h_status = nullptr;      // pinned mirror
  ah::JitCache* jit = nullptr;       // the process-wide kernel cache
  std::mutex stats_mu;               // compile counters are updated from compile threads
  ah::ScanConfig scan_cfg;
  int sm_count = 0;
  // diagnostics
  uint64_t n_launches = 0;
  uint64_t n_scan_launches = 0;
  uint64_t scan_bases = 0;
  double scan_ms = 0.0;
  uint64_t jit_compiles = 0;
  double jit_ms = 0.0;
  int scan_ops_per_group = 0;  // of the last scan kernel launched
  // scan kernel choice: 0 generated kernels, 1 the generic kernel, 2 the generic kernel while a
  // primer set's generated kernels compile, 3 a fixed hand-over (see launch_scan)
  int generic_scan = 0;
  uint64_t n_generic_scans = 0;
  uint64_t generic_bases = 0;  // bases those scans covered with the generic kernel (tile granularity)
  // mode 2: compiles running on threads of this context, each with the flag it sets when done
  // (1 compiled, 2 failed); finished ones are joined when the next starts, the rest on destroy
  std::mutex compile_mu;
  std::vector<std::pair<std::thread, std::shared_ptr<std::atomic<int>>>> compiles;
  bool timing = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // scan-node timings of graph replays: event pairs recorded by the graph, read when the stream is
  // next synchronised (ah::drain_timings), which also advances drain_gen
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  uint64_t drain_gen = 0;
  // fault injection on the host: this many of the next device allocations fail with AH_ENOMEM
  int fail_allocs = 0;
  // degenerate-site Tm kernel: 0 the kernel generated for the primer set (compiled on first use),
  // 1 the built-in kernel, 2 the built-in kernel while the generated one compiles in the background
  int tm_kernel = 0;
  uint64_t tm_split_sites = ah::kTmSplitSitesDefault;  // see ah::TmKernel::split_sites
  uint64_t n_tm_generated = 0;  // Tm launches (outside plans) by a generated kernel
  uint64_t n_tm_builtin = 0;    // ... by the built-in one
};

struct ah_batch {
  ah_ctx* ctx = nullptr;
  uint32_t n_records = 0;
  uint64_t n_bases = 0;
  uint64_t n_groups = 0;      // covered by records (padding included)
  uint64_t alloc_groups = 0;  // n_groups + tail
  uint2* planes = nullptr;
  uint32_t* invalid = nullptr;
  uint64_t* rec_group = nullptr;
  uint32_t* rec_len = nullptr;
  uint32_t* genome_id = nullptr;
  std::vector<uint64_t> h_rec_group;
  std::vector<uint32_t> h_rec_len;
  bool view = false;          // a slice: planes, invalid, rec_len and genome_id belong to another batch
};

struct ah_primers {
  ah_ctx* ctx = nullptr;
  uint32_t n_pairs = 0;
  uint8_t clamp = 0;
  std::vector<std::string> fwd, rev;   // upper-case
  std::vector<uint8_t> k;
  std::vector<ah::Pattern> pats;       // 4 per pair, index 4 * pair + orient
  // device copies for pairing / Tm / extraction
  uint8_t* d_plen = nullptr;           // per pattern length
  uint8_t* d_psets = nullptr;          // [n_pairs][2 primers][32] IUPAC sets of the primers as written
  uint8_t* d_pk = nullptr;             // [n_pairs] mismatch budget
  uint4* d_pmask = nullptr;            // [n_pairs][2 primers] position masks per base code (A, C, T, G)
  ah::GenPattern* d_gen = nullptr;     // the patterns as the generic scan kernel reads them
};

struct ah_quals {
  ah_ctx* ctx = nullptr;
  uint32_t n_records = 0;
  uint8_t* d_qual = nullptr;      // every record's qualities back to back
  uint64_t* d_off = nullptr;      // n_records + 1
  std::vector<uint64_t> h_off;
};

struct ah_hits {
  ah_ctx* ctx = nullptr;
  uint64_t n = 0;
  uint32_t n_pairs = 0;
  ah_hit* d = nullptr;
  uint64_t* d_pair_off = nullptr;      // n_pairs + 1
  std::vector<uint64_t> h_pair_off;
};

struct ah_amplicons {
  ah_ctx* ctx = nullptr;
  uint64_t n = 0;
  ah_amplicon* d = nullptr;
  char* d_arena = nullptr;
  uint64_t arena_bytes = 0;
  uint64_t* d_field_off = nullptr;     // 5 n + 1 when extracted
  int trim = 0;                        // of the last extraction
  char* d_qarena = nullptr;            // qualities of field 0 at its arena offsets (ah_extract_qualities)
};

namespace ah {

// ---- error helpers -----------------------------------------------------------------------
ah_status fail(ah_ctx* ctx, ah_status st, const char* fmt, ...);
#define AH_CUDA(ctx, call)                                                                      \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return ::ah::fail((ctx), AH_ECUDA, "%s failed: %s (%s:%d)", #call, \
                                             cudaGetErrorString(e_), __FILE__, __LINE__);       \
  } while (0)

// ---- device memory (stream-ordered pool) ---------------------------------------------------
template <class T>
ah_status dalloc(ah_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (ctx->fail_allocs > 0) {
    ctx->fail_allocs--;
    return fail(ctx, AH_ENOMEM, "device allocation of %zu bytes failed: injected failure", count * sizeof(T));
  }
  cudaError_t e = cudaMallocFromPoolAsync((void**)p, count * sizeof(T), ctx->pool, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, AH_ENOMEM, "device allocation of %zu bytes failed: %s", count * sizeof(T),
                                    cudaGetErrorString(e));
  return AH_OK;
}
void dfree(ah_ctx* ctx, void* p);

// ---- exclusive scan over counts: out[i] = sum(in[0..i)), out[n] = total ------------------------
ah_status exclusive_scan_u32(ah_ctx* ctx, const uint32_t* d_in, uint64_t* d_out, uint64_t n);
ah_status exclusive_scan_u64(ah_ctx* ctx, const uint64_t* d_in, uint64_t* d_out, uint64_t n);
// device -> host copy into caller memory, synchronous: page-locked destinations directly, pageable
// ones through the context's two page-locked bounce buffers, so that no copy takes the driver's
// pageable path (one staging pipeline for every stream of the process)
ah_status copy_to_host(ah_ctx* ctx, void* dst, const void* src, uint64_t bytes);
constexpr uint64_t kBounceBytes = 8ull << 20;  // each of a context's two bounce buffers
// read one uint64 from device memory (synchronises the stream)
ah_status read_u64(ah_ctx* ctx, const uint64_t* d, uint64_t* h);
// A batch of n records whose bases lie in device memory at d_seq[rank[r], rank[r + 1]) (rank[n] =
// total), with the ranks both on the device (d_rank, n values) and on the host (h_rank, n + 1
// values).  Lengths, group offsets and packing items are computed on the device; the batch's host
// record table from h_rank; no per-record array crosses the host link.  The caller has checked that
// the ranks do not decrease and that every record is shorter than 2^32 bases (the device reads each
// record's bytes by them).  Synchronises.
ah_status pack_batch_ranked(ah_ctx* ctx, uint32_t n, const uint8_t* d_seq, const uint64_t* d_rank,
                            const uint64_t* h_rank, const uint32_t* genome_ids, ah_batch** out);
// Repack every record of b from host (or device) memory at h_seq[h_offsets[r], h_offsets[r + 1]) in
// staged chunks, calling on_chunk after each chunk's packing is enqueued on ctx->stream with the
// number of leading groups it completes (b->n_groups for the last).  Returns without waiting for
// the stream.
ah_status pack_host_staged(ah_ctx* ctx, ah_batch* b, const uint8_t* h_seq, const uint64_t* h_offsets,
                           const std::function<void(uint64_t)>& on_chunk);
// The batch's invalid words from a sparse host list (groups already checked against the batch), in
// two steps on the context's stream: the list's upload (copies), then every word cleared and the
// listed ones written (kernels), which also releases the list.
struct InvalidList {
  uint64_t n = 0;
  uint64_t* groups = nullptr;
  uint32_t* words = nullptr;
};
ah_status upload_invalid_list(ah_ctx* ctx, uint64_t n_invalid, const uint64_t* inv_groups, const uint32_t* inv_words,
                              InvalidList* out);
ah_status scatter_invalid_list(ah_ctx* ctx, ah_batch* b, InvalidList* l);
// The batch's records laid end to end in device memory (record r's bases at d_src[start[r],
// start[r] + its length)), packed into the batch as they become available: every call packs what
// lies below `to` and the cursor has not packed yet (a record not complete in whole groups only),
// and returns in done_groups the groups written so far from the batch's first (all of a record's
// padding groups once it is complete).  Enqueued on the context's stream.
struct ConcatCursor {
  uint32_t r = 0;     // the first record not packed completely
  uint64_t off = 0;   // its bases packed
};
ah_status pack_concat_upto(ah_ctx* ctx, ah_batch* b, const uint8_t* d_src, const uint64_t* start, uint64_t to,
                           ConcatCursor* cur, uint64_t* done_groups);
// FASTA text into an existing batch (as ah_fasta_pack_into) with a hook that packs the compacted
// record bases chunk by chunk (see fasta_pack in ah_fasta.cu)
using FastaChunkHook = std::function<ah_status(const uint8_t* d_concat, uint64_t avail, bool last)>;
ah_status fasta_pack_hooked(ah_ctx* ctx, const char* text, uint64_t n_bytes, ah_batch* into, const FastaChunkHook& hook);
// read and clear the device status word (synchronises)
ah_status check_status(ah_ctx* ctx);
// accumulate the pending scan-node timings of graph replays into the context's counters (syncs)
ah_status drain_timings(ah_ctx* ctx);

// count a kernel launch of this context (diagnostics)
inline void launched(ah_ctx* ctx, uint64_t n = 1) { ctx->n_launches += n; }

// scan pipeline (ah_scan.cu)
ah_status scan_primers(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out);
ah_status scan_primers_per_record(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out);
// pairing (ah_pair.cu)
ah_status pair_amplicons(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, uint32_t min_len,
                         uint32_t max_len, uint32_t orient_mask, ah_amplicons** out);
// the allocation-free pairing's device array, loaded on the current device (ah_pair.cu)
cudaError_t noalloc_prepare();
// melting temperature (ah_tm.cu)
ah_status tm_filter(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, ah_amplicons* a,
                    const ah_tm_params* params);
ah_status tm_duplexes(ah_ctx* ctx, uint32_t n, const char* const* seqs, const char* const* cseqs,
                      const ah_tm_params* params, double* out);
ah_status tm_sites(ah_ctx* ctx, uint32_t n, const char* const* primers, const char* const* sites, const uint8_t* k,
                   const uint8_t* clamp, const ah_tm_params* params, double* out);
// extraction (ah_extract.cu)
ah_status extract(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, ah_amplicons* a, int trim,
                  uint32_t fb, uint32_t rb);

// ---- stream-level launchers used by captured plans (no allocation, no host synchronisation) -----
struct ScanKernel;
uint64_t scan_scratch_elems(uint64_t n);
void exclusive_scan_u32_s(cudaStream_t s, const uint32_t* d_in, uint64_t* d_out, uint64_t n, uint64_t* scratch);
void exclusive_scan_u64_s(cudaStream_t s, const uint64_t* d_in, uint64_t* d_out, uint64_t n, uint64_t* scratch);
void launch_scan_kernel(cudaStream_t s, const ScanKernel& k, const ah_batch* b, uint64_t* slots, uint32_t* tile_count,
                        uint32_t cap, uint32_t* status, unsigned long long* work, uint64_t n_tiles, int grid);
// a one-CTA-per-tile kernel over groups [g0, g1) of b (g0 a multiple of the tile, g1 of it or the end)
void launch_scan_range(cudaStream_t s, const ScanKernel& k, const ah_batch* b, uint64_t* slots, uint32_t* tile_count,
                       uint32_t cap, uint32_t* status, uint64_t g0, uint64_t g1);
void launch_tile_max(cudaStream_t s, const uint32_t* tile_count, uint64_t n_tiles, uint32_t* out);
// sorts every tile's keys and counts them per pair; big: n_tiles + 1 words of device scratch, used
// when cap exceeds 256; returns the kernels launched
int launch_tile_sort(cudaStream_t s, uint64_t* slots, const uint32_t* tile_count, uint32_t cap, uint64_t n_tiles,
                     uint32_t n_pairs, uint32_t* tpc, uint32_t* big, int sm_count);
void launch_emit_hits(cudaStream_t s, const uint64_t* slots, const uint32_t* tile_count, uint32_t cap, uint64_t n_tiles,
                      uint64_t tile_groups, const uint64_t* off, const ah_batch* b, ah_hit* hits,
                      const uint64_t* tile_base, uint64_t hit_cap, uint32_t* overflow, uint64_t* pair_off,
                      uint32_t n_pairs);
void launch_pair_walk(cudaStream_t s, bool emit, const ah_hit* hits, uint64_t cap, const uint64_t* d_n,
                      const uint64_t* pair_off, const uint8_t* plen, uint32_t min_len, uint32_t max_len, uint32_t mask,
                      uint32_t* counts, const uint64_t* out_off, ah_amplicon* out, uint64_t out_cap,
                      uint32_t* overflow);
constexpr size_t kTmRunBytes = 256;  // room for the Tm run constants a plan keeps
ah_status tm_prepare(ah_ctx* ctx, const ah_tm_params* params, void* run_out, size_t run_size);
// A degenerate-site Tm kernel generated for one primer set (ah_tm_jit.cpp); fn null: the built-in one.
struct TmKernel {
  cudaKernel_t fn = nullptr;
  int weight_words = 0;        // weight words per thread
  const int32_t* image = nullptr;  // the parameter tables as the kernel's shared memory holds them
  uint64_t split_sites = ~0ull;    // site capacity from which it is launched once per group of primers
};
// Larger primer sets take the built-in kernel: compile time grows with the primers and, about 40 ms
// each, with the transitions between adjacent degenerate positions.
constexpr int kTmJitMaxPrimers = 32;
constexpr int kTmJitMaxAdjacent = 96;
// transitions between adjacent degenerate positions over a set's distinct primers
int tm_chain_adjacent(const std::vector<std::string>& primers);
// The kernel for p by the context's choice (ctx->tm_kernel): generated (compiled now if need be,
// unless !wait and mode 2), or fn = null for the built-in kernel.
// slot: the nearest-neighbour set of the run (tm_run_slot), whose tables the kernel reads.
ah_status tm_kernel_for(ah_ctx* ctx, const ah_primers* p, bool wait, int slot, TmKernel* out);
int tm_run_slot(const void* run);
std::string tm_chain_source(const std::vector<std::string>& primers, int* weight_words);
size_t tm_run_bytes();
// the parameter tables of nearest-neighbour set `slot` laid out as the generated kernels copy them
// into shared memory, on ctx's device (built once per device and set)
ah_status tm_tab_image(ah_ctx* ctx, int slot, const int32_t** out);
void launch_tm(cudaStream_t s, const void* run, const ah_hit* hits, uint64_t hit_cap, const uint64_t* d_nhits,
               const ah_primers* p, uint32_t* status, const uint2* planes, const uint64_t* rec_group, double* hit_tm,
               ah_amplicon* amps, uint64_t amp_cap, const uint64_t* d_namps, int filter, double min_tm, uint32_t* keep,
               uint32_t* defer, int sm_count, const TmKernel& tk);
void launch_compact_amps(cudaStream_t s, const ah_amplicon* in, uint64_t cap, const uint32_t* keep, const uint64_t* off,
                         ah_amplicon* out);
void launch_extract(cudaStream_t s, bool write, const ah_amplicon* amps, uint64_t cap, const uint64_t* d_n,
                    const ah_hit* hits, const uint2* planes, const uint32_t* invalid, const uint64_t* rec_group,
                    const uint32_t* rec_len, const uint8_t* plen, int trim, uint32_t fb, uint32_t rb, uint64_t* len_or_base,
                    char* arena, uint64_t* field_off, uint64_t arena_cap, uint32_t* overflow);

// ---- run-time specialised scan kernels (ah_jit.cpp) ------------------------------------------
struct ScanKernel {
  cudaKernel_t fn = nullptr;
  int threads = 0, groups_per_thread = 0;
  int alu_ops_per_group = 0;  // LOP3 + funnel-shift instructions of the generated circuit per 32 positions
};
std::string scan_source(const std::vector<Pattern>& pats, const ScanConfig& cfg, int* alu_ops_per_group = nullptr);
// NVRTC for this device's architecture (host work only); fills cubin or returns a message
ah_status nvrtc_compile(int device, const std::string& src, const char* name, std::vector<char>* cubin,
                        std::string* err);
// the same for compute capability sm (e.g. 103), with no device needed
ah_status nvrtc_compile_sm(int sm, const std::string& src, const char* name, std::vector<char>* cubin,
                           std::string* err);
// Generated scan kernels, one process-wide cache keyed by source text: a kernel is compiled once,
// callers that ask for it while it compiles wait for that compile.  Kernels stay loaded for the
// life of the process.
class JitCache {
 public:
  static JitCache& global();
  ah_status get(ah_ctx* ctx, const std::vector<Pattern>& pats, const ScanConfig& cfg, ScanKernel* out);
  // several pattern sets, the missing kernels compiled on parallel host threads
  ah_status get_many(ah_ctx* ctx, const std::vector<std::vector<Pattern>>& sets, const ScanConfig& cfg,
                     std::vector<ScanKernel>* out);
  // every set's kernel compiled and loaded for this device (starts no compile)
  bool ready(int device, const std::vector<std::vector<Pattern>>& sets, const ScanConfig& cfg);
  // compiles the sets' missing kernels for this device (parallel host threads) without loading
  // them (the first get loads) and returns the first failure's status; for a background thread
  // (stats: the context whose compile counters it adds to, or null; reports no error to it)
  ah_status prefetch(int device, ah_ctx* stats, const std::vector<std::vector<Pattern>>& sets,
                     const ScanConfig& cfg);
 private:
  struct Entry;
  // stats: the context whose compile counters a compile adds to (may be null); load_it: load the
  // kernel into the process and fill out (else compile only)
  ah_status get_impl(int device, ah_ctx* stats, const std::vector<Pattern>& pats, const ScanConfig& cfg,
                     ScanKernel* out, std::string* err, bool load_it);
  void many_impl(int device, ah_ctx* stats, const std::vector<std::vector<Pattern>>& sets, const ScanConfig& cfg,
                 std::vector<ScanKernel>* out, std::vector<ah_status>* st, std::vector<std::string>* err,
                 bool load_it);
  std::mutex mu_;
  std::unordered_map<std::string, std::shared_ptr<Entry>> cache_;
  // fn(0..n-1) on the compile workers and the calling thread.  The workers start on first use and
  // live for the process, so a compile does not pay for starting a thread.
  void run_parallel(size_t n, const std::function<void(size_t)>& fn);
  std::mutex pool_mu_;
  std::condition_variable pool_cv_;
  std::deque<std::function<void()>> tasks_;
  std::vector<std::thread> workers_;
};

// the pattern sets a scan with cfg.pairs_per_kernel launches, in pair order
std::vector<std::vector<Pattern>> scan_groups(const std::vector<Pattern>& pats, const ScanConfig& cfg);

}  // namespace ah
