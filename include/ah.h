/*
 * ah.h -- C ABI of the GB300 in-silico PCR engine.
 *
 * The engine implements the hot path of AmpliconHunter2 (Howard-Stone & Mandoiu, arXiv
 * 2511.00170):
 *   1. pack genome records to 2 bits (Abstract; Section "Implementations", AHv2.alpha);
 *   2. scan both strands for degenerate primers with <= k mismatches and an exact 3' clamp
 *      (Supplementary, "Primer matching and clamp logic");
 *   3. pair sites into FR/RF/FF/RR amplicons inside a length window, stopping at the next
 *      same-sense site (Supplementary, "Amplicon calling and orientation");
 *   4. nearest-neighbour melting temperature in double precision and an optional minimum-Tm
 *      filter (Section "Implementations", AHv2; Section "Primer degeneracy");
 *   5. amplicon sequences, primer trimming, flanking barcodes and primer-site snippets
 *      (Supplementary, "Primer trimming and barcode extraction", "Headers and outputs").
 *
 * Conventions
 *   - Every call returns ah_status.  On failure the context keeps a message for ah_last_error().
 *   - Work is enqueued on the context's CUDA stream.  Calls that must size an output read a count
 *     back from the device and therefore synchronise that stream; this is stated per call.
 *   - Objects (ah_batch, ah_primers, ah_hits, ah_amplicons) are owned by the library and released
 *     only by their ah_*_free call, which enqueues the release on the owning context's stream.
 *     Freeing NULL is a no-op.  A packed batch may be read by any context on the same device (the
 *     serving loop's workers share one); other objects are used with the context that made them.
 *   - Host pointers are plain host memory (pinned memory makes copies asynchronous and fast).
 *   - Device-side checks never trap: a kernel that detects an inconsistency sets a status word
 *     that the next synchronising call turns into AH_EINTERNAL (AH_ELIMIT for a degenerate-site Tm
 *     over its work bound).  No kernel waits on another, so no call waits on the device unbounded.
 *   - All sizes are in bases unless stated otherwise.
 */
#ifndef AH_H
#define AH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AH_OK = 0,
  AH_EINVAL = 1,     /* invalid argument (bad IUPAC code, sizes, parameters) */
  AH_ENOMEM = 2,     /* device or host allocation failed */
  AH_ECUDA = 3,      /* a CUDA runtime/driver call failed */
  AH_EOVERFLOW = 4,  /* an output would exceed a caller-given capacity */
  AH_ETIMEOUT = 5,   /* a bounded device wait ran out */
  AH_EJIT = 6,       /* run-time compilation of a specialised kernel failed */
  AH_EINTERNAL = 7,  /* a device self-check failed */
  AH_ELIMIT = 8,     /* an exact computation would exceed its work bound (degenerate site Tm) */
  AH_ECANCELED = 9   /* a served request was cancelled (ah_server_cancel) */
} ah_status;

typedef struct ah_ctx ah_ctx;
typedef struct ah_batch ah_batch;
typedef struct ah_primers ah_primers;
typedef struct ah_hits ah_hits;
typedef struct ah_amplicons ah_amplicons;

/* ------------------------------------------------------------------------------------------ */
/* context                                                                                      */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to enqueue on, or
 * NULL for a stream the context creates (non-blocking) and destroys. */
ah_status ah_ctx_create(ah_ctx** out, int device, void* cuda_stream);
void ah_ctx_destroy(ah_ctx* ctx);
/* Message of the last failing call on this context (owned by the context, valid until the next
 * call). */
const char* ah_last_error(const ah_ctx* ctx);
/* Wait for all work enqueued on the context's stream and report device self-check failures. */
ah_status ah_ctx_synchronize(ah_ctx* ctx);
/* The stream the context enqueues on (a cudaStream_t). */
void* ah_ctx_stream(const ah_ctx* ctx);

/* Diagnostics of one context (not part of the paper's method): how many kernels it launched,
 * and, when timing is enabled, the device time of the bit-sliced scan kernel measured with CUDA
 * events recorded on the context's stream around each of its launches. */
typedef struct {
  uint64_t kernel_launches; /* kernels launched by this context since the last reset (a plan replay
                               counts every kernel node of its graph) */
  uint64_t scan_launches;   /* scans of a batch (a scan may launch one kernel per pair group;
                               timed ones only, for plan replays) */
  double scan_ms;           /* summed device time of those launches (timing enabled) */
  uint64_t scan_bases;      /* bases covered by those launches */
  uint64_t jit_compiles;    /* scan kernels compiled at run time (NVRTC), background compiles of
                               generic-scan mode 2 included (counted when they finish) */
  double jit_ms;            /* host time spent compiling them */
  int32_t scan_ops_per_group; /* ALU instructions (LOP3 and funnel shifts) of the last scan's
                                 generated circuits (all its kernels) per 32 positions; 0 after a
                                 scan by the generic kernel */
  uint64_t generic_scans;   /* scans run by the generic (compile-free) kernel, wholly or in part */
  uint64_t generic_bases;   /* bases of those scans the generic kernel covered (whole tiles) */
  uint64_t tm_generated;    /* degenerate-site Tm launches of ah_tm_filter by a kernel generated for
                               the primer set (see ah_ctx_set_tm_kernel) */
  uint64_t tm_builtin;      /* ... by the kernel built into the library */
} ah_ctx_stats;
ah_status ah_ctx_stats_get(const ah_ctx* ctx, ah_ctx_stats* out);
ah_status ah_ctx_stats_reset(ah_ctx* ctx);
/* Regular scans (ah_scan_primers) of this context generate kernels of at most `pairs` primer pairs
 * each (0, the default: one kernel for every pair).  Smaller kernels compile faster and in parallel
 * on the host's cores, which bounds the latency of a new primer set; one kernel for every pair
 * shares more work between patterns and scans fastest.  Plans always use one kernel.  Generated
 * kernels are cached process-wide, keyed by their source.  AH_EINVAL outside 0..256. */
ah_status ah_ctx_set_pairs_per_kernel(ah_ctx* ctx, int pairs);

/* Which scan kernel regular scans (ah_scan_primers) use; all find the same sites (Supplementary,
 * "Primer matching and clamp logic").
 *   0 (the default): kernels generated and compiled for the primer set (on first use, then cached
 *     process-wide).
 *   1: the generic kernel built into the library, which reads the primer set from a table and needs
 *     no compile, but scans several times slower.
 *   2: the generated kernels when they are compiled already.  Otherwise the generic kernel scans
 *     leading tiles while a host thread of the context compiles the generated kernels, which scan
 *     the rest once they are ready; a scan the generic kernel finishes first does not wait for the
 *     compile (the context joins that thread later, at the latest in ah_ctx_destroy).  Server
 *     contexts use this mode.
 *   3: the generic kernel over the first half of the tiles and the generated kernels over the rest
 *     (a fixed hand-over point, for tests).
 * Plans always use a generated kernel.  AH_EINVAL for another mode. */
ah_status ah_ctx_set_generic_scan(ah_ctx* ctx, int mode);

/* Which kernel computes the degenerate-site Tm of the default reading (every concrete variant
 * counts; Section "Primer degeneracy"); all give the same maximum within 1e-9 degC.
 *   0 (the default): a kernel generated for the primer set: each primer's chain of variants as
 *     straight-line code over the transitions that exist (compiled with NVRTC on first use, then
 *     cached process-wide).  Sets of more than 16 pairs, or whose distinct primers hold more than 96
 *     transitions between adjacent degenerate positions (their compile time), take the built-in
 *     kernel.
 *   1: the kernel built into the library, which walks any primer's chain from position masks.
 *   2: the generated kernel when it is compiled already, else the built-in kernel while a host
 *     thread of the context compiles it (server contexts use this mode).
 * Plans use the generated kernel unless the mode is 1.  AH_EINVAL for another mode. */
ah_status ah_ctx_set_tm_kernel(ah_ctx* ctx, int mode);
/* Site capacity from which the generated Tm kernel is launched once per group of primers (at most
 * 4 launches), so that each launch runs fewer primers' straight-line code and it stays in the
 * instruction cache; each launch re-reads the site marks.  0 restores the default (4 Mi sites),
 * UINT64_MAX keeps one launch, 1 always splits.  Results do not depend on it.  A plan takes the
 * value set when it is created. */
ah_status ah_ctx_set_tm_split(ah_ctx* ctx, uint64_t sites);
/* Diagnostics (no device needed): generate the Tm kernel for n primers (IUPAC, 2..32 nt; index
 * 2 * pair + primer as in a primer set) and compile it with NVRTC for compute capability sm (e.g.
 * 103).  AH_OK if it compiles; AH_EJIT with the compiler's log in log (log_cap bytes, NUL-ended)
 * if not; AH_EINVAL for a bad argument or more than 64 primers. */
ah_status ah_tm_kernel_check(const char* const* primers, uint32_t n, int sm, char* log, uint64_t log_cap);

/* Time every scan launch with CUDA events on the context's stream (scan_ms).  Synchronises the
 * stream to collect the timings of plan replays still pending. */
ah_status ah_ctx_set_timing(ah_ctx* ctx, int enable);
/* Fault injection on the host (no GPU fault): the context's next n device allocations fail with
 * AH_ENOMEM, as when the device is out of memory.  The call that meets one fails cleanly and the
 * context stays usable. */
ah_status ah_ctx_inject_alloc_failures(ah_ctx* ctx, int n);

/* Shape of the scan kernel used by ah_scan_primers on this context (a tuning knob; results do not
 * depend on it): threads per CTA (32..1024, a multiple of 32), groups of 32 positions per thread
 * (1..16), initial site slots per tile (16..4096, a power of two), and how pattern positions are
 * aligned (0: funnel shifts on the ALU pipe, 1: pairs of integer multiply-adds on the FMA pipe,
 * 2: alternate).  AH_EINVAL outside those ranges. */
ah_status ah_ctx_set_scan_config(ah_ctx* ctx, int threads, int groups_per_thread, int slot_cap, int shift_mode);
/* The generated scan circuit of this context (tuning knobs, results do not depend on them):
 * min_blocks, the blocks per SM the kernel's register allocation must allow (0: no bound, else
 * 1..32); vote_windows, the windows per warp vote the split between the circuit's two phases is
 * drawn for (1..1048576; 1024 = 32 lanes x 32 positions on uniform random bases, larger values
 * give a longer first phase); emit_queue, 0 to emit candidate sites where they are found, 1 to
 * queue them per warp and emit them with the whole warp after its block (faster where sites are
 * dense).  A plan without autotuning takes them as set here; the autotuner starts from them.
 * AH_EINVAL outside those ranges. */
ah_status ah_ctx_set_scan_circuit(ah_ctx* ctx, int min_blocks, int vote_windows, int emit_queue);

/* ------------------------------------------------------------------------------------------ */
/* 1. packing                                                                                   */
/*
 * Device layout of a packed batch (Section "Implementations": FASTA is compressed into 2-bit
 * batches that store headers, lengths and packed bases; here headers stay on the host):
 *   - bases are grouped 32 to a group; group g holds bases [32g, 32g+32) of the batch;
 *   - planes[g] is a uint2 {lo, hi}: bit b of lo/hi is the low/high bit of the 2-bit code of
 *     base 32g+b, with codes A=0, C=1, T=2, G=3 (lo = ASCII bit 1, hi = ASCII bit 2 of ACGTacgt);
 *   - invalid[g] is a uint32: bit b set iff base 32g+b is not one of ACGTacgt (N, other IUPAC
 *     codes, padding); such bases are stored as code 0;
 *   - record r starts at group rec_group[r] (a multiple of 2, so every record starts 16-byte
 *     aligned) and has rec_len[r] bases; it occupies 2 * (rec_len[r] / 64 + 1) groups, so at
 *     least one padding base (invalid, code 0) follows every record, the empty record included;
 *   - the plane and invalid arrays extend at least 64 groups past the last record (code 0,
 *     invalid).
 */
typedef struct {
  uint32_t n_records;
  uint64_t n_bases;          /* sum of record lengths */
  uint64_t n_groups;         /* groups covered by records, padding included */
  const void* planes;        /* device uint2[n_groups + tail] */
  const uint32_t* invalid;   /* device uint32[n_groups + tail] */
  const uint64_t* rec_group; /* device uint64[n_records] */
  const uint32_t* rec_len;   /* device uint32[n_records] */
  const uint32_t* genome_id; /* device uint32[n_records] */
} ah_batch_view;

/* Pack host ASCII records.  seqs[i] points at lens[i] characters (no terminator needed);
 * genome_ids may be NULL (then record i has genome id i).  Characters other than ACGTacgt are
 * invalid bases.  Records are copied to the device by the copy engines in chunks of up to 256 Mi
 * bases (64 MB packed), one copy per run of records contiguous in host memory, on a second stream,
 * and each chunk is packed from device memory while the next one is in flight; page-locked host
 * memory (cudaHostAlloc, cudaHostRegister, pinned tensors) moves at the full host-link rate.
 * Records already in device memory are packed in place.  Synchronises the stream before
 * returning (the host buffers may be reused afterwards).  AH_EINVAL: n_rec == 0, a record longer
 * than 2^32-1 bases, or a NULL pointer with a nonzero length. */
ah_status ah_pack_batch(ah_ctx* ctx, uint32_t n_rec, const char* const* seqs, const uint64_t* lens,
                        const uint32_t* genome_ids, ah_batch** out);

/* FASTA input (Abstract: the pipeline packs FASTA into 2-bit batches).  `text` holds n_bytes of
 * FASTA, in host or device memory: each record is a header line starting with '>' and the sequence
 * lines up to the next header.  It is parsed on the device (host text is copied there first): line
 * breaks and '\r', ' ', '\t' in sequence lines are dropped, every other byte is a base (non-ACGT
 * bytes become invalid bases as in ah_pack_batch), bytes before the first header are ignored, and a
 * record may be empty.  Returns the packed batch (genome_ids as in ah_pack_batch, may be NULL) and,
 * if names_out is not NULL, the records' header lines (without '>' and a trailing '\r').
 * AH_EINVAL when no line starts with '>'.  Synchronises the stream. */
typedef struct ah_fasta ah_fasta;
ah_status ah_fasta_pack(ah_ctx* ctx, const char* text, uint64_t n_bytes, const uint32_t* genome_ids,
                        ah_batch** batch_out, ah_fasta** names_out);
/* The same into an existing batch (not a slice) whose records have the text's number and lengths
 * (AH_EINVAL otherwise), e.g. the batch of a plan: FASTA text in, packed bases where the plan reads
 * them. */
ah_status ah_fasta_pack_into(ah_ctx* ctx, const char* text, uint64_t n_bytes, ah_batch* batch, ah_fasta** names_out);
/* FASTQ input with qualities (future work the paper names: FASTQ input with quality
 * propagation).  Records are four lines: '@' and the name, the bases, a '+' line, the qualities (one
 * byte per base); '\r' is dropped and empty lines after the last record are ignored.  Parsed on the
 * device like ah_fasta_pack.  Returns the packed bases, the qualities (*quals_out, one byte per base
 * of every record, kept on the device for ah_extract_qualities) and optionally the names.
 * AH_EINVAL when the text is not such records or a record's qualities differ in length from its
 * bases.  Synchronises the stream. */
typedef struct ah_quals ah_quals;
ah_status ah_fastq_pack(ah_ctx* ctx, const char* text, uint64_t n_bytes, const uint32_t* genome_ids,
                        ah_batch** batch_out, ah_quals** quals_out, ah_fasta** names_out);
/* File front end (Abstract: FASTA files in): the whole file at `path` is read into page-locked host
 * memory by parallel reads, then parsed and packed as ah_fasta_pack / ah_fastq_pack do.  AH_EINVAL
 * when the file cannot be opened or read (the message names it), AH_ENOMEM when the page-locked
 * buffer cannot be had.  Synchronises. */
ah_status ah_fasta_pack_file(ah_ctx* ctx, const char* path, const uint32_t* genome_ids, ah_batch** batch_out,
                             ah_fasta** names_out);
ah_status ah_fastq_pack_file(ah_ctx* ctx, const char* path, const uint32_t* genome_ids, ah_batch** batch_out,
                             ah_quals** quals_out, ah_fasta** names_out);
uint32_t ah_quals_count(const ah_quals* q);
/* The record offsets (n + 1 entries; the last is the total) and, when out is not NULL, all
 * qualities back to back (cap >= the total, else AH_EOVERFLOW) into host memory. */
ah_status ah_quals_copy(const ah_quals* q, char* out, uint64_t cap, uint64_t* offsets_out);
void ah_quals_free(ah_quals* q);
uint32_t ah_fasta_count(const ah_fasta* f);
/* header line of record i (owned by f), NULL past the end */
const char* ah_fasta_name(const ah_fasta* f, uint32_t i);
/* All names back to back and their offsets (count + 1 entries; the last is the total); out = NULL
 * only fills the offsets.  AH_EOVERFLOW when cap is short. */
ah_status ah_fasta_names_copy(const ah_fasta* f, char* out, uint64_t cap, uint64_t* offsets_out);
void ah_fasta_free(ah_fasta* f);

/* Pack records that are already in device memory: d_seq holds all records back to back and
 * h_offsets (host, n_rec+1 entries) gives record r as d_seq[h_offsets[r], h_offsets[r+1]).
 * Asynchronous; d_seq must stay valid until the stream reaches this work. */
ah_status ah_pack_batch_device(ah_ctx* ctx, uint32_t n_rec, const uint8_t* d_seq, const uint64_t* h_offsets,
                               const uint32_t* genome_ids, ah_batch** out);

/* Streaming: lay out a batch for n_rec records of the given lengths (device memory allocated, nothing
 * packed), then pack consecutive record ranges into it with ah_batch_pack_range.  Synchronises. */
ah_status ah_batch_create(ah_ctx* ctx, uint32_t n_rec, const uint64_t* lens, const uint32_t* genome_ids, ah_batch** out);
/* Store and reload a packed batch (Section "Implementations": AHv2 keeps genomes as 2-bit batches
 * on disk and streams those).  ah_batch_export copies the bases out in the device layout: planes
 * (uint2[n_groups], 0.25 bytes per base; n_groups from ah_batch_view_get) and, sparsely, the
 * nonzero invalid words (group index and word; about 1 % of groups at 0.5 % N, plus padding).
 * *n_invalid: capacity in, count out; with NULL lists only the count.  AH_EOVERFLOW when the lists
 * are too short.  Synchronises.
 * ah_batch_import copies them into a batch laid out for the same record lengths (ah_batch_create),
 * clearing the other invalid words: 4x fewer bytes over the host link than ASCII.  Page-locked
 * buffers move at the full link rate.  AH_EINVAL for a group index past the batch.  Synchronises. */
ah_status ah_batch_export(const ah_batch* b, void* planes_out, uint64_t* n_invalid, uint64_t* inv_groups,
                          uint32_t* inv_words);
ah_status ah_batch_import(ah_ctx* ctx, ah_batch* b, const void* planes, uint64_t n_invalid, const uint64_t* inv_groups,
                          const uint32_t* inv_words);

/* Pack records [first, first + count) of b: d_seq holds them back to back, at any alignment, in
 * device memory (packed in place) or host memory (copied in chunks as ah_pack_batch does), and h_offsets
 * (host, count + 1 entries, starting at 0) delimits them; their lengths must match the layout.
 * Repacking a batch that a plan was created on refreshes the plan's input.  Synchronises (d_seq
 * may be released afterwards). */
ah_status ah_batch_pack_range(ah_ctx* ctx, ah_batch* b, uint32_t first, uint32_t count, const uint8_t* d_seq,
                              const uint64_t* h_offsets);
ah_status ah_batch_view_get(const ah_batch* b, ah_batch_view* out);
/* A view of records [first, first + count) of `db` that shares db's packed planes (no copy) and owns
 * only a record table rebased to the slice; record indices in results are relative to `first`.
 * Any context on db's device may create and use it; db must outlive it.  Synchronises. */
ah_status ah_batch_slice(ah_ctx* ctx, const ah_batch* db, uint32_t first, uint32_t count, ah_batch** out);
void ah_batch_free(ah_batch* b);

/* ------------------------------------------------------------------------------------------ */
/* primers                                                                                      */

/* n_pairs pairs of IUPAC primers (5'->3', any case) with a mismatch budget per pair and one 3'
 * clamp length.  AH_EINVAL: n_pairs == 0 or > 256, a character outside the 15 IUPAC codes, a
 * length outside [clamp+1, 32], k > 15 or k > length. */
ah_status ah_primers_create(ah_ctx* ctx, uint32_t n_pairs, const char* const* fwd, const char* const* rev,
                            const uint8_t* k, uint8_t clamp, ah_primers** out);
void ah_primers_free(ah_primers* p);

/* ------------------------------------------------------------------------------------------ */
/* 2. scan                                                                                      */

/* One binding site.  pattern = 4 * pair + orient, orient = 2 * strand + primer, where primer 0
 * is the forward primer, 1 the reverse primer, strand 0 means the primer as written matches the
 * top strand and strand 1 means its reverse complement does.  [pos, pos + length of the primer)
 * is the site on the top strand of record `record`; mism counts mismatched primer positions. */
typedef struct {
  uint32_t record;
  uint32_t pos;
  uint16_t pattern;
  uint8_t mism;
  uint8_t flags;  /* reserved, 0 */
} ah_hit;

/* Every site of every pattern: a window [pos, pos+L) inside its record with no invalid base,
 * at most k mismatches against the pattern's IUPAC sets, and all c clamp positions matching
 * (the primer's 3' end: the last c positions as written, the first c of its reverse complement).
 * Hits are ordered by (pair, record, pos, orient).  Synchronises the stream to size the output. */
ah_status ah_scan_primers(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out);

/* The same sites as ah_scan_primers, scanned in the plain form: one kernel launch per record and
 * per primer pair (each with that pair's four oriented patterns), as a baseline for the batched
 * forms.  Same output order and contents.  Synchronises the stream. */
ah_status ah_scan_primers_per_record(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, ah_hits** out);

ah_status ah_hits_count(const ah_hits* h, uint64_t* n);
/* Device view: hits in device memory (ah_hit[n]) and, per pair, the range of its hits
 * (uint64[n_pairs+1], device). */
ah_status ah_hits_device(const ah_hits* h, const ah_hit** d_hits, const uint64_t** d_pair_offsets);
/* Copy min(n, cap) hits to host memory; synchronises. */
ah_status ah_hits_copy(const ah_hits* h, ah_hit* host_out, uint64_t cap);
void ah_hits_free(ah_hits* h);

/* ------------------------------------------------------------------------------------------ */
/* 3. pairing                                                                                   */

#define AH_FR 1u
#define AH_RF 2u
#define AH_FF 4u
#define AH_RR 8u

/* Amplicon record.  [start, end) on the top strand; orient 0 FR, 1 RF, 2 FF, 3 RR.
 * tm is filled by ah_tm_filter (NaN before).  flags: bit0 the threshold decision (Tm defined and
 * >= min_tm), bit1 Tm within 1e-9 C of min_tm (the decision then rests on the last digits of an
 * FP64 value: a caller who needs it stable re-checks these), bit2 Tm undefined (a site with no
 * parameterised variant).  With the filter on, only amplicons with bit0 remain; with it off the
 * bits annotate every amplicon against min_tm (pass -infinity for no threshold). */
typedef struct {
  uint32_t hit_i, hit_j; /* indices into the hits: the + anchor site and the - site */
  uint32_t record;
  uint32_t start, end;
  uint16_t pair;
  uint8_t orient;
  uint8_t flags;
  double tm;
} ah_amplicon;

/* For each + site i of a pair (in site order), walk the following sites of the same record and
 * pair: a + site stops the walk; a - site j whose amplicon end_j - pos_i exceeds max_len stops
 * it; a - site with min_len <= length is paired.  Orientation (primer_i, primer_j): (F,R) FR,
 * (R,F) RF, (F,F) FF, (R,R) RR; only orientations in orient_mask are output (the walk is not
 * affected).  Amplicons are ordered by (hit_i, hit_j).  Synchronises the stream. */
ah_status ah_pair_amplicons(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h,
                            uint32_t min_len, uint32_t max_len, uint32_t orient_mask, ah_amplicons** out);

/* Allocation-free pairing (the paper has no counterpart; this exists for callers of the library).
 * Some callers cannot allocate device memory while they run this step: an application that has
 * handed all of the GPU's memory to its own pool before loading the library, or a latency-bound
 * loop that cannot accept a cudaMalloc and the synchronisation it brings.  This call does the same
 * pairing as ah_pair_amplicons on buffers the caller owns and allocates nothing:
 *   d_hits, n_hits      sites in ah_scan_primers order (device), e.g. from ah_hits_device();
 *   d_pair_offsets      per-pair site ranges, n_pairs + 1 entries (device);
 *   d_pattern_len       primer length per pattern id 4 * pair + orient (device, uint8);
 *   d_out, out_capacity amplicon records (device) and their capacity;
 *   *n_out              (host) number of amplicons found, also when they do not fit.
 * Returns AH_EINVAL when n_hits exceeds AH_PAIR_NOALLOC_MAX_SITES (1,048,576) or an argument is
 * missing, AH_EOVERFLOW (with *n_out set, nothing written) when the amplicons exceed out_capacity.
 * Scratch memory is one file-scope device array of about 12 MiB (partner counts, prefix sums and
 * block sums for up to AH_PAIR_NOALLOC_MAX_SITES sites).  CUDA loads the library's device code onto a
 * device lazily, and the array is allocated with it, on the first ah_ctx_create on that device or
 * the first call of this entry point there, whichever comes first; it then stays until the process
 * exits.  A caller that will hand the rest of the GPU's memory to its own pool must therefore make
 * one of those calls first (a call with n_hits = 0 only does this set-up), and make it before any
 * stream capture.  All calls share the array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  The call works on the current device
 * and enqueues on `cuda_stream`; it waits for the count pass, then returns with the emit pass
 * enqueued.  AH_ECUDA without enqueuing anything when an error from earlier work is pending on the
 * calling thread (left in place for its owner); AH_ECUDA after a failed launch, with the passes
 * before it still enqueued. */
#define AH_PAIR_NOALLOC_MAX_SITES (1u << 20)
ah_status ah_pair_amplicons_noalloc(void* cuda_stream, const ah_hit* d_hits, uint64_t n_hits,
                                    const uint64_t* d_pair_offsets, const uint8_t* d_pattern_len, uint32_t min_len,
                                    uint32_t max_len, uint32_t orient_mask, ah_amplicon* d_out,
                                    uint64_t out_capacity, uint64_t* n_out);

/* ------------------------------------------------------------------------------------------ */
/* 4. melting temperature                                                                       */

typedef struct {
  double Na, K, Tris, Mg, dNTPs; /* mM */
  double dnac1, dnac2;           /* nM, the two strand concentrations */
  int32_t saltcorr;              /* 0 none; 1-7 as in Biopython's salt_correction (7: Owczarzy et
                                    al. 2008, Mg2+ and dNTPs modelled directly); default 5 */
  int32_t filter;                /* nonzero: drop amplicons with Tm < min_tm or undefined Tm;
                                    zero: keep all, flags still report the decision */
  double min_tm;                 /* degrees C (flags bits 0 and 1 are taken against it) */
  int32_t variants;              /* degenerate primers: 0 every concrete variant (default);
                                    1 only variants matching the site within k and the clamp */
  int32_t selfcomp;              /* 1: self-complementary duplexes (symmetry term, C = dnac1) */
  int32_t nn_table;              /* Watson-Crick nearest-neighbour set, Biopython's Tm_NN numbering:
                                    0 or 3 DNA_NN3, Allawi & SantaLucia 1997 (the default);
                                    1 DNA_NN1, Breslauer et al. 1986; 2 DNA_NN2, Sugimoto et al.
                                    1996; 4 DNA_NN4, SantaLucia & Hicks 2004; 5 RNA_NN1, Freier et
                                    al. 1986; 8 R_DNA_NN1, Sugimoto et al. 1995 (the primer strand
                                    taken as the RNA).  6 and 7 (RNA_NN2, RNA_NN3) are not built:
                                    AH_EINVAL.  The mismatch tables are the default ones for every
                                    set, as in Tm_NN. */
} ah_tm_params;

/* Fill tm and flags of every amplicon (Section "Implementations": Biopython's Tm_NN in C; Section
 * "Primer degeneracy": Tm over the primer's variants).  The nearest-neighbour Tm (FP64) of each site
 * that some amplicon pairs (no other site needs one) is the maximum of Tm(variant, site) over every
 * concrete variant of its primer, or with
 * params->variants = 1 over those that match the site under the scan's rule (at most the pair's k
 * differing positions, none in the 3' clamp).  The amplicon's Tm is the lower of its two sites'.  With filter set, the amplicon list is compacted to
 * the kept ones (order preserved).  Synchronises the stream.  AH_ELIMIT when a site has more than
 * 2^20 qualifying variants and the exact chain method does not apply (salt methods 6 and 7, whose
 * corrections depend on each variant's G/C content, or a variant whose entropy sum could reach
 * zero); that site's Tm is then NaN. */
ah_status ah_tm_filter(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h, ah_amplicons* a,
                       const ah_tm_params* params);

/* Tm of n given duplexes (utility and test surface): seqs[i] (5'->3', ACGT) over cseqs[i] (the
 * opposite strand written 3'->5', same length 2..32).  Writes tm_out[i] (NaN if undefined).
 * Synchronises. */
ah_status ah_tm_duplexes(ah_ctx* ctx, uint32_t n, const char* const* seqs, const char* const* cseqs,
                         const ah_tm_params* params, double* tm_out);

/* Tm of n (possibly degenerate) primers at given sites: primers[i] in IUPAC codes (5'->3'), sites[i]
 * the genome bases under it in the primer's orientation (A, C, G, T; same length 2..32).  The
 * maximum over the primer's concrete variants with at most k[i] positions differing from the site
 * and none among its last clamp[i] positions, as ah_tm_filter computes per site: enumerated for at
 * most 64 such variants, otherwise exact by Dinkelbach iterations over a chain Viterbi whose states
 * count mismatches, falling back to enumeration (up to 2^20 variants) for salt methods 6 and 7.  k == NULL
 * or k[i] >= the primer length: no mismatch limit; otherwise k[i] <= 15.  clamp == NULL: no clamp;
 * clamp[i] <= length (params->variants is not read: k and clamp say which variants count).
 * tm_out[i] is NaN when no qualifying variant has a defined Tm.  Synchronises; AH_ELIMIT as for
 * ah_tm_filter. */
ah_status ah_tm_sites(ah_ctx* ctx, uint32_t n, const char* const* primers, const char* const* sites,
                      const uint8_t* k, const uint8_t* clamp, const ah_tm_params* params, double* tm_out);

/* ------------------------------------------------------------------------------------------ */
/* 5. sequences and barcodes                                                                    */

/* For every amplicon, five strings into one device byte arena: the amplicon (top strand for FR,
 * FF, RR; reverse complement for RF) or, with trim, the part between its two sites (empty when
 * they overlap); the forward barcode (fb_len bases upstream of the forward primer: left of site i
 * for FR/FF/RR, right of site j reverse-complemented for RF); the reverse barcode (rb_len bases:
 * right of site j, or left of site i reverse-complemented for RF); and the bases of site i and of
 * site j in their primers' 5'->3' orientation.  Barcodes are clipped at record ends.  Invalid
 * bases are written as 'N'.  Synchronises the stream to size the arena. */
ah_status ah_extract_barcodes(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_hits* h,
                              ah_amplicons* a, int trim, uint32_t fb_len, uint32_t rb_len);

/* FASTA output (Supplementary "Headers and outputs"), host code over host copies of the results
 * (ah_amplicons_copy, ah_amplicons_seq_copy): per amplicon a header line
 *   >{id}.source={source}.coordinates={start+1}-{end}.Tm={tm}.orientation={FR|RF|FF|RR}
 *    .fprimer={forward primer's site}.rprimer={reverse primer's site}[.fb={fb}.rb={rb}]
 * (one line, fields joined by '.') and the amplicon sequence on the next.  id is the record's header
 * line up to its first blank (record_names[record], e.g. from ah_fasta_name); .source= is omitted
 * when record_sources is NULL or its entry is; coordinates are 1-based and inclusive on the top
 * strand, primer sites included; Tm has two decimals, NA when undefined; for RF the forward
 * primer's site is site j; .fb/.rb only when barcodes is nonzero.  Writes the text to out when it
 * fits out_cap (AH_EOVERFLOW otherwise) and its length to *out_len; out = NULL only measures.
 * AH_EINVAL for a record index >= n_records. */
ah_status ah_amplicons_fasta(uint64_t n_amps, const ah_amplicon* amps, const char* arena, const uint64_t* field_off,
                             uint32_t n_records, const char* const* record_names, const char* const* record_sources,
                             int barcodes, char* out, uint64_t out_cap, uint64_t* out_len);
/* The same as FASTQ: '@' instead of '>', then after the sequence a '+' line and the qualities
 * (qual_arena: ah_amplicons_qual_copy's output, field 0 of each amplicon). */
ah_status ah_amplicons_fastq(uint64_t n_amps, const ah_amplicon* amps, const char* arena, const char* qual_arena,
                             const uint64_t* field_off, uint32_t n_records, const char* const* record_names,
                             const char* const* record_sources, int barcodes, char* out, uint64_t out_cap,
                             uint64_t* out_len);

/* Qualities of the amplicon sequences (field 0 of ah_extract_barcodes: the amplicon or its trimmed
 * interior), taken from the qualities q of batch b's records and reversed for RF as the bases are
 * (not complemented).  Run after ah_extract_barcodes on the same objects; AH_EINVAL when q does not
 * match b's records.  ah_amplicons_qual_copy copies them out in the layout of the sequence arena:
 * amplicon m's qualities at the offsets of its field 0, other bytes unspecified (cap >= the arena's
 * size). */
ah_status ah_extract_qualities(ah_ctx* ctx, const ah_quals* q, const ah_batch* b, const ah_primers* p,
                               const ah_hits* h, ah_amplicons* a);
ah_status ah_amplicons_qual_copy(const ah_amplicons* a, char* out, uint64_t cap);

ah_status ah_amplicons_count(const ah_amplicons* a, uint64_t* n);
ah_status ah_amplicons_copy(const ah_amplicons* a, ah_amplicon* host_out, uint64_t cap);
/* Bytes in the arena written by ah_extract_barcodes (0 before). */
ah_status ah_amplicons_arena_size(const ah_amplicons* a, uint64_t* bytes);
/* Copy the arena and the field offsets (uint64[5*n+1]: field f of amplicon m spans
 * [off[5m+f], off[5m+f+1])).  Synchronises. */
ah_status ah_amplicons_seq_copy(const ah_amplicons* a, char* arena_out, uint64_t arena_cap, uint64_t* offsets_out,
                                uint64_t offsets_cap);
void ah_amplicons_free(ah_amplicons* a);

/* ------------------------------------------------------------------------------------------ */
/* batched, graph-captured form                                                                 */
/*
 * A plan holds the whole path for one packed batch and one primer set as a CUDA graph: one launch
 * scans every record for every pair (optionally with persistent CTAs taking tiles from a device
 * counter), and the site compaction, pairing, Tm, filter and extraction that follow are sized on
 * the device, so a replay needs no host round trip.  The scan kernel's shape is chosen by an
 * autotuner that times candidate shapes on the batch.  Outputs live in fixed-capacity buffers
 * sized from one exact run at creation (plus 25 %); a run that exceeds a capacity is reported, and
 * ah_plan_run grows the buffers, re-captures and runs again.
 */
typedef struct ah_plan ah_plan;
typedef struct {
  uint32_t min_len, max_len, orient_mask; /* as ah_pair_amplicons */
  ah_tm_params tm;                        /* as ah_tm_filter */
  int32_t extract;                        /* nonzero: sequences, trimming and barcodes as ah_extract_barcodes */
  int32_t trim;
  uint32_t fb_len, rb_len;
  int32_t autotune;                       /* nonzero: choose the scan kernel shape by timing candidates */
  int32_t persistent;                     /* -1 autotuner decides, 0 one CTA per tile, 1 persistent CTAs */
  uint64_t hit_capacity, amp_capacity, arena_capacity; /* 0: sized from an exact run */
} ah_plan_params;
typedef struct {
  int32_t threads, groups_per_thread, shift_mode, persistent, grid;
  uint32_t slot_cap, max_tile_sites;
  uint64_t hit_capacity, amp_capacity, arena_capacity;
  uint64_t n_hits, n_amps, n_kept, arena_bytes; /* of the last checked run */
  double autotune_ms, best_scan_ms;
  int32_t min_blocks;   /* the scan kernel's register bound: blocks per SM it allows (0: none) */
  int32_t vote_windows; /* windows per warp vote the scan circuit's phase split was drawn for (1024:
                           uniform random bases; the autotuner also tries 4x that) */
  int32_t emit_queue;   /* 1: candidate sites queued per warp and emitted after its block */
} ah_plan_info;
/* Build: autotune, size every buffer from one exact run of the regular path, capture, then one
 * checked replay that grows whatever this batch overflowed (per-tile slot lists included).  The
 * batch and primers must outlive the plan.  Synchronises. */
ah_status ah_plan_create(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_plan_params* params,
                         ah_plan** out);
/* One graph launch of the whole step on the context's stream (asynchronous).  With timing on
 * (ah_ctx_set_timing), the scan node of each replay is bracketed by its own pair of CUDA events;
 * their elapsed times are added to the context's scan_ms when the stream is next synchronised by
 * ah_ctx_synchronize or ah_ctx_set_timing. */
ah_status ah_plan_launch(ah_plan* plan);
/* The step on genomes in host memory: every record of the plan's batch is packed again from
 * h_seq[h_offsets[r], h_offsets[r + 1]) (the lengths must be the batch's), the text crossing the link
 * in staged chunks as ah_batch_pack_range does, and each range of scan tiles whose bases (and the
 * group after them) have landed is scanned while the next chunk is copied; the rest of the step
 * follows the last chunk as one graph launch.  Results as after ah_plan_launch (ah_plan_check,
 * ah_plan_copy_results).  Returns with the work enqueued on the context's stream; h_seq must stay
 * valid until the stream is synchronised (page-locked memory is fastest).  The plan's batch is
 * overwritten. */
ah_status ah_plan_launch_host(ah_plan* plan, const uint8_t* h_seq, const uint64_t* h_offsets);
/* The step on genomes stored as 2-bit batches in host memory (the layout ah_batch_export writes for
 * the plan's batch: planes, n_invalid sparse invalid words at groups inv_groups; Abstract and Section
 * "Implementations": AHv2 streams 2-bit batches): the invalid words are written first, then the
 * planes cross the link in chunks of 256 Mi bases straight into the batch, and each range of scan
 * tiles whose groups (and the group after them) have landed is scanned while the next chunk is
 * copied; the rest of the step follows as one graph launch.  Results as after ah_plan_launch.
 * Returns with the work enqueued on the context's stream; the host arrays must stay valid until the
 * stream is synchronised (page-locked memory is fastest).  AH_EINVAL for a group past the batch or a
 * plan over a slice.  The plan's batch is overwritten. */
ah_status ah_plan_launch_packed(ah_plan* plan, const void* h_planes, uint64_t n_invalid, const uint64_t* inv_groups,
                                const uint32_t* inv_words);
/* The step on FASTA text (host or device memory; Abstract: the pipeline starts from FASTA files)
 * whose records have the plan's batch's number and lengths: the text is parsed on the device in
 * chunks as it lands (as ah_fasta_pack_into does), the record bases each chunk completes are
 * packed into the batch at once, and each range of scan tiles whose groups (and the group after
 * them) are packed is scanned while the next chunk crosses the link; the rest of the step follows
 * as one graph launch.  Results as after ah_plan_launch.  AH_EINVAL when the text's records differ
 * from the batch's (found after the last chunk; the results are then not valid).  Synchronises
 * the stream between chunks; the plan's batch is overwritten. */
ah_status ah_plan_launch_fasta(ah_plan* plan, const char* text, uint64_t n_bytes);
/* Synchronise and check the last run: AH_EOVERFLOW when a capacity was exceeded (sizes in the info). */
ah_status ah_plan_check(ah_plan* plan);
/* Launch and check, growing capacities and re-capturing on overflow. */
ah_status ah_plan_run(ah_plan* plan);
ah_status ah_plan_info_get(const ah_plan* plan, ah_plan_info* out);
/* Copy the last run's sites, amplicons (the kept ones when the Tm filter is on) and, with
 * extraction, the sequence arena and its 5n+1 field offsets straight from the plan's buffers into
 * caller memory (any host memory; page-locked is fastest).  Capacities are in elements (bytes for
 * the arena); a NULL buffer skips that output.  Checks the run like ah_plan_check first, then
 * AH_EOVERFLOW if a buffer is too small (ah_plan_info_get then gives the counts).  Synchronises. */
ah_status ah_plan_copy_results(ah_plan* plan, ah_hit* hits, uint64_t hits_cap, ah_amplicon* amps, uint64_t amps_cap,
                               char* arena, uint64_t arena_cap, uint64_t* field_off, uint64_t field_off_cap);
/* Copies of the last run's sites and (kept) amplicons, with sequences when extraction is on. */
ah_status ah_plan_results(ah_plan* plan, ah_hits** hits, ah_amplicons** amps);
void ah_plan_free(ah_plan* plan);

/* ------------------------------------------------------------------------------------------ */
/* serving: continuous batching over a device-resident database                                 */
/*
 * A server keeps one packed batch (the database) resident and runs requests on `n_slots` workers,
 * each with its own context, CUDA stream and host thread.  Requests wait in arrival order; the
 * oldest is admitted as soon as a worker is free and its estimated device memory fits under the
 * budget beside the requests already running (a request alone on the device is always admitted),
 * so requests that arrive while others run join as slots and memory free up and their kernels
 * overlap on the GPU.  Any queued request that fits is admitted, not only the oldest: a small
 * request does not wait behind a large one that waits for memory, and a request passed over 8
 * times is then waited for (no starvation).  A running request holds its estimate
 * (ah_server_request_bytes) against the budget, grown to the memory its context actually holds
 * after each stage.  A request runs the whole path on a slice of the database (no genome copy).
 * Each worker has a CUDA stream per priority class (up to three of the device's priorities); a
 * request runs at the priority of its scan work, bases x 4 x pairs (below 1e11, below 1e12,
 * above), so small requests are scheduled ahead of large ones running beside them.  By default
 * the scan of a primer set whose generated kernels are not compiled starts on the generic kernel
 * while they compile (ah_ctx_set_generic_scan mode 2); ah_server_set_scan_mode changes that.
 */
typedef struct ah_server ah_server;
typedef struct {
  uint32_t n_pairs;
  const char* const* fwd; /* copied at submission */
  const char* const* rev;
  const uint8_t* k;
  uint8_t clamp;
  uint32_t first_record, n_records; /* the genome subset: a contiguous range of database records */
  uint32_t min_len, max_len, orient_mask;
  ah_tm_params tm;
  int32_t extract, trim;
  uint32_t fb_len, rb_len;
} ah_request;
typedef struct {
  ah_status status;
  uint64_t n_hits, n_amps, arena_bytes, bases;
  ah_hit* hits;          /* host arrays owned by the result; record indices are database indices */
  ah_amplicon* amps;
  char* arena;           /* when extraction was requested */
  uint64_t* field_off;   /* 5 * n_amps + 1 */
  double t_submit, t_admit, t_done; /* seconds on the server's clock */
  char error[256];
  double t_stage[5];     /* when each stage ended: slice and primers, scan, pairing, Tm, sequences
                            and host copies (t_done) */
} ah_result;
/* memory_budget: device bytes requests may reserve (0: 60 % of the free memory now).  The database
 * must outlive the server. */
ah_status ah_server_create(const ah_batch* db, int n_slots, uint64_t memory_budget, ah_server** out);
/* Queue a request (copied); returns at once with a ticket.  AH_EINVAL on a bad record range. */
ah_status ah_server_submit(ah_server* s, const ah_request* r, uint64_t* ticket);
/* Block until the request is done; the result is the caller's (ah_result_free).  Returns the
 * request's status. */
ah_status ah_server_wait(ah_server* s, uint64_t ticket, ah_result** out);
/* Generic-scan mode (ah_ctx_set_generic_scan: 0, 1 or 2; default 2) of requests admitted from now
 * on.  Mode 1 serves without any run-time compilation.  AH_EINVAL for another mode. */
ah_status ah_server_set_scan_mode(ah_server* s, int mode);
ah_status ah_server_now(const ah_server* s, double* seconds);
/* Cancel a request: a queued one finishes at once, a running one at its next stage boundary; its
 * result (ah_server_wait) has status AH_ECANCELED.  AH_EINVAL for an unknown or collected ticket. */
ah_status ah_server_cancel(ah_server* s, uint64_t ticket);
/* Device bytes the server reserves for a request when admitting it (its estimate). */
ah_status ah_server_request_bytes(const ah_server* s, const ah_request* r, uint64_t* bytes);
/* The budget, the bytes reserved now and the most ever reserved at once (any may be NULL). */
ah_status ah_server_memory(const ah_server* s, uint64_t* budget, uint64_t* reserved, uint64_t* reserved_peak);
/* Fault injection on the host (no GPU fault): the next n admitted requests find their first
 * device allocation failing; each fails with AH_ENOMEM and the server goes on serving. */
ah_status ah_server_inject_alloc_failures(ah_server* s, int n);
void ah_result_free(ah_result* r);
/* Finish queued requests, stop the workers and release the server. */
void ah_server_destroy(ah_server* s);

#ifdef __cplusplus
}
#endif
#endif /* AH_H */
