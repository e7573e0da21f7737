// Serving loop over a device-resident genome database (continuous batching).
//
// The database is one packed batch kept in HBM.  A request brings a primer set, its parameters and
// a genome subset (a contiguous range of database records).  The server runs `n_slots` workers,
// each with its own context (CUDA stream) and host thread.  Requests queue in arrival order; one
// is admitted as soon as a worker is free and its device memory fits under the budget next to the
// requests already running, so requests of different sizes that arrive while others are on the
// GPU join as slots and memory free up, and their kernels overlap on the device.
// Each admitted request runs the whole path on a slice of the database (no copy of the genomes)
// and its results are copied to host memory owned by the request's result.
//
// Admission takes the oldest queued request that fits, so a small request is not held behind a
// large one that must wait for memory; a request that has been passed over kMaxBypass times is
// then waited for, so large requests are not starved.  A running request's reservation starts at
// its estimate and grows to the memory its context's pool actually holds, measured after each
// stage (sites, amplicons and sequences are only known then), so later admissions see real use.
//
// Each worker owns one CUDA stream per priority class.  A request runs on the stream of its class,
// chosen by its scan work (bases x 4 x pairs): the smaller the request, the higher the priority,
// so the blocks of a small request are scheduled ahead of those of large ones already running and
// its latency stays close to its own run time instead of growing with the load.
//
// A request whose primer set has no compiled scan kernels yet starts scanning with the generic
// kernel while a thread compiles the generated kernels; the rest of the scan uses them once they
// are ready (generic-scan mode 2).  A small request may finish before its compile does; its
// context joins that thread later, and requests with the same primers find the kernels cached.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>

#include "ah_internal.h"

namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Job {
  uint64_t ticket = 0;
  // owned copy of the request
  std::vector<std::string> fwd, rev;
  std::vector<uint8_t> k;
  ah_request req{};
  uint64_t est_bytes = 0;
  uint64_t reserved = 0;          // bytes held against the budget while it runs
  int bypassed = 0;               // later requests admitted ahead of it
  std::atomic<bool> cancel{false};
  int inject_enomem = 0;          // device allocations of this run that fail (fault injection)
  ah_result* result = nullptr;
  bool done = false;
};

// later requests that may be admitted ahead of a waiting one before it blocks the queue
constexpr int kMaxBypass = 8;

}  // namespace

struct ah_server {
  const ah_batch* db = nullptr;
  int device = 0;
  uint64_t budget = 0, reserved = 0;
  std::chrono::steady_clock::time_point t0;
  std::vector<ah_ctx*> ctxs;
  std::vector<std::vector<cudaStream_t>> streams;  // [slot][priority class], class 0 the highest
  std::atomic<int> scan_mode{2};                   // generic-scan mode of the requests' scans
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::unordered_map<uint64_t, Job*> jobs;
  uint64_t next_ticket = 1;
  bool stop = false;
  int running = 0;
  int inject_enomem = 0;          // admitted requests still to fail their first device allocation
  uint64_t reserved_peak = 0;
};

namespace ah {
namespace {

// device bytes a request needs beyond the database: tile slot lists, per-(pair, tile) counts and
// offsets for its slice, plus room for sites, amplicons and sequences
uint64_t estimate_bytes(const ah_server* s, const ah_request& r, int slot_cap, uint64_t tile_groups) {
  const ah_batch* db = s->db;
  const uint64_t g0 = db->h_rec_group[r.first_record];
  const uint64_t g1 = (uint64_t)r.first_record + r.n_records < db->n_records ? db->h_rec_group[r.first_record + r.n_records]
                                                                             : db->n_groups;
  const uint64_t tiles = (g1 - g0) / tile_groups + 1;
  return tiles * ((uint64_t)slot_cap * 8 + 8 + 12ull * r.n_pairs) + (64ull << 20);
}

// priority class of a request of `work` base-patterns: 0 below 1e11, 1 below 1e12, 2 above
// (capped by the classes the device offers)
int priority_class(double work, int n_classes) {
  const int c = work < 1e11 ? 0 : work < 1e12 ? 1 : 2;
  return std::min(c, n_classes - 1);
}

// index in the queue of the request to admit now, or -1: the oldest that fits beside the running
// ones (any request when nothing runs), but none past a request that has been passed over
// kMaxBypass times
long pick_job(const ah_server* s) {
  for (size_t q = 0; q < s->queue.size(); ++q) {
    const Job* j = s->queue[q];
    if (s->reserved == 0 || s->reserved + j->reserved <= s->budget) return (long)q;
    if (j->bypassed >= kMaxBypass) return -1;
  }
  return -1;
}

// grow a running request's reservation to what its context's pool holds now
void account(ah_server* s, Job* j, ah_ctx* ctx) {
  unsigned long long used = 0;   // the attribute is a 64-bit unsigned count
  if (cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(s->mu);
  if ((uint64_t)used > j->reserved) {
    s->reserved += (uint64_t)used - j->reserved;
    j->reserved = (uint64_t)used;
    s->reserved_peak = std::max(s->reserved_peak, s->reserved);
  }
}

void fill_error(ah_result* res, ah_status st, const char* msg) {
  res->status = st;
  snprintf(res->error, sizeof res->error, "%s", msg ? msg : "");
}

void run_job(ah_server* s, int slot, Job* j) {
  ah_ctx* ctx = s->ctxs[slot];
  ah_result* res = j->result;
  const ah_request& r = j->req;
  {
    const ah_batch* db = s->db;
    const uint64_t g0 = db->h_rec_group[r.first_record];
    const uint64_t g1 = (uint64_t)r.first_record + r.n_records < db->n_records
                            ? db->h_rec_group[r.first_record + r.n_records]
                            : db->n_groups;
    const double work = (double)(g1 - g0) * 32.0 * 4.0 * r.n_pairs;
    ctx->stream = s->streams[slot][priority_class(work, (int)s->streams[slot].size())];
    ctx->generic_scan = s->scan_mode.load();
    // the Tm kernel generated for a new primer set compiles in the background, like its scan
    // kernels, unless the request asked for built-in kernels only
    ctx->tm_kernel = ctx->generic_scan == 1 ? 1 : 2;
  }
  ah_batch* slice = nullptr;
  ah_primers* pr = nullptr;
  ah_hits* h = nullptr;
  ah_amplicons* a = nullptr;
  std::vector<const char*> f(r.n_pairs), rv(r.n_pairs);
  for (uint32_t i = 0; i < r.n_pairs; ++i) f[i] = j->fwd[i].c_str(), rv[i] = j->rev[i].c_str();
  // stage end times; a stage that synchronises the stream anyway is timed when it returns
  auto stage = [&](int i) { res->t_stage[i] = now_s(s->t0); };
  ctx->fail_allocs = j->inject_enomem;
  // between stages: a cancelled request stops, and its reservation follows its real use
  auto next = [&](ah_status st) {
    account(s, j, ctx);
    if (!st && j->cancel.load()) return fail(ctx, AH_ECANCELED, "request cancelled");
    return st;
  };
  ah_status st = j->cancel.load() ? fail(ctx, AH_ECANCELED, "request cancelled") : AH_OK;
  if (!st) st = ah_batch_slice(ctx, s->db, r.first_record, r.n_records, &slice);
  if (!st) st = ah_primers_create(ctx, r.n_pairs, f.data(), rv.data(), j->k.data(), r.clamp, &pr);
  stage(0);
  if (!st) st = next(ah_scan_primers(ctx, slice, pr, &h));
  stage(1);
  if (!st) st = next(ah_pair_amplicons(ctx, slice, pr, h, r.min_len, r.max_len, r.orient_mask, &a));
  stage(2);
  if (!st) st = next(ah_tm_filter(ctx, slice, pr, h, a, &r.tm));
  stage(3);
  if (!st && r.extract) st = next(ah_extract_barcodes(ctx, slice, pr, h, a, r.trim, r.fb_len, r.rb_len));
  ctx->fail_allocs = 0;
  if (!st) {
    res->n_hits = h->n;
    res->n_amps = a->n;
    res->bases = slice->n_bases;
    res->hits = (ah_hit*)malloc(std::max<uint64_t>(1, h->n) * sizeof(ah_hit));
    res->amps = (ah_amplicon*)malloc(std::max<uint64_t>(1, a->n) * sizeof(ah_amplicon));
    st = ah_hits_copy(h, res->hits, h->n);
    if (!st) st = ah_amplicons_copy(a, res->amps, a->n);
    if (!st && r.extract) {
      res->arena_bytes = a->arena_bytes;
      res->arena = (char*)malloc(std::max<uint64_t>(1, a->arena_bytes));
      res->field_off = (uint64_t*)malloc((5 * a->n + 1) * sizeof(uint64_t));
      st = ah_amplicons_seq_copy(a, res->arena, a->arena_bytes, res->field_off, 5 * a->n + 1);
    }
    // record indices relative to the database
    for (uint64_t i = 0; i < res->n_hits && !st; ++i) res->hits[i].record += r.first_record;
    for (uint64_t i = 0; i < res->n_amps && !st; ++i) res->amps[i].record += r.first_record;
  }
  if (st) fill_error(res, st, ah_last_error(ctx));
  ah_amplicons_free(a);
  ah_hits_free(h);
  ah_primers_free(pr);
  ah_batch_free(slice);
  cudaStreamSynchronize(ctx->stream);
}

void worker(ah_server* s, int slot) {
  cudaSetDevice(s->device);
  for (;;) {
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      long q = -1;
      s->cv_work.wait(lock, [&] {
        if (s->stop && s->queue.empty()) return true;
        // the oldest request whose memory fits next to the running ones (always one when the device
        // is otherwise idle, so an oversized request still runs alone)
        q = pick_job(s);
        return q >= 0;
      });
      if (q < 0) return;   // stopping, nothing queued
      j = s->queue[(size_t)q];
      for (long e = 0; e < q; ++e) s->queue[(size_t)e]->bypassed++;
      s->queue.erase(s->queue.begin() + q);
      s->reserved += j->reserved;
      s->reserved_peak = std::max(s->reserved_peak, s->reserved);
      s->running++;
      if (s->inject_enomem > 0) {
        s->inject_enomem--;
        j->inject_enomem = 1;
      }
      j->result->t_admit = now_s(s->t0);
    }
    s->cv_work.notify_all();
    run_job(s, slot, j);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      j->result->t_done = j->result->t_stage[4] = now_s(s->t0);
      s->reserved -= j->reserved;
      s->running--;
      j->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace
}  // namespace ah

using namespace ah;

extern "C" {

ah_status ah_server_create(const ah_batch* db, int n_slots, uint64_t memory_budget, ah_server** out) {
  if (!db || !out || n_slots < 1 || n_slots > 64) return AH_EINVAL;
  *out = nullptr;
  ah_server* s = new ah_server();
  s->db = db;
  s->device = db->ctx->device;
  s->t0 = std::chrono::steady_clock::now();
  cudaSetDevice(s->device);
  if (!memory_budget) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    memory_budget = (uint64_t)(free_b * 0.6);
  }
  s->budget = memory_budget;
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const int n_classes = std::max(1, std::min(3, least - greatest + 1));
  for (int i = 0; i < n_slots; ++i) {
    s->streams.emplace_back();
    for (int c = 0; c < n_classes; ++c) {
      // class 0 the greatest priority, the last class the least
      const int prio = n_classes == 1 ? least : greatest + (least - greatest) * c / (n_classes - 1);
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess) {
        ah_server_destroy(s);
        return AH_ECUDA;
      }
      s->streams.back().push_back(st);
    }
    ah_ctx* c = nullptr;
    ah_status st = ah_ctx_create(&c, s->device, s->streams.back().back());
    if (st) {
      ah_server_destroy(s);
      return st;
    }
    c->scan_cfg.slot_cap = 64;  // requests are sparse; dense tiles are re-run with room
    // a worker's pool keeps its freed memory (the default of ah_ctx_create): returning memory at a
    // synchronisation and mapping it again for the next large request would stall the other
    // workers' streams
    // a request's primer set is compiled as kernels of 4 pairs on parallel host threads: a cold
    // 32-pair set compiles in about the time of one 4-pair kernel instead of 8x longer
    c->scan_cfg.pairs_per_kernel = 4;
    s->ctxs.push_back(c);
    // the page-locked bounce buffers for result copies exist before the first request
    for (int b = 0; b < 2; ++b)
      if (cudaMallocHost(&c->bounce[b], kBounceBytes) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->bounce_ev[b], cudaEventDisableTiming) != cudaSuccess) {
        ah_server_destroy(s);
        return AH_ENOMEM;
      }
  }
  for (int i = 0; i < n_slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return AH_OK;
}

ah_status ah_server_submit(ah_server* s, const ah_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket || r->n_pairs == 0 || !r->fwd || !r->rev || !r->k) return AH_EINVAL;
  if (r->n_records == 0 || (uint64_t)r->first_record + r->n_records > s->db->n_records) return AH_EINVAL;
  Job* j = new Job();
  for (uint32_t i = 0; i < r->n_pairs; ++i) {
    if (!r->fwd[i] || !r->rev[i]) {
      delete j;
      return AH_EINVAL;
    }
    j->fwd.emplace_back(r->fwd[i]);
    j->rev.emplace_back(r->rev[i]);
    j->k.push_back(r->k[i]);
  }
  j->req = *r;
  j->req.fwd = j->req.rev = nullptr;
  j->req.k = nullptr;
  j->result = (ah_result*)calloc(1, sizeof(ah_result));
  j->est_bytes = estimate_bytes(s, *r, 64, (uint64_t)s->ctxs[0]->scan_cfg.threads * s->ctxs[0]->scan_cfg.groups_per_thread);
  j->reserved = j->est_bytes;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    j->ticket = s->next_ticket++;
    j->result->t_submit = now_s(s->t0);
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    *ticket = j->ticket;
  }
  s->cv_work.notify_all();
  return AH_OK;
}

ah_status ah_server_wait(ah_server* s, uint64_t ticket, ah_result** out) {
  if (!s || !out) return AH_EINVAL;
  *out = nullptr;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return AH_EINVAL;
  Job* j = it->second;
  s->cv_done.wait(lock, [&] { return j->done; });
  s->jobs.erase(it);
  *out = j->result;
  delete j;
  return (*out)->status;
}

ah_status ah_server_cancel(ah_server* s, uint64_t ticket) {
  if (!s) return AH_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return AH_EINVAL;
    Job* j = it->second;
    auto q = std::find(s->queue.begin(), s->queue.end(), j);
    if (q != s->queue.end()) {   // still queued: finished at once, never admitted
      s->queue.erase(q);
      fill_error(j->result, AH_ECANCELED, "request cancelled before admission");
      j->result->t_admit = j->result->t_done = now_s(s->t0);
      j->done = true;
    } else {
      j->cancel.store(true);     // running: stops at its next stage boundary
    }
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return AH_OK;
}

ah_status ah_server_inject_alloc_failures(ah_server* s, int n) {
  if (!s || n < 0) return AH_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  s->inject_enomem = n;
  return AH_OK;
}

ah_status ah_server_request_bytes(const ah_server* s, const ah_request* r, uint64_t* bytes) {
  if (!s || !r || !bytes || r->n_records == 0 || (uint64_t)r->first_record + r->n_records > s->db->n_records)
    return AH_EINVAL;
  *bytes = estimate_bytes(s, *r, 64, (uint64_t)s->ctxs[0]->scan_cfg.threads * s->ctxs[0]->scan_cfg.groups_per_thread);
  return AH_OK;
}

ah_status ah_server_memory(const ah_server* s, uint64_t* budget, uint64_t* reserved, uint64_t* reserved_peak) {
  if (!s) return AH_EINVAL;
  std::lock_guard<std::mutex> lock(const_cast<ah_server*>(s)->mu);
  if (budget) *budget = s->budget;
  if (reserved) *reserved = s->reserved;
  if (reserved_peak) *reserved_peak = s->reserved_peak;
  return AH_OK;
}

ah_status ah_server_set_scan_mode(ah_server* s, int mode) {
  if (!s || mode < 0 || mode > 2) return AH_EINVAL;
  s->scan_mode.store(mode);
  return AH_OK;
}

ah_status ah_server_now(const ah_server* s, double* seconds) {
  if (!s || !seconds) return AH_EINVAL;
  *seconds = now_s(s->t0);
  return AH_OK;
}

void ah_result_free(ah_result* r) {
  if (!r) return;
  free(r->hits);
  free(r->amps);
  free(r->arena);
  free(r->field_off);
  free(r);
}

void ah_server_destroy(ah_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->jobs) {
    ah_result_free(kv.second->result);
    delete kv.second;
  }
  for (ah_ctx* c : s->ctxs) ah_ctx_destroy(c);
  for (auto& v : s->streams)
    for (cudaStream_t st : v) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
