// Batched, graph-captured form of the whole path over one packed batch and one primer set.
//
// ah_plan_create picks the scan kernel's shape with an autotuner (timing candidate shapes, shift
// modes and the persistent form on the batch), sizes every output from one exact run of the
// step, allocates fixed-capacity buffers, and captures the step into a CUDA graph: memsets, the
// scan (one launch over all records and pairs), per-tile sort, prefix sums, site emission,
// pairing, FP64 Tm, the Tm filter and extraction, all sized on the device.  ah_plan_launch replays
// it as one graph launch.  Capacities are checked after a run (ah_plan_check); ah_plan_run grows
// them and re-captures when a different batch of the same size would not fit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "ah_internal.h"

struct ah_plan {
  ah_ctx* ctx = nullptr;
  const ah_batch* b = nullptr;
  const ah_primers* p = nullptr;
  ah_plan_params prm{};
  ah::ScanConfig cfg;
  ah::ScanKernel kern;
  int grid = 0;                 // persistent grid (0: one CTA per tile)
  uint64_t tile_groups = 0, n_tiles = 0, n_cells = 0;
  uint32_t slot_cap = 0;
  uint64_t hit_cap = 0, amp_cap = 0, arena_cap = 0;
  // device buffers
  uint64_t* slots = nullptr;
  uint32_t* tile_count = nullptr;
  uint32_t* tpc = nullptr;
  uint32_t* big = nullptr;      // n_tiles + 1: tiles with more than 256 keys (count first)
  uint64_t* tpc_off = nullptr;  // n_cells + 1; [n_cells] = sites found
  uint64_t* scratch = nullptr;  // prefix-sum block sums
  ah_hit* hits = nullptr;
  uint64_t* pair_off = nullptr;
  uint32_t* pcount = nullptr;
  uint64_t* poff = nullptr;     // hit_cap + 1; [hit_cap] = amplicons found
  ah_amplicon* amps = nullptr;
  double* hit_tm = nullptr;
  uint32_t* tm_defer = nullptr;  // hit_cap + 1: sites the Tm chain does not cover
  uint32_t* keep = nullptr;
  uint64_t* koff = nullptr;     // amp_cap + 1; [amp_cap] = amplicons kept
  ah_amplicon* kept = nullptr;
  uint64_t* elen = nullptr;
  uint64_t* ebase = nullptr;    // amp_cap + 1; [amp_cap] = arena bytes
  char* arena = nullptr;
  uint64_t* field_off = nullptr;
  uint32_t* ctr = nullptr;      // [0] fullest tile, [1] overflow bits, [2..3] persistent work counter
  uint64_t* h_out = nullptr;    // pinned: counters read back after a run
  alignas(8) unsigned char tm_run[ah::kTmRunBytes];
  ah::TmKernel tm_k;  // the degenerate-site Tm kernel generated for p (fn null: the built-in one)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // The scan node is bracketed by two event-record nodes.  Timed replays use a ring of executable
  // copies of the graph whose nodes record their own event pairs, so no executable graph is
  // updated between launches; a slot is reused only after its timing has been read.
  static constexpr int kRing = 16;
  cudaEvent_t scan_ev[2] = {nullptr, nullptr};
  cudaGraphNode_t scan_ev_node[2] = {nullptr, nullptr};
  cudaGraphExec_t ring[kRing] = {};
  cudaEvent_t ring_ev[kRing][2] = {};
  uint64_t ring_gen[kRing] = {};  // the context's drain generation when the slot was launched (+1)
  int ring_next = 0;
  uint64_t kernel_nodes = 0;    // kernels one replay launches
  ah_plan_info info{};
  // the step after the scan as a graph of its own, and a one-CTA-per-tile scan kernel, for runs
  // whose scan is launched range by range as the input lands (ah_plan_launch_host)
  cudaGraphExec_t post_exec = nullptr;
  uint64_t post_kernel_nodes = 0;
  ah::ScanKernel range_kern;
};

namespace ah {
namespace {

void free_buffers(ah_plan* pl) {
  ah_ctx* c = pl->ctx;
  for (void* q : {(void*)pl->slots, (void*)pl->tile_count, (void*)pl->tpc, (void*)pl->big, (void*)pl->tpc_off, (void*)pl->scratch,
                  (void*)pl->hits, (void*)pl->pair_off, (void*)pl->pcount, (void*)pl->poff, (void*)pl->amps,
                  (void*)pl->hit_tm, (void*)pl->tm_defer, (void*)pl->keep, (void*)pl->koff, (void*)pl->kept, (void*)pl->elen,
                  (void*)pl->ebase, (void*)pl->arena, (void*)pl->field_off, (void*)pl->ctr})
    dfree(c, q);
  pl->slots = nullptr, pl->tile_count = nullptr, pl->tpc = nullptr, pl->big = nullptr, pl->tpc_off = nullptr, pl->scratch = nullptr;
  pl->hits = nullptr, pl->pair_off = nullptr, pl->pcount = nullptr, pl->poff = nullptr, pl->amps = nullptr;
  pl->hit_tm = nullptr, pl->tm_defer = nullptr, pl->keep = nullptr, pl->koff = nullptr, pl->kept = nullptr, pl->elen = nullptr;
  pl->ebase = nullptr, pl->arena = nullptr, pl->field_off = nullptr, pl->ctr = nullptr;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->post_exec) cudaGraphExecDestroy(pl->post_exec);
  pl->post_exec = nullptr;
  for (auto& x : pl->ring)
    if (x) cudaGraphExecDestroy(x), x = nullptr;
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->exec = nullptr;
  pl->graph = nullptr;
}

ah_status alloc_buffers(ah_plan* pl) {
  ah_ctx* c = pl->ctx;
  ah_status st;
  const uint64_t scan_n = std::max({pl->n_cells, pl->hit_cap, pl->amp_cap});
  if ((st = dalloc(c, &pl->slots, pl->n_tiles * pl->slot_cap)) || (st = dalloc(c, &pl->tile_count, pl->n_tiles)) ||
      (st = dalloc(c, &pl->tpc, pl->n_cells)) || (st = dalloc(c, &pl->big, pl->n_tiles + 1)) || (st = dalloc(c, &pl->tpc_off, pl->n_cells + 1)) ||
      (st = dalloc(c, &pl->scratch, scan_scratch_elems(scan_n))) || (st = dalloc(c, &pl->hits, pl->hit_cap)) ||
      (st = dalloc(c, &pl->pair_off, pl->p->n_pairs + 1)) || (st = dalloc(c, &pl->pcount, pl->hit_cap)) ||
      (st = dalloc(c, &pl->poff, pl->hit_cap + 1)) || (st = dalloc(c, &pl->amps, pl->amp_cap)) ||
      (st = dalloc(c, &pl->hit_tm, pl->hit_cap)) || (st = dalloc(c, &pl->tm_defer, pl->hit_cap + 1)) ||
      (st = dalloc(c, &pl->keep, pl->amp_cap)) ||
      (st = dalloc(c, &pl->koff, pl->amp_cap + 1)) || (st = dalloc(c, &pl->kept, pl->amp_cap)) ||
      (st = dalloc(c, &pl->elen, pl->amp_cap)) || (st = dalloc(c, &pl->ebase, pl->amp_cap + 1)) ||
      (st = dalloc(c, &pl->arena, pl->arena_cap)) || (st = dalloc(c, &pl->field_off, 5 * pl->amp_cap + 1)) ||
      (st = dalloc(c, &pl->ctr, 4)))
    return st;
  return AH_OK;
}

// the step, enqueued on stream s (captured into the graph): the counters' reset, the scan, and
// everything after the scan
void enqueue_pre(ah_plan* pl, cudaStream_t s) {
  cudaMemsetAsync(pl->tile_count, 0, pl->n_tiles * sizeof(uint32_t), s);
  cudaMemsetAsync(pl->tpc, 0, pl->n_cells * sizeof(uint32_t), s);
  cudaMemsetAsync(pl->ctr, 0, 4 * sizeof(uint32_t), s);
}

void enqueue_post(ah_plan* pl, cudaStream_t s);

void enqueue_step(ah_plan* pl, cudaStream_t s) {
  enqueue_pre(pl, s);
  // external records become event-record nodes of the captured graph
  cudaEventRecordWithFlags(pl->scan_ev[0], s, cudaEventRecordExternal);
  launch_scan_kernel(s, pl->kern, pl->b, pl->slots, pl->tile_count, pl->slot_cap, pl->ctx->d_status,
                     (unsigned long long*)(pl->ctr + 2), pl->n_tiles, pl->grid);
  cudaEventRecordWithFlags(pl->scan_ev[1], s, cudaEventRecordExternal);
  enqueue_post(pl, s);
}

void enqueue_post(ah_plan* pl, cudaStream_t s) {
  const ah_batch* b = pl->b;
  const ah_primers* p = pl->p;
  const ah_plan_params& q = pl->prm;
  launch_tile_max(s, pl->tile_count, pl->n_tiles, pl->ctr + 0);
  launch_tile_sort(s, pl->slots, pl->tile_count, pl->slot_cap, pl->n_tiles, p->n_pairs, pl->tpc, pl->big,
                   pl->ctx->sm_count);
  exclusive_scan_u32_s(s, pl->tpc, pl->tpc_off, pl->n_cells, pl->scratch);
  launch_emit_hits(s, pl->slots, pl->tile_count, pl->slot_cap, pl->n_tiles, pl->tile_groups, pl->tpc_off, b, pl->hits,
                   nullptr, pl->hit_cap, pl->ctr + 1, pl->pair_off, p->n_pairs);
  const uint64_t* n_hits = pl->tpc_off + pl->n_cells;
  launch_pair_walk(s, false, pl->hits, pl->hit_cap, n_hits, pl->pair_off, p->d_plen, q.min_len, q.max_len,
                   q.orient_mask & 15u, pl->pcount, nullptr, nullptr, 0, nullptr);
  exclusive_scan_u32_s(s, pl->pcount, pl->poff, pl->hit_cap, pl->scratch);
  launch_pair_walk(s, true, pl->hits, pl->hit_cap, n_hits, pl->pair_off, p->d_plen, q.min_len, q.max_len,
                   q.orient_mask & 15u, nullptr, pl->poff, pl->amps, pl->amp_cap, pl->ctr + 1);
  const uint64_t* n_amps = pl->poff + pl->hit_cap;
  launch_tm(s, pl->tm_run, pl->hits, pl->hit_cap, n_hits, p, pl->ctx->d_status, b->planes, b->rec_group, pl->hit_tm,
            pl->amps, pl->amp_cap, n_amps, q.tm.filter, q.tm.min_tm, pl->keep, pl->tm_defer, pl->ctx->sm_count,
            pl->tm_k);
  const ah_amplicon* out = pl->amps;
  const uint64_t* n_out = n_amps;
  if (q.tm.filter) {
    exclusive_scan_u32_s(s, pl->keep, pl->koff, pl->amp_cap, pl->scratch);
    launch_compact_amps(s, pl->amps, pl->amp_cap, pl->keep, pl->koff, pl->kept);
    out = pl->kept;
    n_out = pl->koff + pl->amp_cap;
  }
  if (q.extract) {
    launch_extract(s, false, out, pl->amp_cap, n_out, pl->hits, b->planes, b->invalid, b->rec_group, b->rec_len,
                   p->d_plen, q.trim, q.fb_len, q.rb_len, pl->elen, nullptr, nullptr, 0, nullptr);
    exclusive_scan_u64_s(s, pl->elen, pl->ebase, pl->amp_cap, pl->scratch);
    launch_extract(s, true, out, pl->amp_cap, n_out, pl->hits, b->planes, b->invalid, b->rec_group, b->rec_len,
                   p->d_plen, q.trim, q.fb_len, q.rb_len, pl->ebase, pl->arena, pl->field_off, pl->arena_cap,
                   pl->ctr + 1);
  }
}

ah_status capture(ah_plan* pl) {
  ah_ctx* c = pl->ctx;
  cudaStream_t s = c->stream;
  AH_CUDA(c, cudaStreamSynchronize(s));
  ah_status dst = drain_timings(c);  // the ring's events are recorded afresh from here on
  if (dst) return dst;
  AH_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  enqueue_step(pl, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return fail(c, AH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  pl->graph = g;
  // count the kernels of one replay and find the two event-record nodes around the scan
  size_t n = 0;
  AH_CUDA(c, cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) AH_CUDA(c, cudaGraphGetNodes(g, nodes.data(), &n));
  pl->kernel_nodes = 0;
  pl->scan_ev_node[0] = pl->scan_ev_node[1] = nullptr;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    AH_CUDA(c, cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) pl->kernel_nodes++;
    if (t == cudaGraphNodeTypeEventRecord) {
      cudaEvent_t e = nullptr;
      AH_CUDA(c, cudaGraphEventRecordNodeGetEvent(nd, &e));
      for (int i = 0; i < 2; ++i)
        if (e == pl->scan_ev[i]) pl->scan_ev_node[i] = nd;
    }
  }
  if (!pl->scan_ev_node[0] || !pl->scan_ev_node[1]) return fail(c, AH_EINTERNAL, "plan: scan timing nodes not captured");
  AH_CUDA(c, cudaGraphInstantiate(&pl->exec, g, 0));
  // the timing ring: the same graph with each slot's events in the two record nodes
  for (int i = 0; i < ah_plan::kRing; ++i) {
    for (int k = 0; k < 2; ++k) {
      if (!pl->ring_ev[i][k]) AH_CUDA(c, cudaEventCreate(&pl->ring_ev[i][k]));
      AH_CUDA(c, cudaGraphEventRecordNodeSetEvent(pl->scan_ev_node[k], pl->ring_ev[i][k]));
    }
    AH_CUDA(c, cudaGraphInstantiate(&pl->ring[i], g, 0));
    pl->ring_gen[i] = 0;
  }
  for (int k = 0; k < 2; ++k) AH_CUDA(c, cudaGraphEventRecordNodeSetEvent(pl->scan_ev_node[k], pl->scan_ev[k]));
  return AH_OK;
}

// time the scan kernel of one shape through the regular path (ms per launch, on this batch)
ah_status time_shape(ah_ctx* c, const ah_batch* b, const ah_primers* p, const ScanConfig& cfg, int reps, double* ms,
                     uint64_t* n_hits) {
  const ScanConfig saved = c->scan_cfg;
  const bool timing = c->timing;
  c->scan_cfg = cfg;
  ah_status st = ah_ctx_set_timing(c, 1);
  ah_hits* h = nullptr;
  if (!st) st = scan_primers(c, b, p, &h);  // compiles and warms
  if (h) {
    *n_hits = h->n;
    ah_hits_free(h);
  }
  const double ms0 = c->scan_ms;
  const uint64_t l0 = c->n_scan_launches;
  for (int r = 0; r < reps && !st; ++r) {
    h = nullptr;
    st = scan_primers(c, b, p, &h);
    ah_hits_free(h);
  }
  if (!st) *ms = (c->scan_ms - ms0) / std::max<uint64_t>(1, c->n_scan_launches - l0);
  c->scan_cfg = saved;
  c->timing = timing;
  return st;
}

// After an overflowing run: enlarge the per-tile slot lists and every capacity that overflowed (with
// `all` false, only those the plan sized itself), free the buffers and capture again.  AH_OK with
// nothing changed when only caller-given capacities overflowed.
ah_status grow(ah_plan* pl, bool all) {
  const ah_plan_info& i = pl->info;
  const ah_plan_params& q = pl->prm;
  bool changed = false;
  if (i.max_tile_sites > pl->slot_cap) {
    uint32_t need = 1;
    while (need < i.max_tile_sites) need <<= 1;
    if (need > 4096) return fail(pl->ctx, AH_EOVERFLOW, "plan: a tile holds more than 4096 sites");
    pl->slot_cap = need;
    changed = true;
  }
  auto enlarge = [&](uint64_t& cap, uint64_t used, uint64_t given, uint64_t slack) {
    if (used > cap && (all || !given)) cap = std::max(cap, used + used / 4 + slack), changed = true;
  };
  enlarge(pl->hit_cap, i.n_hits, q.hit_capacity, 1024);
  enlarge(pl->amp_cap, i.n_amps, q.amp_capacity, 1024);
  if (q.extract) enlarge(pl->arena_cap, i.arena_bytes, q.arena_capacity, 4096);
  if (!changed) return AH_OK;
  free_buffers(pl);
  ah_status st;
  if ((st = alloc_buffers(pl)) || (st = capture(pl))) return st;
  return AH_OK;
}

}  // namespace
}  // namespace ah

using namespace ah;

extern "C" {

ah_status ah_plan_create(ah_ctx* ctx, const ah_batch* b, const ah_primers* p, const ah_plan_params* prm,
                         ah_plan** out) {
  if (!ctx || !b || !p || !prm || !out) return fail(ctx, AH_EINVAL, "ah_plan_create: NULL argument");
  if (prm->min_len > prm->max_len) return fail(ctx, AH_EINVAL, "ah_plan_create: min_len > max_len");
  if (prm->tm.saltcorr < 0 || prm->tm.saltcorr > 7) return fail(ctx, AH_EINVAL, "ah_plan_create: bad salt method");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  ah_plan* pl = new ah_plan();
  pl->ctx = ctx;
  pl->b = b;
  pl->p = p;
  pl->prm = *prm;
  pl->cfg = ctx->scan_cfg;
  pl->cfg.pairs_per_kernel = 0;  // a plan captures one scan kernel over every pair
  ah_status st = tm_prepare(ctx, &prm->tm, pl->tm_run, sizeof pl->tm_run);
  if (!st && !prm->tm.variants) st = tm_kernel_for(ctx, p, true, tm_run_slot(pl->tm_run), &pl->tm_k);
  for (int i = 0; i < 2 && !st; ++i)
    if (cudaEventCreate(&pl->scan_ev[i]) != cudaSuccess) st = fail(ctx, AH_ECUDA, "ah_plan_create: event creation failed");
  const auto t0 = std::chrono::steady_clock::now();
  uint64_t n_hits = 0;
  if (!st && prm->autotune) {
    // candidate shapes x alignment modes, then the persistent form of the best; a candidate replaces
    // the incumbent only when it is at least 3 % faster, so near-equal shapes do not flip between runs
    const int shapes[][2] = {{256, 8}, {128, 8}, {256, 4}, {128, 4}};
    double best = 1e30;
    ScanConfig win = pl->cfg;
    for (int mode = 0; mode < 2 && !st; ++mode) {
      for (auto& sh : shapes) {
        ScanConfig c = pl->cfg;
        c.threads = sh[0];
        c.groups_per_thread = sh[1];
        c.shift_mode = mode;
        c.persistent = 0;
        double ms = 0;
        if ((st = time_shape(ctx, b, p, c, 2, &ms, &n_hits))) break;
        if (ms < best * 0.97) best = ms, win = c;
      }
    }
    // a large circuit (the 8-pair batched set: 166 registers, 3 blocks of 128 threads per SM) may
    // run faster with registers bounded for 4 blocks: more warps, a few spills to L1
    if (!st && win.threads == 128 && ctx->scan_ops_per_group > 400) {
      ScanConfig c = win;
      c.min_blocks = 4;
      double ms = 0;
      if (!(st = time_shape(ctx, b, p, c, 2, &ms, &n_hits)) && ms < best * 0.97) best = ms, win = c;
    }
    // the phase split: the circuit drawn for windows surviving phase one four times as often as on
    // uniform random bases (a longer phase one) pays off on sequence whose composition lets more
    // windows through; a 1.5 % margin, the measured difference being a few percent
    if (!st) {
      ScanConfig c = win;
      c.vote_windows = 4 * win.vote_windows;
      double ms = 0;
      if (!(st = time_shape(ctx, b, p, c, 2, &ms, &n_hits)) && ms < best * 0.985) best = ms, win = c;
    }
    // candidates queued per warp and emitted by the whole warp after its block: pays where sites are
    // dense (tandem repeats: the dense workload's scan went from 8.6 to 6.2 ms), costs a little
    // elsewhere (registers and shared memory)
    if (!st) {
      ScanConfig c = win;
      c.emit_queue = 1;
      double ms = 0;
      if (!(st = time_shape(ctx, b, p, c, 2, &ms, &n_hits)) && ms < best * 0.97) best = ms, win = c;
    }
    if (!st && prm->persistent != 0) {
      ScanConfig c = win;
      c.persistent = 1;
      double ms = 0;
      if (!(st = time_shape(ctx, b, p, c, 2, &ms, &n_hits)) && (ms < best * 0.97 || prm->persistent > 0))
        best = ms, win = c;
    }
    pl->cfg = win;
    pl->info.best_scan_ms = best;
  } else if (prm->persistent > 0) {
    pl->cfg.persistent = 1;
  }
  pl->info.autotune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  // one exact run of the regular path sizes every buffer
  ah_hits* h = nullptr;
  ah_amplicons* a = nullptr;
  const ScanConfig saved = ctx->scan_cfg;
  ctx->scan_cfg = pl->cfg;
  if (!st) st = scan_primers(ctx, b, p, &h);
  if (!st) st = pair_amplicons(ctx, b, p, h, prm->min_len, prm->max_len, prm->orient_mask & 15u, &a);
  const uint64_t n_amps_all = a ? a->n : 0;
  if (!st) st = tm_filter(ctx, b, p, h, a, &prm->tm);
  if (!st && prm->extract) st = extract(ctx, b, p, h, a, prm->trim, prm->fb_len, prm->rb_len);
  ctx->scan_cfg = saved;
  if (!st) {
    auto grow = [](uint64_t x) { return x + x / 4 + 1024; };
    pl->hit_cap = prm->hit_capacity ? prm->hit_capacity : grow(h->n);
    pl->amp_cap = prm->amp_capacity ? prm->amp_capacity : grow(n_amps_all);
    pl->arena_cap = prm->arena_capacity ? prm->arena_capacity : grow(a->arena_bytes);
  }
  ah_hits_free(h);
  ah_amplicons_free(a);
  if (!st) st = ctx->jit->get(ctx, p->pats, pl->cfg, &pl->kern);
  if (!st) {
    pl->tile_groups = (uint64_t)pl->cfg.threads * pl->cfg.groups_per_thread;
    pl->n_tiles = std::max<uint64_t>(1, (b->n_groups + pl->tile_groups - 1) / pl->tile_groups);
    pl->n_cells = (uint64_t)p->n_pairs * pl->n_tiles;
    pl->slot_cap = (uint32_t)pl->cfg.slot_cap;
    if (pl->n_tiles > 0x7fffffffull) st = fail(ctx, AH_EINVAL, "ah_plan_create: batch too large for one launch");
  }
  if (!st && pl->cfg.persistent) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)pl->kern.fn, pl->cfg.threads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    pl->grid = (int)std::min<uint64_t>(pl->n_tiles, (uint64_t)per_sm * ctx->sm_count);
  }
  if (!st && cudaMallocHost(&pl->h_out, 8 * sizeof(uint64_t)) != cudaSuccess)
    st = fail(ctx, AH_ENOMEM, "ah_plan_create: pinned allocation failed");
  if (!st) st = alloc_buffers(pl);
  if (!st) st = capture(pl);
  // checked replays: the per-tile slot lists (sized from the context's default) and the capacities
  // the plan sized itself grow here if this batch needs more, so later replays fit unchecked;
  // capacities the caller fixed are left as given (ah_plan_check reports them)
  for (int attempt = 0; attempt < 4 && !st; ++attempt) {
    if ((st = ah_plan_launch(pl))) break;
    const ah_status cs = ah_plan_check(pl);
    if (cs != AH_EOVERFLOW) {
      st = cs;
      break;
    }
    const uint32_t slots = pl->slot_cap;
    const uint64_t caps = pl->hit_cap + pl->amp_cap + pl->arena_cap;
    if ((st = grow(pl, false))) break;  // e.g. a tile with more than 4096 sites
    if (pl->slot_cap == slots && pl->hit_cap + pl->amp_cap + pl->arena_cap == caps) break;  // only fixed ones
  }
  if (st) {
    ah_plan_free(pl);
    return st;
  }
  pl->info.threads = pl->cfg.threads;
  pl->info.groups_per_thread = pl->cfg.groups_per_thread;
  pl->info.shift_mode = pl->cfg.shift_mode;
  pl->info.persistent = pl->cfg.persistent;
  pl->info.min_blocks = pl->cfg.min_blocks;
  pl->info.vote_windows = pl->cfg.vote_windows;
  pl->info.emit_queue = pl->cfg.emit_queue;
  pl->info.grid = pl->grid ? pl->grid : (int32_t)pl->n_tiles;
  *out = pl;
  return AH_OK;
}

ah_status ah_plan_launch(ah_plan* pl) {
  if (!pl) return AH_EINVAL;
  ah_ctx* c = pl->ctx;
  cudaGraphExec_t x = pl->exec;
  if (c->timing) {
    // the next ring slot; if its previous replay's timing is still unread, read it first
    const int i = pl->ring_next;
    pl->ring_next = (i + 1) % ah_plan::kRing;
    if (pl->ring_gen[i] == c->drain_gen + 1) {
      ah_status st = drain_timings(c);
      if (st) return st;
    }
    x = pl->ring[i];
    pl->ring_gen[i] = c->drain_gen + 1;
    c->ev_pending.emplace_back(pl->ring_ev[i][0], pl->ring_ev[i][1]);
    c->n_scan_launches++;
    c->scan_bases += pl->b->n_bases;
  }
  AH_CUDA(c, cudaGraphLaunch(x, c->stream));
  c->n_launches += pl->kernel_nodes;
  c->scan_ops_per_group = pl->kern.alu_ops_per_group;
  return AH_OK;
}

namespace {

// the post-scan graph, captured on first use after the plan's buffers last changed
ah_status ensure_post(ah_plan* pl) {
  if (pl->post_exec) return AH_OK;
  ah_ctx* c = pl->ctx;
  cudaStream_t s = c->stream;
  AH_CUDA(c, cudaStreamSynchronize(s));
  AH_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  enqueue_post(pl, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return fail(c, AH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) cudaGraphGetNodes(g, nodes.data(), &n);
  pl->post_kernel_nodes = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) pl->post_kernel_nodes++;
  }
  e = cudaGraphInstantiate(&pl->post_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, AH_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  return AH_OK;
}

}  // namespace

ah_status ah_plan_launch_host(ah_plan* pl, const uint8_t* h_seq, const uint64_t* h_offsets) {
  if (!pl || !h_seq || !h_offsets) return AH_EINVAL;
  ah_ctx* c = pl->ctx;
  cudaSetDevice(c->device);
  ah_status st;
  if (!pl->range_kern.fn) {
    if (pl->cfg.persistent) {
      ScanConfig cfg = pl->cfg;
      cfg.persistent = 0;
      if ((st = c->jit->get(c, pl->p->pats, cfg, &pl->range_kern))) return st;
    } else {
      pl->range_kern = pl->kern;
    }
  }
  if ((st = ensure_post(pl))) return st;
  ah_batch* b = const_cast<ah_batch*>(pl->b);
  enqueue_pre(pl, c->stream);
  // tiles whose groups and the group after them are packed are scanned at once, while the next
  // chunk crosses the link
  const uint64_t tg = (uint64_t)pl->range_kern.threads * pl->range_kern.groups_per_thread;
  uint64_t scanned = 0;
  uint64_t scan_launches = 0;
  auto on_chunk = [&](uint64_t done) {
    const uint64_t upto = done >= b->n_groups ? b->n_groups : (done > 0 ? (done - 1) / tg * tg : 0);
    if (upto > scanned) {
      launch_scan_range(c->stream, pl->range_kern, b, pl->slots, pl->tile_count, pl->slot_cap, c->d_status, scanned,
                        upto);
      scanned = upto;
      ++scan_launches;
    }
  };
  if ((st = pack_host_staged(c, b, h_seq, h_offsets, on_chunk))) return st;
  on_chunk(b->n_groups);
  AH_CUDA(c, cudaGetLastError());
  AH_CUDA(c, cudaGraphLaunch(pl->post_exec, c->stream));
  c->n_launches += pl->post_kernel_nodes + scan_launches;
  c->scan_ops_per_group = pl->range_kern.alu_ops_per_group;
  return AH_OK;
}

ah_status ah_plan_launch_packed(ah_plan* pl, const void* h_planes, uint64_t n_invalid, const uint64_t* inv_groups,
                               const uint32_t* inv_words) {
  if (!pl || !h_planes || (n_invalid && (!inv_groups || !inv_words))) return AH_EINVAL;
  ah_ctx* c = pl->ctx;
  ah_batch* b = const_cast<ah_batch*>(pl->b);
  if (b->view) return fail(c, AH_EINVAL, "ah_plan_launch_packed: the plan's batch is a slice of another batch");
  for (uint64_t i = 0; i < n_invalid; ++i)
    if (inv_groups[i] >= b->n_groups)
      return fail(c, AH_EINVAL, "ah_plan_launch_packed: invalid word %llu at group %llu, past the batch's %llu groups",
                  (unsigned long long)i, (unsigned long long)inv_groups[i], (unsigned long long)b->n_groups);
  cudaSetDevice(c->device);
  ah_status st;
  if (!pl->range_kern.fn) {
    if (pl->cfg.persistent) {
      ScanConfig cfg = pl->cfg;
      cfg.persistent = 0;
      if ((st = c->jit->get(c, pl->p->pats, cfg, &pl->range_kern))) return st;
    } else {
      pl->range_kern = pl->kern;
    }
  }
  if ((st = ensure_post(pl))) return st;
  enqueue_pre(pl, c->stream);
  // the invalid words first (a small list), then the planes in chunks of kChunkBases bases on a
  // copy stream straight into the batch; each range of scan tiles whose groups (and the group after
  // them) have landed is scanned while the next chunk crosses the link
  const uint64_t chunk = kChunkBases / kGroupBases;  // groups per copy (64 MiB of planes)
  const uint64_t n_chunks = (b->n_groups + chunk - 1) / chunk;
  cudaStream_t cs = nullptr;
  cudaEvent_t ready = nullptr;
  std::vector<cudaEvent_t> landed(n_chunks, nullptr);
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  for (uint64_t k = 0; k < n_chunks && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&landed[k], cudaEventDisableTiming);
  // the sparse list crosses the link first (the planes' chunks would queue it behind them on the copy
  // engine); the plane copies wait for earlier work that may still read the planes, and the invalid
  // words are written by kernels meanwhile (only the scans read them)
  InvalidList il;
  if (e == cudaSuccess && (st = upload_invalid_list(c, n_invalid, inv_groups, inv_words, &il))) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaEventRecord(ready, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
  if (e == cudaSuccess && (st = scatter_invalid_list(c, b, &il))) e = cudaErrorUnknown;
  const uint64_t tg = (uint64_t)pl->range_kern.threads * pl->range_kern.groups_per_thread;
  uint64_t scanned = 0, scan_launches = 0;
  for (uint64_t k = 0; k < n_chunks && e == cudaSuccess; ++k) {
    const uint64_t g0 = k * chunk, g1 = std::min(b->n_groups, g0 + chunk);
    e = cudaMemcpyAsync(b->planes + g0, (const uint2*)h_planes + g0, (g1 - g0) * sizeof(uint2), cudaMemcpyHostToDevice,
                        cs);
    if (e == cudaSuccess) e = cudaEventRecord(landed[k], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, landed[k], 0);
    const uint64_t upto = g1 >= b->n_groups ? b->n_groups : (g1 - 1) / tg * tg;
    if (e == cudaSuccess && upto > scanned) {
      launch_scan_range(c->stream, pl->range_kern, b, pl->slots, pl->tile_count, pl->slot_cap, c->d_status, scanned,
                        upto);
      scanned = upto;
      ++scan_launches;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaGraphLaunch(pl->post_exec, c->stream);
  if (il.groups) dfree(c, il.groups);  // a list left over when a step before its scatter failed
  if (il.words) dfree(c, il.words);
  // the stream and events are released once their work is done
  for (cudaEvent_t x : landed)
    if (x) cudaEventDestroy(x);
  if (ready) cudaEventDestroy(ready);
  if (cs) cudaStreamDestroy(cs);
  if (st) return st;
  if (e != cudaSuccess) return fail(c, AH_ECUDA, "ah_plan_launch_packed: %s", cudaGetErrorString(e));
  c->n_launches += pl->post_kernel_nodes + scan_launches;
  c->scan_ops_per_group = pl->range_kern.alu_ops_per_group;
  return AH_OK;
}

ah_status ah_plan_launch_fasta(ah_plan* pl, const char* text, uint64_t n_bytes) {
  if (!pl || !text || n_bytes == 0) return AH_EINVAL;
  ah_ctx* c = pl->ctx;
  ah_batch* b = const_cast<ah_batch*>(pl->b);
  if (b->view) return fail(c, AH_EINVAL, "ah_plan_launch_fasta: the plan's batch is a slice of another batch");
  cudaSetDevice(c->device);
  ah_status st;
  if (!pl->range_kern.fn) {
    if (pl->cfg.persistent) {
      ScanConfig cfg = pl->cfg;
      cfg.persistent = 0;
      if ((st = c->jit->get(c, pl->p->pats, cfg, &pl->range_kern))) return st;
    } else {
      pl->range_kern = pl->kern;
    }
  }
  if ((st = ensure_post(pl))) return st;
  enqueue_pre(pl, c->stream);
  // the records laid end to end as the parser compacts them
  std::vector<uint64_t> start(b->n_records + 1, 0);
  for (uint32_t r = 0; r < b->n_records; ++r) start[r + 1] = start[r] + b->h_rec_len[r];
  ConcatCursor cur;
  const uint64_t tg = (uint64_t)pl->range_kern.threads * pl->range_kern.groups_per_thread;
  uint64_t scanned = 0, scan_launches = 0;
  // after each chunk: pack the record bases it completed, then scan the tiles whose groups (and the
  // group after them) are packed, while the next chunk of text crosses the link
  const FastaChunkHook hook = [&](const uint8_t* d_concat, uint64_t avail, bool last) -> ah_status {
    uint64_t done = 0;
    ah_status s = pack_concat_upto(c, b, d_concat, start.data(), last ? start[b->n_records] : avail, &cur, &done);
    if (s) return s;
    const uint64_t upto = done >= b->n_groups ? b->n_groups : (done > 0 ? (done - 1) / tg * tg : 0);
    if (upto > scanned) {
      launch_scan_range(c->stream, pl->range_kern, b, pl->slots, pl->tile_count, pl->slot_cap, c->d_status, scanned,
                        upto);
      scanned = upto;
      ++scan_launches;
    }
    return AH_OK;
  };
  if ((st = fasta_pack_hooked(c, text, n_bytes, b, hook))) return st;
  AH_CUDA(c, cudaGetLastError());
  AH_CUDA(c, cudaGraphLaunch(pl->post_exec, c->stream));
  c->n_launches += pl->post_kernel_nodes + scan_launches;
  c->scan_ops_per_group = pl->range_kern.alu_ops_per_group;
  return AH_OK;
}

ah_status ah_plan_check(ah_plan* pl) {
  if (!pl) return AH_EINVAL;
  ah_ctx* c = pl->ctx;
  cudaStream_t s = c->stream;
  AH_CUDA(c, cudaMemcpyAsync(pl->h_out + 0, pl->ctr, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  AH_CUDA(c, cudaMemcpyAsync(pl->h_out + 1, pl->tpc_off + pl->n_cells, 8, cudaMemcpyDeviceToHost, s));
  AH_CUDA(c, cudaMemcpyAsync(pl->h_out + 2, pl->poff + pl->hit_cap, 8, cudaMemcpyDeviceToHost, s));
  if (pl->prm.tm.filter)
    AH_CUDA(c, cudaMemcpyAsync(pl->h_out + 3, pl->koff + pl->amp_cap, 8, cudaMemcpyDeviceToHost, s));
  if (pl->prm.extract)
    AH_CUDA(c, cudaMemcpyAsync(pl->h_out + 4, pl->ebase + pl->amp_cap, 8, cudaMemcpyDeviceToHost, s));
  AH_CUDA(c, cudaStreamSynchronize(s));
  ah_status st = check_status(c);
  if (st) return st;
  const uint32_t* cw = (const uint32_t*)pl->h_out;
  const uint32_t max_tile = cw[0];
  pl->info.n_hits = pl->h_out[1];
  pl->info.n_amps = pl->h_out[2];
  pl->info.n_kept = pl->prm.tm.filter ? pl->h_out[3] : std::min(pl->h_out[2], pl->amp_cap);
  pl->info.arena_bytes = pl->prm.extract ? pl->h_out[4] : 0;
  pl->info.max_tile_sites = max_tile;
  const bool over = max_tile > pl->slot_cap || pl->info.n_hits > pl->hit_cap || pl->info.n_amps > pl->amp_cap ||
                    (pl->prm.extract && pl->info.arena_bytes > pl->arena_cap);
  if (over)
    return fail(c, AH_EOVERFLOW, "plan capacities exceeded: tile %u/%u sites %llu/%llu amplicons %llu/%llu arena %llu/%llu",
                max_tile, pl->slot_cap, (unsigned long long)pl->info.n_hits, (unsigned long long)pl->hit_cap,
                (unsigned long long)pl->info.n_amps, (unsigned long long)pl->amp_cap,
                (unsigned long long)pl->info.arena_bytes, (unsigned long long)pl->arena_cap);
  return AH_OK;
}

ah_status ah_plan_run(ah_plan* pl) {
  if (!pl) return AH_EINVAL;
  for (int attempt = 0; attempt < 4; ++attempt) {
    ah_status st = ah_plan_launch(pl);
    if (st) return st;
    st = ah_plan_check(pl);
    if (st != AH_EOVERFLOW) return st;
    if ((st = grow(pl, true)) != AH_OK) return st;
  }
  return fail(pl->ctx, AH_EOVERFLOW, "plan: capacities kept overflowing");
}

ah_status ah_plan_info_get(const ah_plan* pl, ah_plan_info* out) {
  if (!pl || !out) return AH_EINVAL;
  *out = pl->info;
  out->slot_cap = pl->slot_cap;
  out->hit_capacity = pl->hit_cap;
  out->amp_capacity = pl->amp_cap;
  out->arena_capacity = pl->arena_cap;
  return AH_OK;
}

ah_status ah_plan_copy_results(ah_plan* pl, ah_hit* hits, uint64_t hits_cap, ah_amplicon* amps, uint64_t amps_cap,
                               char* arena, uint64_t arena_cap, uint64_t* field_off, uint64_t field_off_cap) {
  if (!pl) return AH_EINVAL;
  ah_status st = ah_plan_check(pl);
  if (st) return st;
  ah_ctx* c = pl->ctx;
  const ah_plan_info& i = pl->info;
  const uint64_t nf = pl->prm.extract ? 5 * i.n_kept + 1 : 0;
  if ((hits && hits_cap < i.n_hits) || (amps && amps_cap < i.n_kept) ||
      (arena && pl->prm.extract && arena_cap < i.arena_bytes) || (field_off && field_off_cap < nf))
    return fail(c, AH_EOVERFLOW, "ah_plan_copy_results: buffers smaller than the results (%llu sites, %llu amplicons, "
                "%llu arena bytes)", (unsigned long long)i.n_hits, (unsigned long long)i.n_kept,
                (unsigned long long)i.arena_bytes);
  cudaStream_t s = c->stream;
  if (hits && i.n_hits) AH_CUDA(c, cudaMemcpyAsync(hits, pl->hits, i.n_hits * sizeof(ah_hit), cudaMemcpyDeviceToHost, s));
  if (amps && i.n_kept)
    AH_CUDA(c, cudaMemcpyAsync(amps, pl->prm.tm.filter ? pl->kept : pl->amps, i.n_kept * sizeof(ah_amplicon),
                               cudaMemcpyDeviceToHost, s));
  if (arena && pl->prm.extract && i.arena_bytes)
    AH_CUDA(c, cudaMemcpyAsync(arena, pl->arena, i.arena_bytes, cudaMemcpyDeviceToHost, s));
  if (field_off && nf) AH_CUDA(c, cudaMemcpyAsync(field_off, pl->field_off, nf * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  AH_CUDA(c, cudaStreamSynchronize(s));
  return AH_OK;
}

ah_status ah_plan_results(ah_plan* pl, ah_hits** hits_out, ah_amplicons** amps_out) {
  if (!pl || !hits_out || !amps_out) return AH_EINVAL;
  *hits_out = nullptr;
  *amps_out = nullptr;
  ah_status st = ah_plan_check(pl);
  if (st) return st;
  ah_ctx* c = pl->ctx;
  cudaStream_t s = c->stream;
  ah_hits* h = new ah_hits();
  h->ctx = c;
  h->n = pl->info.n_hits;
  h->n_pairs = pl->p->n_pairs;
  ah_amplicons* a = new ah_amplicons();
  a->ctx = c;
  a->n = pl->info.n_kept;
  const uint64_t nf = pl->prm.extract ? 5 * a->n + 1 : 0;
  if ((st = dalloc(c, &h->d, h->n)) || (st = dalloc(c, &h->d_pair_off, h->n_pairs + 1)) || (st = dalloc(c, &a->d, a->n)) ||
      (pl->prm.extract && ((st = dalloc(c, &a->d_arena, pl->info.arena_bytes)) || (st = dalloc(c, &a->d_field_off, nf))))) {
    ah_hits_free(h);
    ah_amplicons_free(a);
    return st;
  }
  AH_CUDA(c, cudaMemcpyAsync(h->d, pl->hits, h->n * sizeof(ah_hit), cudaMemcpyDeviceToDevice, s));
  AH_CUDA(c, cudaMemcpyAsync(h->d_pair_off, pl->pair_off, (h->n_pairs + 1) * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                             s));
  AH_CUDA(c, cudaMemcpyAsync(a->d, pl->prm.tm.filter ? pl->kept : pl->amps, a->n * sizeof(ah_amplicon),
                             cudaMemcpyDeviceToDevice, s));
  if (pl->prm.extract) {
    a->arena_bytes = pl->info.arena_bytes;
    if (a->arena_bytes)
      AH_CUDA(c, cudaMemcpyAsync(a->d_arena, pl->arena, a->arena_bytes, cudaMemcpyDeviceToDevice, s));
    AH_CUDA(c, cudaMemcpyAsync(a->d_field_off, pl->field_off, nf * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  }
  h->h_pair_off.resize(h->n_pairs + 1);
  AH_CUDA(c, cudaMemcpyAsync(h->h_pair_off.data(), pl->pair_off, (h->n_pairs + 1) * sizeof(uint64_t),
                             cudaMemcpyDeviceToHost, s));
  AH_CUDA(c, cudaStreamSynchronize(s));
  *hits_out = h;
  *amps_out = a;
  return AH_OK;
}

void ah_plan_free(ah_plan* pl) {
  if (!pl) return;
  if (pl->ctx) {
    cudaSetDevice(pl->ctx->device);
    // timings of this plan's replays that are still unread are read now
    for (uint64_t g : pl->ring_gen)
      if (g == pl->ctx->drain_gen + 1) {
        drain_timings(pl->ctx);
        break;
      }
    free_buffers(pl);
    if (pl->h_out) cudaFreeHost(pl->h_out);
    for (cudaEvent_t e : pl->scan_ev)
      if (e) cudaEventDestroy(e);
    for (auto& pr : pl->ring_ev)
      for (cudaEvent_t e : pr)
        if (e) cudaEventDestroy(e);
  }
  delete pl;
}

}  // extern "C"
