// weno_engine.cu -- C-ABI of the serving engine (declared in include/weno.h).
//
// Continuous batching of independent 1D/2D Euler solves on one GPU:
//  * device memory is a caller-provided arena; the engine keeps a fixed
//    control region at its start (slot table, tile work list, rotating work
//    counters, per-slot speed slots, clocks, step counts and status) and a
//    first-fit heap for the slots' states (U, U1, U2), so admission is decided
//    by free arena space and never calls the allocator;
//  * every engine step is three launches of one persistent kernel (one per
//    Runge-Kutta stage) that takes tiles of all admitted slots from the work
//    list; the three launches are captured once in a CUDA graph, whose
//    arguments never change -- admission and retirement only rewrite the work
//    list and the slot table in device memory;
//  * each slot advances with its own CFL step to its own t_final; finished
//    slots stop (their tiles return at once) until the host retires them;
//  * a fast slot takes WENO_ENGINE_FAST_STEPS steps per engine step: its
//    tiles sit at the end of the work list, and the graph used while any
//    slot is fast repeats the three launches over that tail.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/weno.h"
#include "weno_internal.h"

using weno::DevStatus;
using weno::EngineTile;
using weno::SlotDev;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

weno_status efail(weno_status s, const std::string &m) {
  weno::set_last_error(m);
  return s;
}

weno_status ecuda(cudaError_t e, const char *what) {
  return efail(WENO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct ControlLayout {
  size_t slots, tiles, ntiles, first, counters, alpha, clock, steps, status, total;
};

ControlLayout control_layout(int max_slots, long long max_tiles) {
  ControlLayout L;
  size_t o = 0;
  L.slots = o;
  o = align256(o + sizeof(SlotDev) * (size_t)max_slots);
  L.tiles = o;
  o = align256(o + sizeof(EngineTile) * (size_t)max_tiles);
  L.ntiles = o;
  o = align256(o + sizeof(int));
  L.first = o;  // [0] = 0, [1] = first entry of the fast slots' tiles
  o = align256(o + 2 * sizeof(int));
  L.counters = o;
  o = align256(o + 3 * sizeof(int));
  L.alpha = o;
  o = align256(o + 24 * sizeof(unsigned long long) * (size_t)max_slots);
  L.clock = o;
  o = align256(o + 3 * sizeof(double) * (size_t)max_slots);
  L.steps = o;
  o = align256(o + sizeof(long long) * (size_t)max_slots);
  L.status = o;
  o = align256(o + sizeof(DevStatus) * (size_t)max_slots);
  L.total = o;
  return L;
}

struct SlotHost {
  bool used = false;
  bool fast = false;
  int ndim = 0, precision = 0;
  long long cells = 0, tiles = 0;
  size_t off = 0, bytes = 0, state_bytes = 0;
};

}  // namespace

struct weno_engine {
  cudaStream_t s = nullptr;
  bool own_stream = false;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  int max_slots = 0;
  long long max_tiles = 0;
  ControlLayout L;
  std::map<size_t, size_t> free_blocks;  // heap offset -> size
  std::vector<SlotHost> slots;
  std::vector<SlotDev> mirror;
  bool dirty = true;
  long long tiles_in_use = 0;
  // stream the graphs run on when the caller lowers the engine's priority
  // (weno_engine_set_priority; one stream per priority used, kept until
  // destroy); events keep it in order with `s`
  cudaStream_t s_run = nullptr;
  std::map<int, cudaStream_t> run_streams;
  int run_priority = 0, greatest_priority = 0;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph = nullptr;       // one sub-step per engine step
  cudaGraphExec_t graph_fast = nullptr;  // WENO_ENGINE_FAST_STEPS sub-steps
  int n_fast = 0;                        // used slots marked fast
  int grid = 0;

  SlotDev *d_slots() const { return (SlotDev *)(arena + L.slots); }
  EngineTile *d_tiles() const { return (EngineTile *)(arena + L.tiles); }
  int *d_ntiles() const { return (int *)(arena + L.ntiles); }
  int *d_first() const { return (int *)(arena + L.first); }
  int *d_counters() const { return (int *)(arena + L.counters); }
  unsigned long long *d_alpha(int k) const { return (unsigned long long *)(arena + L.alpha) + 24 * k; }
  double *d_clock(int k) const { return (double *)(arena + L.clock) + 3 * k; }
  long long *d_steps(int k) const { return (long long *)(arena + L.steps) + k; }
  DevStatus *d_status(int k) const { return (DevStatus *)(arena + L.status) + k; }

  bool heap_alloc(size_t bytes, size_t *off) {
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_blocks.erase(it);
        if (rest) free_blocks[at] = rest;
        return true;
      }
    }
    return false;
  }
  void heap_free(size_t off, size_t bytes) {
    auto it = free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
  size_t heap_largest() const {
    size_t m = 0;
    for (auto &b : free_blocks) m = std::max(m, b.second);
    return m;
  }
};

namespace {

// Upload the slot table and the work list: the normal slots' tiles, then the
// fast slots' tiles; within each part the costliest classes first (2D FP64,
// 2D FP32, 1D), so the atomic work counter hands out the long tiles early
// and the short ones fill the tail.
weno_status upload(weno_engine *E) {
  std::vector<EngineTile> list;
  list.reserve((size_t)E->tiles_in_use);
  const int order[3][2] = {{2, 0}, {2, 1}, {1, -1}};
  int first[2] = {0, 0};
  for (int part = 0; part < 2; ++part) {
    if (part == 1) first[1] = (int)list.size();
    for (auto &cls : order)
      for (int k = 0; k < E->max_slots; ++k) {
        const SlotHost &h = E->slots[k];
        if (!h.used || h.fast != (part == 1) || h.ndim != cls[0]) continue;
        if (cls[1] >= 0 && h.precision != cls[1]) continue;
        for (long long t = 0; t < h.tiles; ++t) list.push_back({k, (int)t});
      }
  }
  const int n = (int)list.size();
  cudaError_t e = cudaSuccess;
  if (n) e = cudaMemcpyAsync(E->d_tiles(), list.data(), sizeof(EngineTile) * n,
                             cudaMemcpyHostToDevice, E->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(E->d_ntiles(), &n, sizeof(int), cudaMemcpyHostToDevice, E->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(E->d_first(), first, sizeof(first), cudaMemcpyHostToDevice, E->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(E->d_slots(), E->mirror.data(), sizeof(SlotDev) * E->max_slots,
                        cudaMemcpyHostToDevice, E->s);
  // the host vectors are pageable: finish the copies before they go out of scope
  if (e == cudaSuccess) e = cudaStreamSynchronize(E->s);
  if (e != cudaSuccess) return ecuda(e, "engine work-list upload");
  E->dirty = false;
  return WENO_OK;
}

// One engine step as a graph of `substeps` x 3 stage launches: the first
// sub-step over the whole work list, the others from the fast slots' first
// entry on.
weno_status build_graph(weno_engine *E, int substeps, cudaGraphExec_t *out) {
  weno::EngineArgs a;
  a.slots = E->d_slots();
  a.tiles = E->d_tiles();
  a.ntiles = E->d_ntiles();
  a.counters = E->d_counters();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(E->s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return ecuda(e, "cudaStreamBeginCapture");
  for (int sub = 0; sub < substeps && e == cudaSuccess; ++sub) {
    a.first = E->d_first() + (sub == 0 ? 0 : 1);
    for (int st = 1; st <= 3; ++st) {
      a.stage = st;
      e = weno::launch_engine_stage(a, E->grid, E->s);
      if (e != cudaSuccess) break;
    }
  }
  cudaError_t e2 = cudaStreamEndCapture(E->s, &g);
  if (e != cudaSuccess) return ecuda(e, "engine stage capture");
  if (e2 != cudaSuccess) return ecuda(e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return ecuda(e, "cudaGraphInstantiate");
  return WENO_OK;
}

}  // namespace

extern "C" {

size_t weno_engine_control_bytes(int max_slots, int64_t max_tiles) {
  if (max_slots < 1 || max_tiles < 1) return 0;
  return control_layout(max_slots, max_tiles).total;
}

size_t weno_engine_slot_bytes(const weno_desc *d) {
  if (weno_workspace_bytes(d) == 0) return 0;
  const int nc = d->ndim == 1 ? 3 : 4;
  return 3 * align256(sizeof(double) * nc * (size_t)d->nx * (size_t)d->ny);
}

weno_status weno_engine_create(void *arena, size_t arena_bytes, int max_slots, int64_t max_tiles,
                               void *stream, weno_engine **out) {
  if (!out) return efail(WENO_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!arena || ((uintptr_t)arena & 255)) return efail(WENO_ERR_ARG, "arena must be 256-byte aligned");
  if (max_slots < 1 || max_tiles < 1 || max_tiles > (1LL << 30))
    return efail(WENO_ERR_ARG, "max_slots and max_tiles must be positive");
  const ControlLayout L = control_layout(max_slots, max_tiles);
  if (arena_bytes < L.total + 256) return efail(WENO_ERR_NOMEM, "arena smaller than the control region");
  weno_engine *E = new weno_engine();
  E->arena = (char *)arena;
  E->arena_bytes = arena_bytes;
  E->max_slots = max_slots;
  E->max_tiles = max_tiles;
  E->L = L;
  E->slots.assign(max_slots, SlotHost());
  E->mirror.assign(max_slots, SlotDev());
  std::memset(E->mirror.data(), 0, sizeof(SlotDev) * max_slots);
  E->free_blocks[L.total] = (arena_bytes - L.total) & ~size_t(255);
  (void)stream;  // the engine works on a stream of its own (a graph needs a capturable stream)
  // ... of the highest priority: while a caller runs a large solve on a
  // stream of lower priority, the block scheduler hands the engine's blocks
  // the next free places on the SMs, so the small solves it holds keep
  // their pace instead of waiting for the large one to finish
  int prio_least = 0, prio_greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&E->s, cudaStreamNonBlocking, prio_greatest);
  E->run_priority = E->greatest_priority = prio_greatest;
  if (e != cudaSuccess) {
    delete E;
    return ecuda(e, "cudaStreamCreateWithFlags");
  }
  E->own_stream = true;
  e = weno::engine_prepare();
  if (e != cudaSuccess) {
    cudaStreamDestroy(E->s);
    delete E;
    return ecuda(e, "engine kernel attributes");
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  E->grid = (sms > 0 ? sms : 1) * weno::kEngineBlocksPerSM;
  e = cudaMemsetAsync(arena, 0, L.total, E->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E->s);
  if (e != cudaSuccess) {
    if (E->own_stream) cudaStreamDestroy(E->s);
    delete E;
    return ecuda(e, "engine control reset");
  }
  weno_status st = upload(E);
  if (st == WENO_OK) st = build_graph(E, 1, &E->graph);
  if (st == WENO_OK) st = build_graph(E, WENO_ENGINE_FAST_STEPS, &E->graph_fast);
  if (st != WENO_OK) {
    if (E->graph) cudaGraphExecDestroy(E->graph);
    if (E->graph_fast) cudaGraphExecDestroy(E->graph_fast);
    if (E->own_stream) cudaStreamDestroy(E->s);
    delete E;
    return st;
  }
  *out = E;
  return WENO_OK;
}

weno_status weno_engine_admit(weno_engine *E, const weno_desc *d, const double *U_host,
                              double t_final, int *slot_out) {
  if (!E || !d || !U_host || !slot_out) return efail(WENO_ERR_ARG, "NULL argument");
  *slot_out = -1;
  if (weno_workspace_bytes(d) == 0) return WENO_ERR_ARG;
  if (d->system != WENO_SYS_EULER || d->nbatch != 1 || d->ai != 1 || d->p != 1.0 ||
      (d->order != 0 && d->order != 6))
    return efail(WENO_ERR_ARG,
                 "the engine serves single sixth-order Euler problems with ai = 1, p = 1");
  if (!(std::isfinite(t_final) && t_final > 0.0)) return efail(WENO_ERR_ARG, "t_final must be > 0");
  int k = -1;
  for (int q = 0; q < E->max_slots; ++q)
    if (!E->slots[q].used) {
      k = q;
      break;
    }
  if (k < 0) return efail(WENO_ERR_NOMEM, "no free slot");
  const long long tiles = weno::engine_tiles_of(d->ndim, d->nx, d->ny);
  if (E->tiles_in_use + tiles > E->max_tiles) return efail(WENO_ERR_NOMEM, "work list full");
  const int nc = d->ndim == 1 ? 3 : 4;
  const size_t sb = align256(sizeof(double) * nc * (size_t)d->nx * (size_t)d->ny);
  size_t off = 0;
  if (!E->heap_alloc(3 * sb, &off)) return efail(WENO_ERR_NOMEM, "arena full");
  SlotHost &h = E->slots[k];
  h.used = true;
  h.ndim = d->ndim;
  h.precision = d->precision;
  h.cells = d->nx * d->ny;
  h.tiles = tiles;
  h.off = off;
  h.bytes = 3 * sb;
  h.state_bytes = sizeof(double) * nc * (size_t)d->nx * (size_t)d->ny;
  E->tiles_in_use += tiles;
  SlotDev &S = E->mirror[k];
  std::memset(&S, 0, sizeof(S));
  S.ndim = d->ndim;
  S.nc = nc;
  S.bc_x = d->bc_x;
  S.bc_y = d->bc_y;
  S.precision = d->precision;
  S.alpha_single = d->alpha_mode == WENO_ALPHA_SINGLE;
  S.active = 1;
  S.nx = d->nx;
  S.ny = d->ny;
  S.dx = (d->x1 - d->x0) / (double)d->nx;
  S.dy = d->ndim == 2 ? (d->y1 - d->y0) / (double)d->ny : 1.0;
  S.gamma = d->gamma;
  S.cfl = d->cfl;
  S.eps = d->eps;
  S.mu0 = d->mu0;
  S.p = d->p;
  S.t_final = t_final;
  S.U = (double *)(E->arena + off);
  S.U1 = (double *)(E->arena + off + sb);
  S.U2 = (double *)(E->arena + off + 2 * sb);
  S.alpha = E->d_alpha(k);
  S.clock = E->d_clock(k);
  S.steps = E->d_steps(k);
  S.status = E->d_status(k);
  cudaError_t e = cudaMemcpyAsync(S.U, U_host, h.state_bytes, cudaMemcpyHostToDevice, E->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.alpha, 0, 24 * sizeof(unsigned long long), E->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.clock, 0, 3 * sizeof(double), E->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.steps, 0, sizeof(long long), E->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(S.status, 0, sizeof(DevStatus), E->s);
  if (e == cudaSuccess) {
    weno::AlphaArgs a = {};
    a.system = 1;
    a.ndim = d->ndim;
    a.nc = nc;
    a.alpha_single = S.alpha_single;
    a.nbatch = 1;
    a.nx = d->nx;
    a.ny = d->ny;
    a.dx = S.dx;
    a.dy = S.dy;
    a.gamma = d->gamma;
    a.cfl = d->cfl;
    a.adv_speed = 0.0;
    a.U = S.U;
    a.alpha_out = S.alpha;  // the speed slot the next stage 1 reads
    a.status = S.status;
    e = weno::launch_alpha(a, E->s);
  }
  // the caller may reuse U_host as soon as this returns
  if (e == cudaSuccess) e = cudaStreamSynchronize(E->s);
  if (e != cudaSuccess) {
    h.used = false;
    E->tiles_in_use -= tiles;
    E->heap_free(off, 3 * sb);
    std::memset(&S, 0, sizeof(S));
    return ecuda(e, "engine admission");
  }
  E->dirty = true;
  *slot_out = k;
  return WENO_OK;
}

weno_status weno_engine_run(weno_engine *E, int nsteps) {
  if (!E || nsteps < 0) return efail(WENO_ERR_ARG, "bad engine or step count");
  if (E->dirty) {
    weno_status st = upload(E);
    if (st != WENO_OK) return st;
  }
  cudaGraphExec_t g = E->n_fast > 0 ? E->graph_fast : E->graph;
  cudaStream_t rs = E->s_run ? E->s_run : E->s;
  cudaError_t e = cudaSuccess;
  if (rs != E->s) {  // the run stream starts after everything enqueued on s
    e = cudaEventRecord(E->ev_in, E->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, E->ev_in, 0);
    if (e != cudaSuccess) return ecuda(e, "engine stream order");
  }
  for (int q = 0; q < nsteps; ++q) {
    e = cudaGraphLaunch(g, rs);
    if (e != cudaSuccess) return ecuda(e, "cudaGraphLaunch");
  }
  if (rs != E->s) {  // and s (polls, admissions) after the run
    e = cudaEventRecord(E->ev_out, rs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(E->s, E->ev_out, 0);
    if (e != cudaSuccess) return ecuda(e, "engine stream order");
  }
  return WENO_OK;
}

weno_status weno_engine_set_priority(weno_engine *E, int priority) {
  if (!E) return efail(WENO_ERR_ARG, "NULL engine");
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e != cudaSuccess) return ecuda(e, "cudaDeviceGetStreamPriorityRange");
  if (priority < greatest) priority = greatest;  // lower numbers are higher priorities
  if (priority > least) priority = least;
  if (priority == E->run_priority) return WENO_OK;
  cudaStream_t ns = nullptr;  // NULL: the engine's own stream (the highest priority)
  if (priority != E->greatest_priority) {
    auto it = E->run_streams.find(priority);
    if (it != E->run_streams.end()) {
      ns = it->second;
    } else {
      e = cudaStreamCreateWithPriority(&ns, cudaStreamNonBlocking, priority);
      if (e == cudaSuccess && !E->ev_in)
        e = cudaEventCreateWithFlags(&E->ev_in, cudaEventDisableTiming);
      if (e == cudaSuccess && !E->ev_out)
        e = cudaEventCreateWithFlags(&E->ev_out, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        if (ns) cudaStreamDestroy(ns);
        return ecuda(e, "engine run stream");
      }
      E->run_streams[priority] = ns;
    }
  }
  // every run on the previous stream is ordered before `s` (run() makes `s`
  // wait for it), and the next run waits for `s`: switching needs no sync
  E->s_run = ns;
  E->run_priority = priority;
  return WENO_OK;
}

weno_status weno_engine_set_fast(weno_engine *E, int slot, int fast) {
  if (!E || slot < 0 || slot >= E->max_slots || !E->slots[slot].used)
    return efail(WENO_ERR_ARG, "no such slot");
  if (fast != 0 && fast != 1) return efail(WENO_ERR_ARG, "fast must be 0 or 1");
  SlotHost &h = E->slots[slot];
  if (h.fast != (fast == 1)) {
    h.fast = fast == 1;
    E->n_fast += fast ? 1 : -1;
    E->dirty = true;
  }
  return WENO_OK;
}

weno_status weno_engine_poll(weno_engine *E, int *done, int max_done, int *n_done, int *n_active) {
  if (!E || !n_done) return efail(WENO_ERR_ARG, "NULL argument");
  std::vector<double> clk(3 * (size_t)E->max_slots);
  std::vector<DevStatus> stv(E->max_slots);
  cudaError_t e = cudaMemcpyAsync(clk.data(), E->d_clock(0), sizeof(double) * clk.size(),
                                  cudaMemcpyDeviceToHost, E->s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(stv.data(), E->d_status(0), sizeof(DevStatus) * stv.size(),
                        cudaMemcpyDeviceToHost, E->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E->s);
  if (e != cudaSuccess) return ecuda(e, "engine poll");
  int nd = 0, na = 0;
  for (int k = 0; k < E->max_slots; ++k) {
    if (!E->slots[k].used) continue;
    ++na;
    const bool fin = !(clk[3 * k] < E->mirror[k].t_final) || stv[k].code != 0;
    if (fin) {
      if (done && nd < max_done) done[nd] = k;
      ++nd;
    }
  }
  *n_done = nd;
  if (n_active) *n_active = na;
  return WENO_OK;
}

weno_status weno_engine_retire(weno_engine *E, int slot, double *U_host, double *t_out,
                               int64_t *steps_out) {
  if (!E || slot < 0 || slot >= E->max_slots || !E->slots[slot].used)
    return efail(WENO_ERR_ARG, "no such slot");
  SlotHost &h = E->slots[slot];
  SlotDev &S = E->mirror[slot];
  double clk[3] = {0, 0, 0};
  long long steps = 0;
  DevStatus st;
  cudaError_t e = cudaSuccess;
  if (U_host) e = cudaMemcpyAsync(U_host, S.U, h.state_bytes, cudaMemcpyDeviceToHost, E->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(clk, S.clock, sizeof(clk), cudaMemcpyDeviceToHost, E->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&steps, S.steps, sizeof(steps), cudaMemcpyDeviceToHost, E->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, S.status, sizeof(st), cudaMemcpyDeviceToHost, E->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E->s);
  if (e != cudaSuccess) return ecuda(e, "engine retire");
  if (t_out) *t_out = clk[0];
  if (steps_out) *steps_out = steps;
  E->heap_free(h.off, h.bytes);
  E->tiles_in_use -= h.tiles;
  if (h.fast) --E->n_fast;
  h = SlotHost();
  std::memset(&S, 0, sizeof(S));
  E->dirty = true;
  if (st.code != 0) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "slot %d: nonphysical state at cell (j=%lld, i=%lld)", slot, st.j,
                  st.i);
    return efail(WENO_ERR_NONPHYSICAL, buf);
  }
  return WENO_OK;
}

weno_status weno_engine_info(const weno_engine *E, size_t *heap_free_bytes, size_t *heap_largest,
                             int64_t *tiles_in_use) {
  if (!E) return efail(WENO_ERR_ARG, "NULL engine");
  size_t tot = 0;
  for (auto &b : E->free_blocks) tot += b.second;
  if (heap_free_bytes) *heap_free_bytes = tot;
  if (heap_largest) *heap_largest = E->heap_largest();
  if (tiles_in_use) *tiles_in_use = E->tiles_in_use;
  return WENO_OK;
}

weno_status weno_engine_destroy(weno_engine *E) {
  if (!E) return WENO_OK;
  cudaStreamSynchronize(E->s);
  for (auto &kv : E->run_streams) {
    cudaStreamSynchronize(kv.second);
    cudaStreamDestroy(kv.second);
  }
  if (E->ev_in) cudaEventDestroy(E->ev_in);
  if (E->ev_out) cudaEventDestroy(E->ev_out);
  if (E->graph) cudaGraphExecDestroy(E->graph);
  if (E->graph_fast) cudaGraphExecDestroy(E->graph_fast);
  if (E->own_stream) cudaStreamDestroy(E->s);
  delete E;
  return WENO_OK;
}

}  // extern "C"
