// weno_api.cu -- the C-ABI of libweno (declared in include/weno.h).
//
// Host-side sequencing only: argument checks, the workspace layout, and the
// launches of one Runge-Kutta step (Section 4 preamble of arXiv 2603.26272:
// three stages of the third-order TVD scheme).  Every arithmetic step of the
// method runs in the kernels of weno_kernels.cu.
//
// Workspace layout (each part 256-byte aligned):
//   DevStatus | alpha slots [3][nbatch][8] (u64 bit patterns of speed maxima)
//   | t[nbatch] | tnext[nbatch] | dt[nbatch] | steps[nbatch] | U1 | U2 [| Uhost copy]
// The three alpha slots rotate through the stage launches: the launch that
// reads slot k accumulates into slot k+1 and clears slot k+2, so no launch
// ever waits on the host and no slot is read while it is written.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/weno.h"
#include "weno_internal.h"

using weno::AlphaArgs;
using weno::DevStatus;
using weno::StageArgs;

namespace {

thread_local std::string g_err;

weno_status fail(weno_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

weno_status cuda_fail(cudaError_t e, const char *what) {
  return fail(WENO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int ncomp(const weno_desc *d) {
  if (d->system != WENO_SYS_EULER) return 1;
  return d->ndim == 1 ? 3 : 4;
}

struct Layout {
  size_t status, alpha, t, tnext, dt, steps, u1, u2, uhost, total, total_host;
  size_t state_bytes;
};

Layout layout(const weno_desc *d) {
  Layout L;
  const size_t nb = (size_t)d->nbatch;
  L.state_bytes = sizeof(double) * nb * ncomp(d) * (size_t)d->nx * (size_t)d->ny;
  size_t o = 0;
  L.status = o;
  o = align256(o + sizeof(DevStatus));
  L.alpha = o;
  o = align256(o + 3 * nb * 8 * sizeof(unsigned long long));
  L.t = o;
  o = align256(o + nb * sizeof(double));
  L.tnext = o;
  o = align256(o + nb * sizeof(double));
  L.dt = o;
  o = align256(o + nb * sizeof(double));
  L.steps = o;
  o = align256(o + nb * sizeof(long long));
  L.u1 = o;
  o = align256(o + L.state_bytes);
  L.u2 = o;
  o = align256(o + L.state_bytes);
  L.total = o;
  L.uhost = o;
  o = align256(o + L.state_bytes);
  L.total_host = o;
  return L;
}

weno_status check_desc(const weno_desc *d) {
  if (!d) return fail(WENO_ERR_ARG, "descriptor is NULL");
  if (d->system < WENO_SYS_ADVECTION || d->system > WENO_SYS_BUCKLEY_LEVERETT)
    return fail(WENO_ERR_ARG, "system must be one of WENO_SYS_*");
  if (d->ndim != 1 && d->ndim != 2) return fail(WENO_ERR_ARG, "ndim must be 1 or 2");
  if (d->system != WENO_SYS_EULER && d->ndim != 1)
    return fail(WENO_ERR_ARG, "the scalar equations are one-dimensional");
  if (d->nbatch < 1 || d->nbatch > 65535) return fail(WENO_ERR_ARG, "nbatch must be in [1, 65535]");
  if (d->nx < 1 || d->ny < 1) return fail(WENO_ERR_ARG, "nx and ny must be >= 1");
  if (d->ndim == 1 && d->ny != 1) return fail(WENO_ERR_ARG, "ny must be 1 in 1D");
  if (d->nx > (1LL << 31) || d->ny > (1LL << 31)) return fail(WENO_ERR_ARG, "grid too large");
  if ((double)d->nbatch * ncomp(d) * (double)d->nx * (double)d->ny > 4.0e12)
    return fail(WENO_ERR_ARG, "state too large");
  if (!(d->x1 > d->x0)) return fail(WENO_ERR_ARG, "x1 must exceed x0");
  if (d->ndim == 2 && !(d->y1 > d->y0)) return fail(WENO_ERR_ARG, "y1 must exceed y0");
  if (d->bc_x != WENO_BC_TRANSMISSIVE && d->bc_x != WENO_BC_PERIODIC)
    return fail(WENO_ERR_ARG, "bc_x must be WENO_BC_TRANSMISSIVE or WENO_BC_PERIODIC");
  if (d->ndim == 2 && d->bc_y != WENO_BC_TRANSMISSIVE && d->bc_y != WENO_BC_PERIODIC)
    return fail(WENO_ERR_ARG, "bc_y must be WENO_BC_TRANSMISSIVE or WENO_BC_PERIODIC");
  if (d->system == WENO_SYS_EULER && !(d->gamma > 1.0))
    return fail(WENO_ERR_ARG, "gamma must exceed 1");
  if (!(d->cfl > 0.0) || !std::isfinite(d->cfl)) return fail(WENO_ERR_ARG, "cfl must be > 0");
  if (!(d->eps > 0.0) || !std::isfinite(d->eps)) return fail(WENO_ERR_ARG, "eps must be > 0");
  if (!(d->mu0 >= 0.0) || !std::isfinite(d->mu0)) return fail(WENO_ERR_ARG, "mu0 must be >= 0");
  if (d->ai && !(d->mu0 > 0.0)) return fail(WENO_ERR_ARG, "mu0 must be > 0 with ai = 1 (eq. (22))");
  // With ai = 1 and p = 1 the kernels rescale the indicators b_k = 4 beta_k +
  // 4 eps mu^2 by an add to their exponent fields, which is exact only for
  // normal numbers.  A field reaches the reconstruction scaled by k >= 2, so
  // the smallest sensitivity term is 4 eps (2 mu0)^2 = 16 eps mu0^2; it must be
  // a normal double (1e-300 leaves eight decades above DBL_MIN), and eps >=
  // 1e-250 keeps every b_k within 1e-254 of the largest, so the rescaled
  // values stay normal too.
  if (d->ai && !(d->eps >= 1e-250 && 16.0 * d->eps * d->mu0 * d->mu0 >= 1e-300))
    return fail(WENO_ERR_ARG, "with ai = 1 the kernels need eps >= 1e-250 and 16 eps mu0^2 >= "
                              "1e-300 (their weights scale exponents, which needs eps mu^2 to stay "
                              "a normal double)");
  if (!(d->p > 0.0) || !std::isfinite(d->p)) return fail(WENO_ERR_ARG, "p must be > 0");
  if (d->ai != 0 && d->ai != 1) return fail(WENO_ERR_ARG, "ai must be 0 or 1");
  if (d->precision != WENO_PREC_FP64 && d->precision != WENO_PREC_FP32_RECON)
    return fail(WENO_ERR_ARG, "precision must be WENO_PREC_FP64 or WENO_PREC_FP32_RECON");
  if (d->precision == WENO_PREC_FP32_RECON && !d->ai)
    return fail(WENO_ERR_ARG, "WENO_PREC_FP32_RECON needs ai = 1 (its normalisation relies on "
                              "the affine-invariant weights)");
  if (d->alpha_mode != WENO_ALPHA_FIELD && d->alpha_mode != WENO_ALPHA_SINGLE)
    return fail(WENO_ERR_ARG, "alpha_mode must be WENO_ALPHA_FIELD or WENO_ALPHA_SINGLE");
  if (d->order != 0 && d->order != 4 && d->order != 6 && d->order != 8 && d->order != 10)
    return fail(WENO_ERR_ARG, "order must be 0 (= 6), 4, 6, 8 or 10");
  if (d->precision == WENO_PREC_FP32_RECON && d->order != 0 && d->order != 6)
    return fail(WENO_ERR_ARG, "WENO_PREC_FP32_RECON is implemented for order 6 only");
  if (d->system == WENO_SYS_ADVECTION && !(std::fabs(d->adv_speed) > 0.0 && std::isfinite(d->adv_speed)))
    return fail(WENO_ERR_ARG, "adv_speed must be finite and non-zero");
  return WENO_OK;
}

weno_status check_ws(const weno_desc *d, void *ws, size_t ws_bytes, size_t need) {
  if (!ws) return fail(WENO_ERR_ARG, "workspace is NULL");
  if (((uintptr_t)ws) & 255) return fail(WENO_ERR_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < need)
    return fail(WENO_ERR_NOMEM, "workspace of " + std::to_string(ws_bytes) + " bytes, need " +
                                    std::to_string(need));
  (void)d;
  return WENO_OK;
}

struct Ctx {
  const weno_desc *d;
  Layout L;
  char *ws;
  cudaStream_t s;
  DevStatus *status() const { return (DevStatus *)(ws + L.status); }
  unsigned long long *slot(int k) const {
    return (unsigned long long *)(ws + L.alpha) + (size_t)(k % 3) * d->nbatch * 8;
  }
  double *t() const { return (double *)(ws + L.t); }
  double *tnext() const { return (double *)(ws + L.tnext); }
  double *dt() const { return (double *)(ws + L.dt); }
  long long *steps() const { return (long long *)(ws + L.steps); }
  double *u1() const { return (double *)(ws + L.u1); }
  double *u2() const { return (double *)(ws + L.u2); }
};

AlphaArgs alpha_args(const Ctx &c, const double *U, unsigned long long *out) {
  const weno_desc *d = c.d;
  AlphaArgs a;
  a.system = d->system;
  a.ndim = d->ndim;
  a.nc = ncomp(d);
  a.nbatch = d->nbatch;
  a.nx = d->nx;
  a.ny = d->ny;
  a.dx = (d->x1 - d->x0) / (double)d->nx;
  a.dy = d->ndim == 2 ? (d->y1 - d->y0) / (double)d->ny : 1.0;
  a.gamma = d->gamma;
  a.cfl = d->cfl;
  a.adv_speed = d->adv_speed;
  a.ustar = weno::bl_speed_argmax();
  a.alpha_single = d->alpha_mode == WENO_ALPHA_SINGLE;
  a.U = U;
  a.alpha_out = out;
  a.status = c.status();
  return a;
}

StageArgs stage_args(const Ctx &c) {
  const weno_desc *d = c.d;
  StageArgs a;
  std::memset(&a, 0, sizeof(a));
  a.system = d->system;
  a.ndim = d->ndim;
  a.nc = ncomp(d);
  a.nbatch = d->nbatch;
  a.nx = d->nx;
  a.ny = d->ny;
  a.dx = (d->x1 - d->x0) / (double)d->nx;
  a.dy = d->ndim == 2 ? (d->y1 - d->y0) / (double)d->ny : 1.0;
  a.bc_x = d->bc_x;
  a.bc_y = d->bc_y;
  a.gamma = d->gamma;
  a.cfl = d->cfl;
  a.eps = d->eps;
  a.mu0 = d->mu0;
  a.p = d->p;
  a.ai = d->ai;
  a.alpha_single = d->alpha_mode == WENO_ALPHA_SINGLE;
  a.precision = d->precision;
  a.order_r = d->order == 0 ? 3 : d->order / 2;
  a.ustar = weno::bl_speed_argmax();
  a.adv_speed = d->adv_speed;
  a.t_final = INFINITY;
  a.t = c.t();
  a.tnext = c.tnext();
  a.dt = c.dt();
  a.steps = c.steps();
  a.status = c.status();
  return a;
}

// Clear status, the three alpha slots, clocks (t = t0) and step counters.
weno_status reset_control(const Ctx &c, double t0) {
  cudaError_t e = cudaMemsetAsync(c.ws, 0, c.L.u1, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (t0 != 0.0) {
    e = weno::launch_fill(c.t(), c.d->nbatch, t0, c.s);
    if (e != cudaSuccess) return cuda_fail(e, "fill");
  }
  return WENO_OK;
}

// Launch the three stages of one SSP-RK3 step; *k is the running slot index.
weno_status launch_step(const Ctx &c, double *U, double dt_fixed, double t_final, int *k,
                        bool last_alpha, int tile) {
  StageArgs a = stage_args(c);
  a.tile_variant = tile;
  a.mode = 0;
  a.dt_fixed = dt_fixed;
  a.t_final = t_final;
  struct S {
    const double *in;
    const double *un;
    double *out;
    double an, as;
  } st[3] = {{U, nullptr, c.u1(), 0.0, 1.0},
             {c.u1(), U, c.u2(), 0.75, 0.25},
             {c.u2(), U, U, 1.0 / 3.0, 2.0 / 3.0}};
  for (int s = 0; s < 3; ++s) {
    a.stage = s + 1;
    a.Uin = st[s].in;
    a.Un = st[s].un;
    a.Uout = st[s].out;
    a.a_n = st[s].an;
    a.a_s = st[s].as;
    a.alpha_in = c.slot(*k);
    a.alpha_out = (s < 2 || last_alpha) ? c.slot(*k + 1) : nullptr;
    a.alpha_zero = c.slot(*k + 2);
    cudaError_t e = weno::launch_stage(a, c.s);
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
    *k += 1;
  }
  return WENO_OK;
}

weno_status read_status(const Ctx &c) {
  DevStatus h;
  cudaError_t e = cudaMemcpyAsync(&h, c.status(), sizeof(h), cudaMemcpyDeviceToHost, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync status");
  e = cudaStreamSynchronize(c.s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (h.code == 5) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "a tile's shared-memory copy did not complete (problem %lld, "
                  "tile at j=%lld, i=%lld)", h.b, h.j, h.i);
    return fail(WENO_ERR_TIMEOUT, buf);
  }
  if (h.code != 0) {
    static const char *where[] = {"wavespeeds", "stage 1", "stage 2", "stage 3", "rhs"};
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "nonphysical state (rho <= 0, p <= 0, c^2 <= 0 or non-finite) in %s, "
                  "problem %lld, cell (j=%lld, i=%lld)",
                  where[(h.stage >= 0 && h.stage <= 4) ? h.stage : 0], h.b, h.j, h.i);
    return fail(WENO_ERR_NONPHYSICAL, buf);
  }
  return WENO_OK;
}

// ---------------------------------------------------------------------------
// Tile autotuner for the 2D stage kernel.  The first call on a new problem
// shape times every tile variant on the caller's data (one right-hand-side
// stage each, written into the scratch state U1) and caches the fastest; all
// variants compute bitwise the same result.  WENO_TILE2D=0|1|2 in the
// environment forces a variant and skips the timing.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::tuple<long long, long long, long long, int, int, int>, int> g_tune;

int tile_override() {
  const char *v = std::getenv("WENO_TILE2D");
  if (!v || !*v) return -1;
  const int t = std::atoi(v);
  return (t >= 0 && t < weno::kTileVariants) ? t : -1;
}

weno_status choose_tile(const Ctx &c, const double *U, const unsigned long long *alpha, int *out) {
  *out = 0;
  const weno_desc *d = c.d;
  if (d->ndim != 2 || (d->order != 0 && d->order != 6)) return WENO_OK;  // one tile shape
  const int forced = tile_override();
  if (forced >= 0) {
    *out = forced;
    return WENO_OK;
  }
  const auto key = std::make_tuple((long long)d->nx, (long long)d->ny, (long long)d->nbatch,
                                   (int)d->precision, (int)d->ai, (int)(d->p == 1.0));
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *out = it->second;
      return WENO_OK;
    }
  }
  StageArgs a = stage_args(c);
  a.mode = 1;
  a.stage = 4;
  a.Uin = U;
  a.Uout = c.u1();
  a.alpha_in = alpha;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fail(WENO_ERR_CUDA, "cudaEventCreate");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(WENO_ERR_CUDA, "cudaEventCreate");
  }
  int best = 0;
  float best_ms = 0.0f;
  weno_status st = WENO_OK;
  for (int v = 0; v < weno::kTileVariants && st == WENO_OK; ++v) {
    a.tile_variant = v;
    cudaError_t e = weno::launch_stage(a, c.s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, c.s);
    if (e == cudaSuccess) e = weno::launch_stage(a, c.s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c.s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "tile autotuner");
      break;
    }
    if (v == 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WENO_OK) return st;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  *out = best;
  return WENO_OK;
}

weno_status prepare(const weno_desc *d, void *ws, size_t ws_bytes, void *stream, bool host,
                    Ctx *c) {
  weno_status st = check_desc(d);
  if (st != WENO_OK) return st;
  c->d = d;
  c->L = layout(d);
  st = check_ws(d, ws, ws_bytes, host ? c->L.total_host : c->L.total);
  if (st != WENO_OK) return st;
  c->ws = (char *)ws;
  c->s = (cudaStream_t)stream;
  g_err.clear();
  return WENO_OK;
}

}  // namespace

void weno::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

// Where the Buckley-Leverett speed f'(u) = u(1-u) / (2 D^2), D = u^2 +
// (1-u)^2 / 4, peaks on [0, 1]: the root of its derivative, i.e. of
// (1 - 2u) D = 2 u (1 - u) D', D' = 2u - (1 - u)/2, found by bisection (the
// left side minus the right side changes sign once on (0, 1)).
double weno::bl_speed_argmax() {
  auto h = [](double u) {
    const double D = u * u + 0.25 * (1.0 - u) * (1.0 - u);
    const double Dp = 2.0 * u - 0.5 * (1.0 - u);
    return (1.0 - 2.0 * u) * D - 2.0 * u * (1.0 - u) * Dp;
  };
  double lo = 0.0, hi = 1.0;  // h(0) = 0.25 > 0, h(1) = -1 < 0
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (h(mid) > 0.0)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

extern "C" {

size_t weno_workspace_bytes(const weno_desc *d) {
  if (check_desc(d) != WENO_OK) return 0;
  return layout(d).total;
}

size_t weno_workspace_bytes_host(const weno_desc *d) {
  if (check_desc(d) != WENO_OK) return 0;
  return layout(d).total_host;
}

const char *weno_last_error(void) { return g_err.c_str(); }

const char *weno_version(void) { return "weno-za6-gb300 0.1 (sm_103a)"; }

weno_status weno_wavespeeds(const weno_desc *d, const double *U, double *alpha, double *dt,
                            void *ws, size_t ws_bytes, void *stream) {
  Ctx c;
  weno_status st = prepare(d, ws, ws_bytes, stream, false, &c);
  if (st != WENO_OK) return st;
  if (!U || (!alpha && !dt)) return fail(WENO_ERR_ARG, "NULL array");
  if ((st = reset_control(c, 0.0)) != WENO_OK) return st;
  AlphaArgs a = alpha_args(c, U, c.slot(0));
  cudaError_t e = weno::launch_alpha(a, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "alpha launch");
  e = weno::launch_alpha_export(a, c.slot(0), alpha, dt, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "alpha export launch");
  return WENO_OK;
}

weno_status weno_rhs(const weno_desc *d, const double *U, double *dUdt, void *ws,
                     size_t ws_bytes, void *stream) {
  Ctx c;
  weno_status st = prepare(d, ws, ws_bytes, stream, false, &c);
  if (st != WENO_OK) return st;
  if (!U || !dUdt) return fail(WENO_ERR_ARG, "NULL array");
  if (U == dUdt) return fail(WENO_ERR_ARG, "dUdt must not overlap U");
  if ((st = reset_control(c, 0.0)) != WENO_OK) return st;
  cudaError_t e = weno::launch_alpha(alpha_args(c, U, c.slot(0)), c.s);
  if (e != cudaSuccess) return cuda_fail(e, "alpha launch");
  int tile = 0;
  if ((st = choose_tile(c, U, c.slot(0), &tile)) != WENO_OK) return st;
  StageArgs a = stage_args(c);
  a.tile_variant = tile;
  a.mode = 1;
  a.stage = 4;
  a.Uin = U;
  a.Uout = dUdt;
  a.alpha_in = c.slot(0);
  e = weno::launch_stage(a, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "rhs launch");
  return WENO_OK;
}

weno_status weno_step(const weno_desc *d, double *U, double dt, double *dt_used, void *ws,
                      size_t ws_bytes, void *stream) {
  Ctx c;
  weno_status st = prepare(d, ws, ws_bytes, stream, false, &c);
  if (st != WENO_OK) return st;
  if (!U) return fail(WENO_ERR_ARG, "NULL state");
  if (!std::isfinite(dt)) return fail(WENO_ERR_ARG, "dt must be finite");
  if ((st = reset_control(c, 0.0)) != WENO_OK) return st;
  cudaError_t e = weno::launch_alpha(alpha_args(c, U, c.slot(0)), c.s);
  if (e != cudaSuccess) return cuda_fail(e, "alpha launch");
  int tile = 0;
  if ((st = choose_tile(c, U, c.slot(0), &tile)) != WENO_OK) return st;
  int k = 0;
  if ((st = launch_step(c, U, dt > 0.0 ? dt : 0.0, INFINITY, &k, false, tile)) != WENO_OK) return st;
  if (dt_used) {
    e = cudaMemcpyAsync(dt_used, c.dt(), sizeof(double) * d->nbatch, cudaMemcpyDeviceToHost, c.s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync dt");
    return read_status(c);
  }
  return WENO_OK;
}

weno_status weno_solve(const weno_desc *d, double *U, double t0, double t_final,
                       int64_t max_steps, double *t_out, int64_t *steps_out, void *ws,
                       size_t ws_bytes, void *stream) {
  Ctx c;
  weno_status st = prepare(d, ws, ws_bytes, stream, false, &c);
  if (st != WENO_OK) return st;
  if (!U) return fail(WENO_ERR_ARG, "NULL state");
  if (!std::isfinite(t0) || !std::isfinite(t_final)) return fail(WENO_ERR_ARG, "t0, t_final must be finite");
  if (max_steps < 0) return fail(WENO_ERR_ARG, "max_steps must be >= 0");
  if ((st = reset_control(c, t0)) != WENO_OK) return st;
  cudaError_t e = weno::launch_alpha(alpha_args(c, U, c.slot(0)), c.s);
  if (e != cudaSuccess) return cuda_fail(e, "alpha launch");
  const long long nb = d->nbatch;
  std::vector<double> th(nb, t0);
  // Steps are launched in chunks; the host reads the clocks and the status
  // between chunks.  Launches past a problem's t_final exit at once.
  const double cells = (double)nb * d->nx * d->ny;
  const int64_t chunk = cells >= 1e6 ? 4 : (cells >= 1e5 ? 16 : 64);
  int tile = 0;
  if ((st = choose_tile(c, U, c.slot(0), &tile)) != WENO_OK) return st;
  int64_t n = 0;
  int k = 0;
  bool done = !(t_final > t0);
  while (!done && n < max_steps) {
    const int64_t m = (max_steps - n < chunk) ? (max_steps - n) : chunk;
    for (int64_t q = 0; q < m; ++q)
      if ((st = launch_step(c, U, 0.0, t_final, &k, true, tile)) != WENO_OK) return st;
    n += m;
    e = cudaMemcpyAsync(th.data(), c.t(), sizeof(double) * nb, cudaMemcpyDeviceToHost, c.s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync t");
    if ((st = read_status(c)) != WENO_OK) break;
    done = true;
    for (long long b = 0; b < nb; ++b)
      if (th[b] < t_final) done = false;
  }
  std::vector<long long> sh(nb, 0);
  e = cudaMemcpyAsync(sh.data(), c.steps(), sizeof(long long) * nb, cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(th.data(), c.t(), sizeof(double) * nb, cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  if (e != cudaSuccess) return cuda_fail(e, "reading clocks");
  for (long long b = 0; b < nb; ++b) {
    if (t_out) t_out[b] = th[b];
    if (steps_out) steps_out[b] = sh[b];
  }
  if (st != WENO_OK) return st;
  if (!done) return fail(WENO_ERR_MAXSTEPS, "max_steps reached before t_final");
  return WENO_OK;
}

weno_status weno_solve_host(const weno_desc *d, double *U_host, double t0, double t_final,
                            int64_t max_steps, double *t_out, int64_t *steps_out, void *ws,
                            size_t ws_bytes, void *stream) {
  Ctx c;
  weno_status st = prepare(d, ws, ws_bytes, stream, true, &c);
  if (st != WENO_OK) return st;
  if (!U_host) return fail(WENO_ERR_ARG, "NULL state");
  double *Ud = (double *)(c.ws + c.L.uhost);
  cudaError_t e = cudaMemcpyAsync(Ud, U_host, c.L.state_bytes, cudaMemcpyHostToDevice, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
  st = weno_solve(d, Ud, t0, t_final, max_steps, t_out, steps_out, ws, ws_bytes, stream);
  if (st != WENO_OK && st != WENO_ERR_MAXSTEPS && st != WENO_ERR_NONPHYSICAL) return st;
  const std::string keep = g_err;
  e = cudaMemcpyAsync(U_host, Ud, c.L.state_bytes, cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
  g_err = keep;
  return st;
}

weno_status weno_step_host(const weno_desc *d, double *U_host, double dt, double *dt_used,
                           void *ws, size_t ws_bytes, void *stream) {
  Ctx c;
  weno_status st = prepare(d, ws, ws_bytes, stream, true, &c);
  if (st != WENO_OK) return st;
  if (!U_host) return fail(WENO_ERR_ARG, "NULL state");
  double *Ud = (double *)(c.ws + c.L.uhost);
  cudaError_t e = cudaMemcpyAsync(Ud, U_host, c.L.state_bytes, cudaMemcpyHostToDevice, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
  std::vector<double> used(d->nbatch);
  st = weno_step(d, Ud, dt, used.data(), ws, ws_bytes, stream);
  if (st != WENO_OK && st != WENO_ERR_NONPHYSICAL) return st;
  const std::string keep = g_err;
  e = cudaMemcpyAsync(U_host, Ud, c.L.state_bytes, cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
  if (dt_used)
    for (long long b = 0; b < d->nbatch; ++b) dt_used[b] = used[b];
  g_err = keep;
  return st;
}

weno_status weno_sync_status(const weno_desc *d, void *ws, size_t ws_bytes, void *stream) {
  Ctx c;
  weno_status st = prepare(d, ws, ws_bytes, stream, false, &c);
  if (st != WENO_OK) return st;
  return read_status(c);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Domain decomposition in y: one strip of rows of a 2D grid per process.
// The global descriptor fixes dx, dy, the boundary conditions and the scheme;
// the strip holds nrows rows.  Per Runge-Kutta stage the caller max-reduces
// the strips' speed maxima (eq. (6) takes its maximum over the whole grid)
// and exchanges r rows with the neighbouring strips; everything else is the
// single-grid stage kernel, so a split solve gives bitwise the single-grid
// result.
// ---------------------------------------------------------------------------
namespace {

weno_status dd_prepare(const weno_desc *g, int64_t nrows, void *ws, size_t ws_bytes, void *stream,
                       weno_desc *local, Ctx *c) {
  weno_status st = check_desc(g);
  if (st != WENO_OK) return st;
  if (g->ndim != 2 || g->system != WENO_SYS_EULER)
    return fail(WENO_ERR_ARG, "domain decomposition is for 2D Euler");
  const int r = g->order == 0 ? 3 : g->order / 2;
  if (nrows < r || nrows > g->ny)
    return fail(WENO_ERR_ARG, "nrows must be at least r = " + std::to_string(r) +
                                  " (the rows a neighbour needs) and at most ny");
  *local = *g;
  local->ny = nrows;
  return prepare(local, ws, ws_bytes, stream, false, c);
}

int order_r_of(const weno_desc *d) { return d->order == 0 ? 3 : d->order / 2; }

}  // namespace

extern "C" {

weno_status weno_dd_begin(const weno_desc *d, int64_t nrows, const double *U, double *send_lo,
                          double *send_hi, void *ws, size_t ws_bytes, void *stream) {
  weno_desc local;
  Ctx c;
  weno_status st = dd_prepare(d, nrows, ws, ws_bytes, stream, &local, &c);
  if (st != WENO_OK) return st;
  if (!U) return fail(WENO_ERR_ARG, "NULL state");
  if ((st = reset_control(c, 0.0)) != WENO_OK) return st;
  AlphaArgs a = alpha_args(c, U, c.slot(0));
  a.dy = (d->y1 - d->y0) / (double)d->ny;
  cudaError_t e = weno::launch_alpha(a, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "alpha launch");
  const int r = order_r_of(d);
  if (send_lo) e = weno::launch_pack_rows(U, d->nbatch, 4, nrows, d->nx, 0, r, send_lo, c.s);
  if (e == cudaSuccess && send_hi)
    e = weno::launch_pack_rows(U, d->nbatch, 4, nrows, d->nx, nrows - r, r, send_hi, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "row pack launch");
  return WENO_OK;
}

weno_status weno_dd_speeds(const weno_desc *d, int64_t nrows, int stage, void *ws, size_t ws_bytes,
                           uint64_t **speeds) {
  weno_desc local;
  Ctx c;
  weno_status st = dd_prepare(d, nrows, ws, ws_bytes, nullptr, &local, &c);
  if (st != WENO_OK) return st;
  if (stage < 1 || stage > 3) return fail(WENO_ERR_ARG, "stage must be 1, 2 or 3");
  if (!speeds) return fail(WENO_ERR_ARG, "NULL output");
  *speeds = (uint64_t *)c.slot(stage - 1);
  return WENO_OK;
}

weno_status weno_dd_stage(const weno_desc *d, int64_t nrows, int stage, double *U, double dt,
                          const double *halo_lo, const double *halo_hi, double *send_lo,
                          double *send_hi, void *ws, size_t ws_bytes, void *stream) {
  weno_desc local;
  Ctx c;
  weno_status st = dd_prepare(d, nrows, ws, ws_bytes, stream, &local, &c);
  if (st != WENO_OK) return st;
  if (stage < 1 || stage > 3) return fail(WENO_ERR_ARG, "stage must be 1, 2 or 3");
  if (!U) return fail(WENO_ERR_ARG, "NULL state");
  if (!std::isfinite(dt)) return fail(WENO_ERR_ARG, "dt must be finite");
  StageArgs a = stage_args(c);
  a.dy = (d->y1 - d->y0) / (double)d->ny;
  const int forced = tile_override();
  a.tile_variant = forced >= 0 ? forced : 3;  // every variant gives the same bits
  a.mode = 0;
  a.stage = stage;
  a.dt_fixed = dt > 0.0 ? dt : 0.0;
  a.t_final = INFINITY;
  if (stage == 1) {
    a.Uin = U; a.Un = nullptr; a.Uout = c.u1(); a.a_n = 0.0; a.a_s = 1.0;
  } else if (stage == 2) {
    a.Uin = c.u1(); a.Un = U; a.Uout = c.u2(); a.a_n = 0.75; a.a_s = 0.25;
  } else {
    a.Uin = c.u2(); a.Un = U; a.Uout = U; a.a_n = 1.0 / 3.0; a.a_s = 2.0 / 3.0;
  }
  a.alpha_in = c.slot(stage - 1);
  a.alpha_out = stage < 3 ? c.slot(stage) : nullptr;
  a.alpha_zero = c.slot(stage + 1);
  a.halo_lo = halo_lo;
  a.halo_hi = halo_hi;
  a.send_lo = send_lo;
  a.send_hi = send_hi;
  cudaError_t e = weno::launch_stage(a, c.s);
  if (e != cudaSuccess) return cuda_fail(e, "stage launch");
  return WENO_OK;
}

}  // extern "C"
