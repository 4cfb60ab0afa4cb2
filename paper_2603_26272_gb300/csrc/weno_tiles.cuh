// weno_tiles.cuh -- the stage kernels of the central-upwind WENO right-hand
// side and the SSP-RK3 stage update for GB300 (sm_103a), templated on the
// stencil half-width r (scheme of order 2r; r = 3 is WENO-ZA6 of Section 3,
// r = 2, 4, 5 the schemes of the Appendix).  Included by weno_kernels.cu
// (r = 3) and weno_orders.cu (r = 2, 4, 5); everything here has internal
// linkage in each translation unit.
//
// One launch = one Runge-Kutta stage over every problem of the batch
// (Section 4 preamble: third-order TVD Runge-Kutta).  A block owns a tile of
// cells and runs three phases:
//   1. stage the tile and its r-cell halo (the 2r-point stencil of eq. (7))
//      into shared memory, with ghost cells by index clamp or wrap, and form
//      per-cell primitives and physical fluxes once;
//   2. compute every interface flux of the tile exactly once -- in 2D the x-
//      and y-faces of one tile come from the same staged data (dimension by
//      dimension, Section 4.3) -- by characteristic-wise global
//      Lax-Friedrichs splitting (eq. (6), Section 4.2) and the central-upwind
//      WENO flux (Sections 2-3) for the positive and the mirrored negative
//      flux;
//   3. per cell, the conservative difference of eq. (5), the Runge-Kutta
//      combination, and -- for the next stage -- the block's maxima of the
//      characteristic speeds, reduced with warp shuffles and one atomicMax
//      per value and block.
#pragma once
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include <cuda.h>  // CUtensorMap (the type only; the encoder is fetched at run time)

#include "weno_device.cuh"
#include "weno_internal.h"

namespace weno {
namespace {

constexpr int kThreads2D = 256;
constexpr int kTX = 32, kTY = 16;
constexpr int kThreads1D = 128;
constexpr int kT1 = kThreads1D - 1;  // cells per 1D tile: one face per thread

__device__ __forceinline__ long long ghost(long long k, long long n, int bc) {
  if (bc == 1) {
    long long m = k % n;
    return m < 0 ? m + n : m;
  }
  return k < 0 ? 0 : (k >= n ? n - 1 : k);
}

__device__ __forceinline__ double bits2d(unsigned long long u) {
  return __longlong_as_double((long long)u);
}

__device__ void record_status(DevStatus *st, int code, int stage, long long b, long long j,
                              long long i) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->stage = stage;
    st->b = b;
    st->j = j;
    st->i = i;
  }
}

// CFL step of problem b from its speed maxima (bit patterns), the rule of
// the oracle: 1D cfl dx / max(|u|+c); 2D cfl / (max(|u|+c)/dx + max(|v|+c)/dy).
// max(|u-c|, |u+c|) = |u| + c exactly (same rounding).
// Scalar systems 2, 3 keep okey(max u) and okey(max -u) in slots 0 and 1.
__device__ __forceinline__ double scalar_alpha_of(int system, double adv, double ustar,
                                                  const unsigned long long *al) {
  if (system == 0) return fabs(adv);
  const double umax = okey_inv(al[0]), umin = -okey_inv(al[1]);
  return scalar_alpha(system, adv, umin, umax, ustar);
}

__device__ double cfl_dt(int system, int ndim, int nc, double cfl, double dx, double dy,
                         double adv, const unsigned long long *al, double ustar = 0.0) {
  if (system == 0) return cfl * dx / fabs(adv);
  if (system >= 2) return cfl * dx / scalar_alpha_of(system, adv, ustar, al);
  const unsigned long long sxb = max(al[0], al[nc == 3 ? 2 : 3]);
  const double sx = bits2d(sxb);
  if (ndim == 1) return cfl * dx / sx;
  const double sy = bits2d(max(al[4], al[7]));
  return cfl / (sx / dx + sy / dy);
}

// Block-level control shared by every stage kernel: clears the slot of the
// stage after next, decides this problem's dt, advances its clock.
// Returns false if the block has nothing to do.
__device__ bool stage_control(const StageArgs &a, long long b, bool first_block_of_b,
                              bool zeroing_block, double &dt_out) {
  __shared__ double s_dt;
  __shared__ int s_go;
  if (a.alpha_zero && zeroing_block)
    for (long long k = threadIdx.x; k < a.nbatch * 8; k += blockDim.x) a.alpha_zero[k] = 0ull;
  if (threadIdx.x == 0) {
    int go = 1;
    double dt = 0.0;
    if (*(volatile int *)&a.status->code != 0) {
      go = 0;
    } else if (a.mode == 0) {
      if (a.stage == 1) {
        const double t = a.t[b];
        if (!(t < a.t_final)) {
          go = 0;
          if (first_block_of_b) a.dt[b] = 0.0;
        } else {
          dt = a.dt_fixed > 0.0 ? a.dt_fixed
                                : cfl_dt(a.system, a.ndim, a.nc, a.cfl, a.dx, a.dy,
                                         a.adv_speed, a.alpha_in + b * 8, a.ustar);
          const double rem = a.t_final - t;
          const bool last = !(dt < rem);
          if (last) dt = rem;
          if (first_block_of_b) {
            a.dt[b] = dt;
            a.tnext[b] = last ? a.t_final : t + dt;
          }
        }
      } else {
        dt = a.dt[b];
        if (dt == 0.0) go = 0;
        if (go && a.stage == 3 && first_block_of_b) {
          a.t[b] = a.tnext[b];
          a.steps[b] += 1;
        }
      }
    }
    s_dt = dt;
    s_go = go;
  }
  __syncthreads();
  dt_out = s_dt;
  return s_go != 0;
}

// Per-field reconstruction parameters; field m arrives scaled by k[m].
__device__ __forceinline__ ReconParams make_rp(const StageArgs &a, double k) {
  ReconParams r;
  r.eps4 = 4.0 * a.eps;
  r.mu0s = k * a.mu0;
  r.efix = 4.0 * a.eps * k * k;
  r.p = a.p;
  const double se = sqrt(4.0 * a.eps);
  r.me = se * (1.0 / 6.0);
  r.mo = se * (k * a.mu0);
  r.e0 = r.mo * r.mo;
  // me^2 = eps / 9 as an FP32 mantissa and an exponent (eps / 9 is a normal
  // double for every eps the boundary accepts with Ai)
  const double me2 = a.eps * (1.0 / 9.0);
  const int hi = __double2hiint(me2);
  r.eme = ((hi >> 20) & 0x7FF) - 1023;
  r.mef = __uint_as_float(0x3F800000u |
                          (__funnelshift_r((unsigned)__double2loint(me2), (unsigned)hi, 29) & 0x7FFFFFu));
  // dev >= 2^(lthr - 1019) implies dev / 6 >= 2^30 scale mu_0: with
  // 6 scale mu_0 < 2^(E + 1), E its exponent, lthr = 1019 + E + 1 + 30
  if (a.mu0 > 0.0) {
    const double m6 = 6.0 * k * a.mu0;
    r.lthr = 1019 + (((__double2hiint(m6) >> 20) & 0x7FF) - 1023) + 31;
  } else {
    r.lthr = -(1 << 20);
  }
  return r;
}

__device__ __forceinline__ Recon32 make_r32(const StageArgs &a) {
  Recon32 r;
  r.eps4 = 4.0e-30f;
  r.p = (float)a.p;
  return r;
}

// Block reduction of NV maxima (bit patterns) and one atomicMax per value into
// dst[slot[q]], and also into dst[dup[q]] where dup[q] >= 0 (the entropy and
// shear fields share the speed |u|).
template <int NV>
__device__ void block_max_atomic(unsigned long long (&v)[NV], unsigned long long *dst,
                                 const int (&slot)[NV], const int (&dup)[NV]) {
  __shared__ unsigned long long red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] = max(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[warp][q] = v[q];
  __syncthreads();
  if (threadIdx.x < NV) {
    unsigned long long m = 0;
    for (int w = 0; w < nw; ++w) m = max(m, red[w][threadIdx.x]);
    atomicMax(dst + slot[threadIdx.x], m);
    if (dup[threadIdx.x] >= 0) atomicMax(dst + dup[threadIdx.x], m);
  }
}

// ---------------------------------------------------------------------------
// Tensor-memory-accelerator (TMA) staging of a 2D tile: one bulk tensor copy
// brings the conserved variables of the tile and its halo -- a box of
// (TX + 2 XO) x (TY + 2 R) cells of all four planes of the problem -- from
// global into shared memory, completing on an mbarrier.  XO is R rounded up
// to even, so the box starts at x = i0 - XO, a multiple of 2 doubles: the
// 16-byte alignment a tiled copy needs for its innermost coordinate.  Only
// interior tiles (the whole box inside the grid) use it; tiles that need
// ghost cells (clamp, wrap, halo rows) load with plain indexed loads.
// ---------------------------------------------------------------------------
template <int R> struct TmaBox {
  static constexpr int XO = (R + 1) & ~1;
};

template <int TX, int TY, int R>
__host__ __device__ constexpr size_t tma_box_bytes() {
  return sizeof(double) * 4 * (TX + 2 * TmaBox<R>::XO) * (TY + 2 * R);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Issue the copy (thread 0 only): barrier armed with the byte count first.
__device__ __forceinline__ void tma_issue_box(const CUtensorMap *tm, unsigned bar, void *dst,
                                              int x, int y, int z, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// SM clock cycles a TMA wait may take before it gives up (about 1 ms at
// 2 GHz; the copy of one box takes microseconds).
constexpr long long kTmaWaitCycles = 2000000;

// The TMA copy of tile (i0, j0)'s box of problem b into `box` (every thread
// of the block calls this).  Returns false -- after recording
// WENO_ERR_TIMEOUT and a second bounded wait for the copy in flight, which
// writes into this block's shared memory -- when the copy did not complete
// in time; the tile is then left undone.
template <int TX, int TY, int R>
__device__ bool tma_stage_box(const StageArgs &a, const CUtensorMap *tm, double *box, long long b,
                              long long i0, long long j0) {
  __shared__ __align__(8) unsigned long long s_bar;
  const unsigned bar = smem_u32(&s_bar);
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    if (a.tma_no_copy)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                   "r"((unsigned)tma_box_bytes<TX, TY, R>())
                   : "memory");
    else
      tma_issue_box(tm, bar, box, (int)(i0 - TmaBox<R>::XO), (int)(j0 - R), (int)(b * 4),
                    (unsigned)tma_box_bytes<TX, TY, R>());
  }
  long long t_start = clock64();
  bool done = false;
  while (!(done = mbar_try_wait(bar, 0)) && clock64() - t_start < kTmaWaitCycles) {
  }
  if (!__syncthreads_and(done)) {
    if (tid == 0) record_status(a.status, 5, a.stage, b, j0, i0);
    t_start = clock64();
    while (!mbar_try_wait(bar, 0) && clock64() - t_start < kTmaWaitCycles) {
    }
    return false;
  }
  return true;
}

// Where staged cell (r, c) of tile (i0, j0) -- r in [0, TY + 2R), c in
// [0, TX + 2R), the tile's cells at [R, R + TY) x [R, R + TX) -- is read from
// without TMA: the array src with plane stride pst and offset o (the stage
// input, or a neighbour's halo rows of a domain split), after the ghost rule
// of each boundary; (gj, gi) is the cell reported on error.
__device__ __forceinline__ void cell_source(const StageArgs &a, const double *Ub, long long b,
                                            long long i0, long long j0, int R, int r, int c,
                                            const double *&src, long long &o, long long &pst,
                                            long long &gj, long long &gi) {
  gi = ghost(i0 - R + c, a.nx, a.bc_x);
  const long long jj = j0 - R + r;
  src = Ub;
  pst = a.nx * a.ny;
  gj = jj;
  if (jj < 0 && a.halo_lo) {  // a neighbour's rows below this strip
    src = a.halo_lo + b * 4 * (R * a.nx);
    o = (jj + R) * a.nx + gi;
    pst = R * a.nx;
  } else if (jj >= a.ny && a.halo_hi) {  // above it (rows beyond ny+R-1 only
    src = a.halo_hi + b * 4 * (R * a.nx);  // fill a partial tile: any halo row)
    o = min(jj - a.ny, (long long)(R - 1)) * a.nx + gi;
    pst = R * a.nx;
  } else {
    gj = ghost(jj, a.ny, a.bc_y);
    o = gj * a.nx + gi;
  }
}

// Phase 3 of a 2D tile: per cell the conservative difference of eq. (5)
// from the faces' 4 F (backproject4, so idx = 0.25 / dx, idy = 0.25 / dy), the
// Runge-Kutta combination with the staged input u_at(r, c, q) of tile cell
// (r, c), the strips' send rows, and the next stage's speed maxima.
template <int TX, int TY, int R, class UAt>
__device__ __forceinline__ void tile2d_update(const StageArgs &a, long long b, long long i0,
                                              long long j0, double dt, const double *fx,
                                              const double *fy, double idx, double idy,
                                              UAt u_at) {
  const long long plane = a.nx * a.ny;
  const double gm1 = a.gamma - 1.0;
  const int tid = threadIdx.x;
  unsigned long long mx6[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  const bool want_alpha = (a.mode == 0) && (a.alpha_out != nullptr);
  for (int k = tid; k < TX * TY; k += blockDim.x) {
    const int r = k / TX, c = k - r * TX;
    const long long gi = i0 + c, gj = j0 + r;
    if (gi >= a.nx || gj >= a.ny) continue;
    const double *Fl = &fx[(r * (TX + 1) + c) * 4];
    const double *Fr = Fl + 4;
    const double *Gb = &fy[(r * TX + c) * 4];
    const double *Gt = &fy[((r + 1) * TX + c) * 4];
    const long long o = b * 4 * plane + gj * a.nx + gi;
    double uo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double L = -(Fr[q] - Fl[q]) * idx - (Gt[q] - Gb[q]) * idy;
      if (a.mode == 1) {
        uo[q] = L;
      } else {
        const double base_s = fma(dt, L, u_at(r, c, q));
        uo[q] = (a.a_n != 0.0) ? fma(a.a_n, a.Un[o + q * plane], a.a_s * base_s) : a.a_s * base_s;
      }
      a.Uout[o + q * plane] = uo[q];
    }
    if (a.send_lo && gj < R)  // edge rows of the output for the strips below / above
#pragma unroll
      for (int q = 0; q < 4; ++q) a.send_lo[((b * 4 + q) * R + gj) * a.nx + gi] = uo[q];
    if (a.send_hi && gj >= a.ny - R)
#pragma unroll
      for (int q = 0; q < 4; ++q) a.send_hi[((b * 4 + q) * R + (gj - (a.ny - R))) * a.nx + gi] = uo[q];
    if (want_alpha) {
      const double ir = rcp_pos(uo[0]);
      const double u = uo[1] * ir, v = uo[2] * ir;
      const double p = gm1 * (uo[3] - 0.5 * fma(uo[1], u, uo[2] * v));
      if (!(pos_finite(uo[0]) && pos_finite(p))) record_status(a.status, 3, a.stage, b, gj, gi);
      const double cs = sqrt_pos(a.gamma * p * ir);
      mx6[0] = max(mx6[0], abs_bits(u - cs));
      mx6[1] = max(mx6[1], abs_bits(u));
      mx6[2] = max(mx6[2], abs_bits(u + cs));
      mx6[3] = max(mx6[3], abs_bits(v - cs));
      mx6[4] = max(mx6[4], abs_bits(v));
      mx6[5] = max(mx6[5], abs_bits(v + cs));
    }
  }
  if (want_alpha) {
    const int slot[6] = {0, 1, 3, 4, 5, 7};
    const int dup[6] = {-1, 2, -1, -1, 6, -1};
    block_max_atomic<6>(mx6, a.alpha_out + b * 8, slot, dup);
  }
}

// ---------------------------------------------------------------------------
// 2D Euler stage kernel of the orders 4, 8, 10 (R = 2, 4, 5).
// Shared planes per staged cell: 0 rho, 1 rho u, 2 rho v, 3 E, 4 u, 5 v, 6 H,
// 7 sqrt(rho), 8 p (the fluxes are projected from u, v, p: project_flux4).
// ---------------------------------------------------------------------------
constexpr int kPlanes2D = 9;

template <int TX, int TY, int R>
__host__ __device__ constexpr size_t smem_euler2d_gen() {
  return sizeof(double) *
         (kPlanes2D * (TX + 2 * R) * (TY + 2 * R) + 4 * ((TX + 1) * TY + TX * (TY + 1)));
}

// Layout of the sixth-order tile (euler2d_tile6), in doubles, after the
// 128-byte aligned start: box, Roe planes, cell-pair differences, faces.
template <int TX, int TY> struct Tile6 {
  static constexpr int R = 3, XO = TmaBox<3>::XO;
  static constexpr int W = TX + 2 * R, HH = TY + 2 * R, BW = TX + 2 * XO, REG = W * HH;
  static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
  static constexpr int NPX = TY * (W - 1), NPY = TX * (HH - 1);  // cell pairs of each sweep
  static constexpr int ND = NPX > NPY ? NPX : NPY;
  static constexpr int PB = HH * BW;  // plane stride of the box
  static constexpr int kBox = 0, kPl = kBox + 4 * PB, kDd = kPl + 4 * REG, kFx = kDd + 7 * ND,
                       kFy = kFx + 4 * NFX, kEnd = kFy + 4 * NFY;
  static constexpr size_t kBytes = sizeof(double) * kEnd + 128;
};

// Dynamic shared memory of one 2D tile.
template <int TX, int TY, int R = 3>
__host__ __device__ constexpr size_t smem_euler2d() {
  return R == 3 ? Tile6<TX, TY>::kBytes : smem_euler2d_gen<TX, TY, R>();
}

// The same for a tile that may stage by TMA (orders 4, 8, 10: the planes and
// faces, then the box, 128-byte aligned; the sixth-order layout always
// holds the box).
template <int TX, int TY, int R = 3>
__host__ __device__ constexpr size_t smem_euler2d_tma() {
  return R == 3 ? Tile6<TX, TY>::kBytes
                : ((smem_euler2d_gen<TX, TY, R>() + 127) & ~size_t(127)) +
                      tma_box_bytes<TX, TY, R>() + 128;
}

// One tile (tile index `tile` of problem b) of a 2D stage, run by one block.
// R: half-width of the stencil (scheme of order 2R, halo of R cells).
// sm: dynamic shared memory of smem_euler2d_tma<TX, TY, R>() bytes.
// tm: tensor map of the stage input as [nbatch * 4][ny][nx] doubles, or NULL
// (plain loads only; the serving engine and tiles of launches without one).
template <int TX, int TY, bool AI, bool P1, int PREC, int R>
__device__ __forceinline__ void euler2d_tile_gen(const StageArgs &a, long long b, long long tile,
                                                 bool zeroing_block, double *sm,
                                                 const CUtensorMap *tm) {
  static_assert(R != 3 && PREC == 0, "orders 4, 8, 10 in FP64");
  constexpr int W = TX + 2 * R, HH = TY + 2 * R, REG = W * HH;
  constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1);
  constexpr int XO = TmaBox<R>::XO, BW = TX + 2 * XO;
  double *const pl = sm;
  double *const fx = sm + kPlanes2D * REG;
  double *const fy = fx + NFX * 4;

  const long long tiles_x = (a.nx + TX - 1) / TX;
  const long long tj = tile / tiles_x, ti = tile - tj * tiles_x;
  const long long i0 = ti * TX, j0 = tj * TY;
  double dt;
  if (!stage_control(a, b, tile == 0, zeroing_block, dt)) return;

  const long long plane = a.nx * a.ny;
  const double *Ub = a.Uin + b * 4 * plane;
  const double gm1 = a.gamma - 1.0;
  const int tid = threadIdx.x;

  // TMA staging of an interior tile: the box of the four conserved planes
  const bool use_tma = tm != nullptr && i0 - XO >= 0 && i0 - XO + BW <= a.nx && j0 - R >= 0 &&
                       j0 + TY + R <= a.ny;
  double *const box = reinterpret_cast<double *>(
      (reinterpret_cast<uintptr_t>(sm) + ((smem_euler2d_gen<TX, TY, R>() + 127) & ~size_t(127)) +
       127) &
      ~uintptr_t(127));
  if (use_tma && !tma_stage_box<TX, TY, R>(a, tm, box, b, i0, j0)) return;

  // Phase 1: stage the cross-shaped region (tile rows with x halo, tile
  // columns with y halo) and per-cell primitives / fluxes.
  for (int k = tid; k < REG; k += blockDim.x) {
    const int r = k / W, c = k - r * W;
    const bool xb = (r >= R) && (r < R + TY), yb = (c >= R) && (c < R + TX);
    if (!(xb || yb)) continue;
    const double *src;
    long long o, pst, gj, gi;
    if (use_tma) {  // the box: x from i0 - XO, y from j0 - R, planes of problem b
      src = box;
      pst = (long long)BW * HH;
      o = (long long)r * BW + (c + XO - R);
      gi = i0 - R + c;
      gj = j0 - R + r;
    } else {
      cell_source(a, Ub, b, i0, j0, R, r, c, src, o, pst, gj, gi);
    }
    const double rho = src[o], mx = src[pst + o], my = src[2 * pst + o], E = src[3 * pst + o];
    const double rs = rsqrt_pos(rho);  // 1/sqrt(rho): gives 1/rho and sqrt(rho)
    const double ir = rs * rs;
    const double u = mx * ir, v = my * ir;
    const double p = gm1 * (E - 0.5 * fma(mx, u, my * v));
    if (!(pos_finite(rho) && pos_finite(p))) record_status(a.status, 3, a.stage, b, gj, gi);
    pl[0 * REG + k] = rho;
    pl[1 * REG + k] = mx;
    pl[2 * REG + k] = my;
    pl[3 * REG + k] = E;
    pl[4 * REG + k] = u;
    pl[5 * REG + k] = v;
    pl[6 * REG + k] = (E + p) * ir;
    pl[7 * REG + k] = rho * rs;
    pl[8 * REG + k] = p;
  }
  __syncthreads();

  // Phase 2: every x- and y-face of the tile once.  Lanes of a warp may mix
  // directions; the code path is the same (only the plane indices differ).
  const unsigned long long *al = a.alpha_in + b * 8;
  const ReconParams rp4 = make_rp(a, 4.0), rp2 = make_rp(a, 2.0);
  for (int f = tid; f < NFX + NFY; f += blockDim.x) {
    int base, stride, dir, fr, fc;
    if (f < NFX) {
      fr = f / (TX + 1);
      fc = f - fr * (TX + 1);
      base = (R + fr) * W + fc;
      stride = 1;
      dir = 0;
    } else {
      const int g = f - NFX;
      fr = g / TX;
      fc = g - fr * TX;
      base = fr * W + R + fc;
      stride = W;
      dir = 1;
    }
    const int pmn = 1 + dir, pmt = 2 - dir, pun = 4 + dir, put = 5 - dir;
    const int kL = base + (R - 1) * stride, kR = base + R * stride;
    FaceState fs;
    if (!roe_face(pl[7 * REG + kL], pl[pun * REG + kL], pl[put * REG + kL], pl[6 * REG + kL],
                  pl[7 * REG + kR], pl[pun * REG + kR], pl[put * REG + kR], pl[6 * REG + kR],
                  gm1, fs))
      record_status(a.status, 3, a.stage, b, j0 + (dir ? fr : fr), i0 + fc);
    double A1 = bits2d(al[4 * dir + 0]), A2 = bits2d(al[4 * dir + 1]);
    double A3 = bits2d(al[4 * dir + 2]), A4 = bits2d(al[4 * dir + 3]);
    if (a.alpha_single) {
      const double m = fmax(fmax(A1, A2), fmax(A3, A4));
      A1 = A2 = A3 = A4 = m;
    }
    double h1, h2, h3, h4;
    {
      // f^+ in stencil order, f^- mirrored (its upwind side is on the right).
      constexpr int N = 2 * R;
      double p1[N], p2[N], p3[N], p4[N], m1[N], m2[N], m3[N], m4[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int k = base + j * stride;
        double w1, w2, w3, w4, g1, g2, g3, g4;
        project4(fs, pl[k], pl[pmn * REG + k], pl[pmt * REG + k], pl[3 * REG + k], w1, w2, w3, w4);
        project_flux4(fs, pl[pun * REG + k], pl[8 * REG + k], w1, w2, w3, w4, g1, g2, g3, g4);
        p1[j] = fma(A1, w1, g1);
        m1[N - 1 - j] = fma(-A1, w1, g1);
        p2[j] = fma(A2, w2, g2);
        m2[N - 1 - j] = fma(-A2, w2, g2);
        p3[j] = fma(A3, w3, g3);
        m3[N - 1 - j] = fma(-A3, w3, g3);
        p4[j] = fma(A4, w4, g4);
        m4[N - 1 - j] = fma(-A4, w4, g4);
      }
      h1 = pair_flux_r<R>(za_r<R, AI, P1>(p1, rp4), za_r<R, AI, P1>(m1, rp4));
      h2 = pair_flux_r<R>(za_r<R, AI, P1>(p2, rp2), za_r<R, AI, P1>(m2, rp2));
      h3 = pair_flux_r<R>(za_r<R, AI, P1>(p3, rp2), za_r<R, AI, P1>(m3, rp2));
      h4 = pair_flux_r<R>(za_r<R, AI, P1>(p4, rp4), za_r<R, AI, P1>(m4, rp4));
    }
    double F0, F1, F2, F3;
    backproject4(fs, h1, h2, h3, h4, F0, F1, F2, F3);
    double *out = dir ? &fy[(fr * TX + fc) * 4] : &fx[(fr * (TX + 1) + fc) * 4];
    out[0] = F0;
    out[1 + dir] = F1;
    out[2 - dir] = F2;
    out[3] = F3;
  }
  __syncthreads();

  tile2d_update<TX, TY, R>(a, b, i0, j0, dt, fx, fy, 0.25 / a.dx, 0.25 / a.dy,
                           [&](int r, int c, int q) { return pl[q * REG + (R + r) * W + R + c]; });
}

// ---------------------------------------------------------------------------
// 2D Euler stage kernel of the sixth-order scheme (R = 3).
//
// The reconstruction of a face needs, per characteristic field, only the
// differences of the split fluxes f+- = g +- alpha w over its six stencil
// cells (field_flux_d), and those are L (F_{j+1} - F_j) +- alpha L (U_{j+1}
// - U_j): the face's left eigenvectors applied to differences of the state
// and of the physical flux between adjacent cells.  Those differences are
// formed once per cell pair and direction and shared by the five faces whose
// stencils hold the pair, so a face projects 10 difference vectors instead
// of 6 states and 6 fluxes and subtracts nothing per field.  The centre
// values g_i + g_{i+1} the reconstruction adds to its differences come back
// through R as the physical 2 (F_i + F_{i+1}) = 2 (2 F_i + dF) (R L = I),
// added after the back-projection.
//
// Phases: 1 stage the conserved variables (TMA or indexed loads) and the Roe
// inputs; then per direction (x, then y) 1d the cell-pair differences and
// 2d the faces; 3 the update (tile2d_update).  Shared memory: Tile6.
// ---------------------------------------------------------------------------

// Components 1..3 of the normal-frame physical flux of a cell (eq. (25)) from
// its state and the staged u_n, H: with p = rho H - E, F1 = m_n u_n + p,
// F2 = m_t u_n, F3 = H m_n (F0 = m_n).
__device__ __forceinline__ void normal_flux(double rho, double mn, double mt, double E, double un,
                                            double H, double &F1, double &F2, double &F3) {
  const double p = fma(rho, H, -E);
  F1 = fma(mn, un, p);
  F2 = mt * un;
  F3 = H * mn;
}

template <int TX, int TY, bool AI, bool P1, int PREC, int DIR>
__device__ __forceinline__ void tile6_sweep(const StageArgs &a, long long b, long long i0,
                                            long long j0, double gm1, double *sm,
                                            const ReconParams &rp2, const ReconParams &rp4) {
  using L = Tile6<TX, TY>;
  constexpr int R = 3, W = L::W, BW = L::BW, XO = L::XO, PB = L::PB, REG = L::REG, ND = L::ND;
  const double *const box = sm + L::kBox;
  const double *const pl = sm + L::kPl;
  double *const dd = sm + L::kDd;
  double *const fo = sm + (DIR ? L::kFy : L::kFx);
  const int tid = threadIdx.x;
  // box offset of staged cell (r, c)
  auto bo = [](int r, int c) { return r * BW + c + XO - R; };

  // 1d: differences of each cell pair along DIR (normal frame: m_n = rho u
  // for x, rho v for y), in dd[q * ND + pair]:
  //   x: pair (rr, pc), rr in [0, TY), pc in [0, W - 1): cells (R + rr, pc), (R + rr, pc + 1)
  //   y: pair (pr, cc), pr in [0, HH - 1), cc in [0, TX): cells (pr, R + cc), (pr + 1, R + cc)
  constexpr int NP = DIR ? L::NPY : L::NPX;
  // the x pairs run from the block's last warp down: with phase 1 and the y
  // pairs starting from warp 0, the partial rounds of the three loops fall
  // on different warps (each warp's FP64 work goes to its own sub-partition)
  const int t0 = DIR ? tid : (int)blockDim.x - 1 - tid;
  for (int k = t0; k < NP; k += blockDim.x) {
    int rA, cA, rB, cB;
    if (DIR == 0) {
      rA = R + k / (W - 1);
      cA = k - (rA - R) * (W - 1);
      rB = rA;
      cB = cA + 1;
    } else {
      rA = k / TX;
      cA = R + (k - rA * TX);
      rB = rA + 1;
      cB = cA;
    }
    const int oA = bo(rA, cA), oB = bo(rB, cB), kA = rA * W + cA, kB = rB * W + cB;
    const double rhoA = box[oA], mnA = box[(1 + DIR) * PB + oA], mtA = box[(2 - DIR) * PB + oA],
                 EA = box[3 * PB + oA];
    const double rhoB = box[oB], mnB = box[(1 + DIR) * PB + oB], mtB = box[(2 - DIR) * PB + oB],
                 EB = box[3 * PB + oB];
    double F1A, F2A, F3A, F1B, F2B, F3B;
    normal_flux(rhoA, mnA, mtA, EA, pl[(1 + DIR) * REG + kA], pl[3 * REG + kA], F1A, F2A, F3A);
    normal_flux(rhoB, mnB, mtB, EB, pl[(1 + DIR) * REG + kB], pl[3 * REG + kB], F1B, F2B, F3B);
    dd[0 * ND + k] = rhoB - rhoA;
    dd[1 * ND + k] = mnB - mnA;  // also dF0
    dd[2 * ND + k] = mtB - mtA;
    dd[3 * ND + k] = EB - EA;
    dd[4 * ND + k] = F1B - F1A;
    dd[5 * ND + k] = F2B - F2A;
    dd[6 * ND + k] = F3B - F3A;
  }
  __syncthreads();

  // 2d: the faces along DIR.  x-face (fr, fc): between cells (R + fr, R - 1 + fc)
  // and (R + fr, R + fc), stencil pairs fr (W - 1) + fc + j; y-face (fr, fc):
  // between (R - 1 + fr, R + fc) and (R + fr, R + fc), pairs (fr + j) TX + fc.
  constexpr int NF = DIR ? L::NFY : L::NFX;
  const unsigned long long *al = a.alpha_in + b * 8 + 4 * DIR;
  double A1 = bits2d(al[0]), A2 = bits2d(al[1]), A3 = bits2d(al[2]), A4 = bits2d(al[3]);
  if (a.alpha_single) {
    const double m = fmax(fmax(A1, A2), fmax(A3, A4));
    A1 = A2 = A3 = A4 = m;
  }
  const Recon32 r32 = make_r32(a);
  for (int f = tid; f < NF; f += blockDim.x) {
    int fr, fc, p0, rL, cL, rR, cR;
    constexpr int PS = DIR ? TX : 1;  // pair stride along the stencil
    if (DIR == 0) {
      fr = f / (TX + 1);
      fc = f - fr * (TX + 1);
      p0 = fr * (W - 1) + fc;
      rL = R + fr;
      cL = R - 1 + fc;
      rR = rL;
      cR = cL + 1;
    } else {
      fr = f / TX;
      fc = f - fr * TX;
      p0 = fr * TX + fc;
      rL = R - 1 + fr;
      cL = R + fc;
      rR = rL + 1;
      cR = cL;
    }
    const int kL = rL * W + cL, kR = rR * W + cR;
    FaceState fs;
    if (!roe_face(pl[kL], pl[(1 + DIR) * REG + kL], pl[(2 - DIR) * REG + kL], pl[3 * REG + kL],
                  pl[kR], pl[(1 + DIR) * REG + kR], pl[(2 - DIR) * REG + kR], pl[3 * REG + kR],
                  gm1, fs))
      record_status(a.status, 3, a.stage, b, j0 + fr, i0 + fc);
    double dw[4][5], dg[4][5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int pj = p0 + j * PS;
      const double dmn = dd[ND + pj];
      project4(fs, dd[pj], dmn, dd[2 * ND + pj], dd[3 * ND + pj], dw[0][j], dw[1][j], dw[2][j],
               dw[3][j]);
      project4(fs, dmn, dd[4 * ND + pj], dd[5 * ND + pj], dd[6 * ND + pj], dg[0][j], dg[1][j],
               dg[2][j], dg[3][j]);
    }
    double h1, h2, h3, h4;
    if constexpr (PREC == 1) {
      h1 = field_flux_f32d<P1>(dw[0], dg[0], A1, r32);
      h2 = field_flux_f32d<P1>(dw[1], dg[1], A2, r32);
      h3 = field_flux_f32d<P1>(dw[2], dg[2], A3, r32);
      h4 = field_flux_f32d<P1>(dw[3], dg[3], A4, r32);
    } else {
      h1 = field_flux_d<AI, P1>(dw[0], dg[0], A1, rp4);
      h2 = field_flux_d<AI, P1>(dw[1], dg[1], A2, rp2);
      h3 = field_flux_d<AI, P1>(dw[2], dg[2], A3, rp2);
      h4 = field_flux_d<AI, P1>(dw[3], dg[3], A4, rp4);
    }
    double F0, F1, F2, F3;
    backproject4(fs, h1, h2, h3, h4, F0, F1, F2, F3);
    // the centre values: 4 F_hat += 2 (F_L + F_R) = 4 F_L + 2 dF of the centre pair
    {
      const int oL = bo(rL, cL), pc = p0 + 2 * PS;
      const double mnL = box[(1 + DIR) * PB + oL];
      double FL1, FL2, FL3;
      normal_flux(box[oL], mnL, box[(2 - DIR) * PB + oL], box[3 * PB + oL],
                  pl[(1 + DIR) * REG + kL], pl[3 * REG + kL], FL1, FL2, FL3);
      F0 = fma(4.0, mnL, fma(2.0, dd[ND + pc], F0));
      F1 = fma(4.0, FL1, fma(2.0, dd[4 * ND + pc], F1));
      F2 = fma(4.0, FL2, fma(2.0, dd[5 * ND + pc], F2));
      F3 = fma(4.0, FL3, fma(2.0, dd[6 * ND + pc], F3));
    }
    double *out = DIR ? &fo[(fr * TX + fc) * 4] : &fo[(fr * (TX + 1) + fc) * 4];
    out[0] = F0;
    out[1 + DIR] = F1;
    out[2 - DIR] = F2;
    out[3] = F3;
  }
  __syncthreads();
}

// One tile of a sixth-order 2D stage (see above).  sm: smem_euler2d<TX, TY>()
// bytes; tm: tensor map of the stage input or NULL, as for euler2d_tile_gen.
template <int TX, int TY, bool AI, bool P1, int PREC>
__device__ __forceinline__ void euler2d_tile6(const StageArgs &a, long long b, long long tile,
                                              bool zeroing_block, double *sm_in,
                                              const CUtensorMap *tm) {
  using L = Tile6<TX, TY>;
  constexpr int R = 3, W = L::W, BW = L::BW, XO = L::XO, PB = L::PB, REG = L::REG;
  double *const sm =
      reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(sm_in) + 127) & ~uintptr_t(127));
  double *const box = sm + L::kBox;
  double *const pl = sm + L::kPl;

  const long long tiles_x = (a.nx + TX - 1) / TX;
  const long long tj = tile / tiles_x, ti = tile - tj * tiles_x;
  const long long i0 = ti * TX, j0 = tj * TY;
  double dt;
  if (!stage_control(a, b, tile == 0, zeroing_block, dt)) return;

  const double *Ub = a.Uin + b * 4 * (a.nx * a.ny);
  const double gm1 = a.gamma - 1.0;
  const int tid = threadIdx.x;

  // per-block constants (published by the barrier after phase 1): the
  // reconstruction parameters of the field scales 2 and 4, 0.25 / dx, dy
  __shared__ ReconParams s_rp[2];
  __shared__ double s_id[2];
  if (tid == 0) {
    s_rp[0] = make_rp(a, 2.0);
    s_rp[1] = make_rp(a, 4.0);
    s_id[0] = 0.25 / a.dx;
    s_id[1] = 0.25 / a.dy;
  }

  const bool use_tma = tm != nullptr && i0 - XO >= 0 && i0 - XO + BW <= a.nx && j0 - R >= 0 &&
                       j0 + TY + R <= a.ny;
  if (use_tma && !tma_stage_box<TX, TY, R>(a, tm, box, b, i0, j0)) return;

  // Phase 1: the cross-shaped region (tile rows with x halo, tile columns
  // with y halo): the conserved variables into the box where TMA did not
  // bring them, and per cell sqrt(rho), u, v, H.
  for (int k = tid; k < REG; k += blockDim.x) {
    const int r = k / W, c = k - r * W;
    const bool xb = (r >= R) && (r < R + TY), yb = (c >= R) && (c < R + TX);
    if (!(xb || yb)) continue;
    const int ob = r * BW + c + XO - R;
    double rho, mx, my, E;
    long long gj, gi;
    if (use_tma) {
      rho = box[ob];
      mx = box[PB + ob];
      my = box[2 * PB + ob];
      E = box[3 * PB + ob];
      gi = i0 - R + c;
      gj = j0 - R + r;
    } else {
      const double *src;
      long long o, pst;
      cell_source(a, Ub, b, i0, j0, R, r, c, src, o, pst, gj, gi);
      rho = src[o];
      mx = src[pst + o];
      my = src[2 * pst + o];
      E = src[3 * pst + o];
      box[ob] = rho;
      box[PB + ob] = mx;
      box[2 * PB + ob] = my;
      box[3 * PB + ob] = E;
    }
    const double rs = rsqrt_pos(rho);  // 1/sqrt(rho): gives 1/rho and sqrt(rho)
    const double ir = rs * rs;
    const double u = mx * ir, v = my * ir;
    const double p = gm1 * (E - 0.5 * fma(mx, u, my * v));
    if (!(pos_finite(rho) && pos_finite(p))) record_status(a.status, 3, a.stage, b, gj, gi);
    pl[k] = rho * rs;
    pl[REG + k] = u;
    pl[2 * REG + k] = v;
    pl[3 * REG + k] = (E + p) * ir;
  }
  __syncthreads();

  tile6_sweep<TX, TY, AI, P1, PREC, 0>(a, b, i0, j0, gm1, sm, s_rp[0], s_rp[1]);
  tile6_sweep<TX, TY, AI, P1, PREC, 1>(a, b, i0, j0, gm1, sm, s_rp[0], s_rp[1]);

  tile2d_update<TX, TY, R>(a, b, i0, j0, dt, sm + L::kFx, sm + L::kFy, s_id[0], s_id[1],
                           [&](int r, int c, int q) { return box[q * PB + (R + r) * BW + XO + c]; });
}

// One tile of a 2D stage of order 2R (sixth order: euler2d_tile6; 4, 8, 10:
// euler2d_tile_gen).
template <int TX, int TY, bool AI, bool P1, int PREC, int R = 3>
__device__ __forceinline__ void euler2d_tile(const StageArgs &a, long long b, long long tile,
                                             bool zeroing_block, double *sm,
                                             const CUtensorMap *tm = nullptr) {
  if constexpr (R == 3)
    euler2d_tile6<TX, TY, AI, P1, PREC>(a, b, tile, zeroing_block, sm, tm);
  else
    euler2d_tile_gen<TX, TY, AI, P1, PREC, R>(a, b, tile, zeroing_block, sm, tm);
}

// MINB: resident blocks per SM the register allocation must allow.
// tm: tensor map of a.Uin (see euler2d_tile), used when a.use_tma is set.
template <int TX, int TY, int NT, int MINB, bool AI, bool P1, int PREC, int R = 3>
__global__ void __launch_bounds__(NT, MINB)
    k_euler2d(const StageArgs a, const __grid_constant__ CUtensorMap tm) {
  extern __shared__ __align__(128) double sm[];
  euler2d_tile<TX, TY, AI, P1, PREC, R>(a, blockIdx.z, blockIdx.x,
                                        blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0, sm,
                                        a.use_tma ? &tm : nullptr);
}

#include "weno_tiles1d.cuh"

// Multiprocessors of the current device (asked once per process and device).
inline int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 152;
  }
  return cached[dev];
}

// Shared memory per SM the resident blocks of a launch may take (228 KB,
// less 1 KB the hardware keeps per block).
constexpr size_t kSmemPerSM = 233472;

template <int TX, int TY, int NT, int MINB, bool AI, bool P1, int PREC, int R = 3>
cudaError_t launch_2d(const StageArgs &a_in, cudaStream_t s) {
  StageArgs a = a_in;
  // TMA staging when the box fits beside the tile's planes at this
  // occupancy and the input is addressable by a tensor map
  constexpr bool kTmaFits = (smem_euler2d_tma<TX, TY, R>() + 1024) * MINB <= kSmemPerSM;
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  a.use_tma = kTmaFits && encode_state_map(a.Uin, a.nbatch, a.ny, a.nx, TX + 2 * TmaBox<R>::XO,
                                           TY + 2 * R, &tm);
  const char *nc = std::getenv("WENO_TEST_TMA_NO_COPY");
  a.tma_no_copy = (nc && nc[0] == '1') ? 1 : 0;
  const size_t smem = kTmaFits ? smem_euler2d_tma<TX, TY, R>() : smem_euler2d<TX, TY, R>();
  auto kern = k_euler2d<TX, TY, NT, MINB, AI, P1, PREC, R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = ((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY);
  dim3 grid((unsigned)tiles, 1, (unsigned)a.nbatch);
  kern<<<grid, NT, smem, s>>>(a, tm);
  return cudaGetLastError();
}

template <bool AI, bool P1, int PREC, int R>
cudaError_t launch_stage_t(const StageArgs &a, cudaStream_t s) {
  if (a.ndim == 2) {
    // tile variants (cells / threads / blocks per SM the registers allow):
    // 0 = 32x16 / 256 / 1 (fewest halo faces), 1 = 16x16 / 128 / 2,
    // 2 = 16x8 / 64 / 4 (more tiles for small grids), 3 = 16x16 / 128 / 3,
    // 4 = 16x8 / 64 / 6, and two shapes whose face count is a multiple of
    // the block's threads, so every warp computes the same number of faces:
    // 5 = 20x12 / 128 / 3 (512 faces), 6 = 26x14 / 128 / 3 (768 faces).
    // For grids too small to fill the GPU, where a stage lasts as long as one
    // thread's chain of faces, about one face per thread: 7 = 16x8 / 256 / 1
    // (280 faces), 8 = 8x8 / 128 / 2 (144 faces).  The sixth-order tile
    // sweeps the x- and then the y-faces; two shapes give every thread
    // exactly two faces of each sweep (warp i of every block runs on the
    // same SM sub-partition, so an uneven count leaves three of the four
    // FP64 pipes idle at the end of a sweep): 9 = 16x15 / 128 / 3 (255 and
    // 256 faces), 10 = 14x17 / 128 / 3 (255 and 252).
    // The other orders use 16x16 / 128 only, 3 blocks per SM at r = 2 and 2
    // at r = 4, 5 (their wider stencils need more registers).
    if constexpr (R != 3) {  // r = 2 fits the 168-register cap of 3 blocks per SM
      return launch_2d<16, 16, 128, (R == 2 ? 3 : 2), AI, P1, PREC, R>(a, s);
    } else {
      switch (a.tile_variant) {
        case 1: return launch_2d<16, 16, 128, 2, AI, P1, PREC>(a, s);
        case 2: return launch_2d<16, 8, 64, 4, AI, P1, PREC>(a, s);
        case 3: return launch_2d<16, 16, 128, 3, AI, P1, PREC>(a, s);
        case 4: return launch_2d<16, 8, 64, 6, AI, P1, PREC>(a, s);
        case 5: return launch_2d<20, 12, 128, 3, AI, P1, PREC>(a, s);
        case 6: return launch_2d<26, 14, 128, 3, AI, P1, PREC>(a, s);
        case 7: return launch_2d<16, 8, 256, 1, AI, P1, PREC>(a, s);
        case 8: return launch_2d<8, 8, 128, 2, AI, P1, PREC>(a, s);
        case 9: return launch_2d<16, 15, 128, 3, AI, P1, PREC>(a, s);
        case 10: return launch_2d<14, 17, 128, 3, AI, P1, PREC>(a, s);
        default: return launch_2d<kTX, kTY, kThreads2D, 1, AI, P1, PREC>(a, s);
      }
    }
  }
  const long long tiles = (a.nx + kT1 - 1) / kT1;
  if constexpr (R == 3) {
    // A problem of fewer tiles than the GPU has SMs is bound by the length
    // of one thread's chain of FP64 operations: spread each face over
    // several threads (and the problem over more blocks) instead.
    if (tiles * a.nbatch < (long long)sm_count() && (a.nc == 3 || PREC == 0)) {
      const int tl1 = a.nc == 3 ? kT1Lanes(3) : kT1Lanes(1);
      dim3 g2((unsigned)((a.nx + tl1 - 1) / tl1), (unsigned)a.nbatch, 1);
      if (a.nc == 3)
        k_line1d_lanes<3, AI, P1, PREC>
            <<<g2, kThreads1D, smem_line1d<3, kT1Lanes(3), 3, 3>(), s>>>(a);
      else if constexpr (PREC == 0)
        k_line1d_lanes<1, AI, P1, PREC>
            <<<g2, kThreads1D, smem_line1d<1, kT1Lanes(1), 3, 2>(), s>>>(a);
      return cudaGetLastError();
    }
  }
  dim3 grid((unsigned)tiles, (unsigned)a.nbatch, 1);
  if (a.nc == 3)
    k_line1d<3, AI, P1, PREC, R><<<grid, kThreads1D, smem_line1d<3, kT1, R>(), s>>>(a);
  else
    k_line1d<1, AI, P1, PREC, R><<<grid, kThreads1D, smem_line1d<1, kT1, R>(), s>>>(a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace weno
