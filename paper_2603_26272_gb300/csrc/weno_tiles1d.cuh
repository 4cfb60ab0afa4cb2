// weno_tiles1d.cuh -- the 1D stage kernels (Euler and scalar equations) of
// the central-upwind WENO right-hand side, templated on the stencil
// half-width r.  Included by weno_tiles.cuh inside its namespaces; it uses
// the helpers defined there (stage_control, make_rp, block_max_atomic, ...).
#pragma once

// ---------------------------------------------------------------------------
// 1D stage kernel: NC = 3 (Euler) or 1 (scalar advection).  Tile of
// kT1 = 127 cells, 128 faces, one face per thread.
// Planes: 0 rho, 1 m, 2 E, 3 u, 4 H, 5 sqrt(rho), 6-8 F  (advection: 0 u).
// Sixth-order Euler projects differences of adjacent cells, as the 2D
// kernel does (euler2d_tile6): dd holds per cell pair d rho, dm, dE, dF1, dF2
// (dF0 = dm), and the centre values come back as 4 F_i + 2 (F_{i+1} - F_i)
// after the back-projection.
// ---------------------------------------------------------------------------
// The centre values of a sixth-order 1D Euler face between cells L and L+1:
// 4 F_hat += 2 (F_L + F_{L+1}) = 4 F_L + 2 dF of pair L (R L = I).
__device__ __forceinline__ void add_centre3(double FL0, double FL1, double FL2, const double *dd,
                                            int nd, int pair, double &F0, double &F1,
                                            double &F2) {
  F0 = fma(4.0, FL0, fma(2.0, dd[nd + pair], F0));
  F1 = fma(4.0, FL1, fma(2.0, dd[3 * nd + pair], F1));
  F2 = fma(4.0, FL2, fma(2.0, dd[4 * nd + pair], F2));
}

template <int NC, int T, int R = 3, int LANES = 1>
constexpr size_t smem_line1d() {
  return sizeof(double) * (((NC == 3) ? 9 : 2) * (T + 2 * R) + (T + 1) * NC +
                           (LANES > 1 ? (T + 1) * NC : 0) +
                           ((NC == 3 && R == 3) ? 5 * (T + 2 * R - 1) : 0));
}

// One tile of T cells (T + 1 faces) of a 1D stage with a stencil of
// half-width R (order 2R).  LANES threads share a face: 1 (blockDim = T + 1,
// the throughput layout), or -- for problems too small to fill the GPU, where
// a stage's time is one thread's chain of FP64 operations -- 3 for Euler (one
// characteristic field each; blockDim >= 3 (T + 1)) and 2 for a scalar (the
// positive and the negative flux; blockDim >= 2 (T + 1)).  Every lane layout
// runs the same arithmetic per field, so the results are bitwise identical.
// sm: dynamic shared memory of smem_line1d<NC, T, R, LANES>() bytes.
template <int NC, bool AI, bool P1, int PREC, int T, int R = 3, int LANES = 1>
__device__ __forceinline__ void line1d_tile(const StageArgs &a, long long b, long long tile,
                                            bool zeroing_block, double *sm) {
  static_assert(R == 3 || PREC == 0, "FP32 reconstruction is sixth order only");
  static_assert(LANES == 1 || (R == 3 && LANES == (NC == 3 ? 3 : 2) && (NC == 3 || PREC == 0)),
                "lane layouts: 3 per face for Euler, 2 for a scalar in FP64, sixth order");
  constexpr int REG = T + 2 * R, N = 2 * R;
  constexpr int NP = (NC == 3) ? 9 : 2;
  double(*pl)[REG] = reinterpret_cast<double(*)[REG]>(sm);
  double(*fl)[NC] = reinterpret_cast<double(*)[NC]>(sm + NP * REG);
  double *const hb = sm + NP * REG + (T + 1) * NC;  // LANES > 1: per-field fluxes
  constexpr bool kDiff = (NC == 3 && R == 3);
  constexpr int ND = REG - 1;  // cell pairs of the tile
  double *const dd = hb + (LANES > 1 ? (T + 1) * NC : 0);  // kDiff: [5][ND]
  const long long i0 = tile * T;
  double dt;
  if (!stage_control(a, b, tile == 0, zeroing_block, dt)) return;
  const long long nx = a.nx;
  const double *Ub = a.Uin + b * NC * nx;
  const double gm1 = a.gamma - 1.0;
  const int tid = threadIdx.x;
  // per-block constants, published by the barrier after the staging: the
  // reconstruction parameters of the field scales 2 and 4, FP32 ones, and
  // the flux difference's factor (the faces hold 4 F for Euler, 2 F for a
  // scalar: the split without 1/2)
  __shared__ ReconParams s_rp[2];
  __shared__ Recon32 s_r32;
  __shared__ double s_idx;
  if (tid == 0) {
    s_rp[0] = make_rp(a, 2.0);
    s_rp[1] = make_rp(a, 4.0);
    s_r32 = make_r32(a);
    s_idx = (NC == 3 ? 0.25 : 0.5) / a.dx;
  }

  for (int k = tid; k < REG; k += blockDim.x) {
    const long long gi = ghost(i0 - R + k, nx, a.bc_x);
    if (NC == 1) {
      const double u = Ub[gi];
      if (!(u == u) || fabs(u) > 1.7e308) record_status(a.status, 3, a.stage, b, 0, gi);
      pl[0][k] = u;
      pl[1][k] = scalar_flux(a.system, a.adv_speed, u);
    } else {
      const double rho = Ub[gi], m = Ub[nx + gi], E = Ub[2 * nx + gi];
      const double rs = rsqrt_pos(rho);
      const double ir = rs * rs;
      const double u = m * ir;
      const double p = gm1 * (E - 0.5 * (m * u));
      if (!(pos_finite(rho) && pos_finite(p))) record_status(a.status, 3, a.stage, b, 0, gi);
      const double rH = E + p;
      pl[0][k] = rho;
      pl[1][k] = m;
      pl[2][k] = E;
      pl[3][k] = u;
      pl[4][k] = rH * ir;
      pl[5][k] = rho * rs;
      pl[6][k] = m;
      pl[7][k] = fma(m, u, p);
      pl[8][k] = rH * u;
    }
  }
  __syncthreads();
  if constexpr (kDiff) {
    for (int k = tid; k < ND; k += blockDim.x) {
      dd[k] = pl[0][k + 1] - pl[0][k];
      dd[ND + k] = pl[1][k + 1] - pl[1][k];
      dd[2 * ND + k] = pl[2][k + 1] - pl[2][k];
      dd[3 * ND + k] = pl[7][k + 1] - pl[7][k];
      dd[4 * ND + k] = pl[8][k + 1] - pl[8][k];
    }
    __syncthreads();
  }

  if constexpr (LANES == 3) {
    // one characteristic field per thread; the field-0 thread back-projects
    const int f = tid / 3, q = tid - 3 * f;
    const bool act = (f <= T) && (i0 + f - 1 < nx);
    FaceState fs;
    if (act) {
      const int kL = f + 2, kR = f + 3;
      if (!roe_face(pl[5][kL], pl[3][kL], 0.0, pl[4][kL], pl[5][kR], pl[3][kR], 0.0, pl[4][kR],
                    gm1, fs) && q == 0)
        record_status(a.status, 3, a.stage, b, 0, i0 + f);
      const unsigned long long *al = a.alpha_in + b * 8;
      double A = bits2d(al[q]);
      if (a.alpha_single) A = fmax(fmax(bits2d(al[0]), bits2d(al[1])), bits2d(al[2]));
      double h;
      double dW[5], dG[5];  // the field's projected differences over pairs f .. f+4
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        const int k = f + j;
        dW[j] = project3_field(fs, q, dd[k], dd[ND + k], dd[2 * ND + k]);
        dG[j] = project3_field(fs, q, dd[ND + k], dd[3 * ND + k], dd[4 * ND + k]);
      }
      if constexpr (PREC == 1)
        h = field_flux_f32d<P1>(dW, dG, A, s_r32);
      else
        h = field_flux_d<AI, P1>(dW, dG, A, s_rp[q == 1 ? 0 : 1]);
      hb[3 * f + q] = h;
    }
    __syncthreads();
    if (act && q == 0) {
      double F0, F1, F2;
      backproject3(fs, hb[3 * f], hb[3 * f + 1], hb[3 * f + 2], F0, F1, F2);
      add_centre3(pl[6][f + 2], pl[7][f + 2], pl[8][f + 2], dd, ND, f + 2, F0, F1, F2);
      fl[f][0] = F0;
      fl[f][1] = F1;
      fl[f][2] = F2;
    }
  } else if constexpr (LANES == 2) {
    // the positive (even lane) and the mirrored negative flux (odd lane) of a
    // scalar face; the partial sums meet by a lane shuffle
    // (the differences and the centre sum as field_flux forms them)
    const int f = tid >> 1, sgn = tid & 1;
    const bool act = (f <= T) && (i0 + f - 1 < nx);
    ZA6Part part = {0.0, 1.0};
    double base = 0.0;
    if (act) {
      const double A = scalar_alpha_of(a.system, a.adv_speed, a.ustar, a.alpha_in + b * 8);
      const ReconParams rp = s_rp[0];
      double dd[5], dw2 = 0.0;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        const double dw = pl[0][f + j + 1] - pl[0][f + j], dg = pl[1][f + j + 1] - pl[1][f + j];
        if (sgn)
          dd[4 - j] = fma(A, dw, -dg);
        else
          dd[j] = fma(A, dw, dg);
        if (j == 2) dw2 = dw;
      }
      base = fma(-A, dw2, pl[1][f + 2] + pl[1][f + 3]);
      part = za6d<AI, P1>(dd[0], dd[1], dd[2], dd[3], dd[4], rp);
    }
    const ZA6Part other = {__shfl_xor_sync(0xffffffffu, part.num, 1),
                           __shfl_xor_sync(0xffffffffu, part.den, 1)};
    if (act && sgn == 0) fl[f][0] = pair_flux(base, part, other);
  } else {
    const int f = tid;  // face between cells i0+f-1 and i0+f; stencil f..f+2R-1
    if (f <= T && i0 + f - 1 < nx) {
      if (NC == 1) {
        const double A = scalar_alpha_of(a.system, a.adv_speed, a.ustar, a.alpha_in + b * 8);
        double h;
        if constexpr (PREC == 1) {
          double w[6], g[6];
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            w[j] = pl[0][f + j];
            g[j] = pl[1][f + j];
          }
          h = field_flux_f32<P1>(w, g, A, s_r32);
        } else if constexpr (R == 3) {
          double w[6], g[6];
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            w[j] = pl[0][f + j];
            g[j] = pl[1][f + j];
          }
          h = field_flux<AI, P1>(w, g, A, s_rp[0]);
        } else {
          const ReconParams rp = s_rp[0];
          double pp[N], mm[N];  // f^+ in stencil order, f^- mirrored
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const double v = pl[0][f + j], fv = pl[1][f + j];
            pp[j] = fma(A, v, fv);
            mm[N - 1 - j] = fma(-A, v, fv);
          }
          h = pair_flux_r<R>(za_r<R, AI, P1>(pp, rp), za_r<R, AI, P1>(mm, rp));
        }
        fl[f][0] = h;  // 2 F (the split without 1/2); 1/2 goes with 1/dx
      } else {
        const int kL = f + R - 1, kR = f + R;
        FaceState fs;
        if (!roe_face(pl[5][kL], pl[3][kL], 0.0, pl[4][kL], pl[5][kR], pl[3][kR], 0.0, pl[4][kR],
                      gm1, fs))
          record_status(a.status, 3, a.stage, b, 0, i0 + f);
        const unsigned long long *al = a.alpha_in + b * 8;
        double A1 = bits2d(al[0]), A2 = bits2d(al[1]), A3 = bits2d(al[2]);
        if (a.alpha_single) A1 = A2 = A3 = fmax(fmax(A1, A2), A3);
        double h1, h2, h3;
        if constexpr (R == 3) {
          double dW[3][5], dG[3][5];  // projected differences over pairs f .. f+4
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            const int k = f + j;
            project3(fs, dd[k], dd[ND + k], dd[2 * ND + k], dW[0][j], dW[1][j], dW[2][j]);
            project3(fs, dd[ND + k], dd[3 * ND + k], dd[4 * ND + k], dG[0][j], dG[1][j],
                     dG[2][j]);
          }
          if constexpr (PREC == 1) {
            h1 = field_flux_f32d<P1>(dW[0], dG[0], A1, s_r32);
            h2 = field_flux_f32d<P1>(dW[1], dG[1], A2, s_r32);
            h3 = field_flux_f32d<P1>(dW[2], dG[2], A3, s_r32);
          } else {
            h1 = field_flux_d<AI, P1>(dW[0], dG[0], A1, s_rp[1]);
            h2 = field_flux_d<AI, P1>(dW[1], dG[1], A2, s_rp[0]);
            h3 = field_flux_d<AI, P1>(dW[2], dG[2], A3, s_rp[1]);
          }
        } else {
          const ReconParams rp4 = s_rp[1], rp2 = s_rp[0];
          double p1[N], p2[N], p3[N], m1[N], m2[N], m3[N];  // f^- mirrored
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const int k = f + j;
            double w1, w2, w3, g1, g2, g3;
            project3(fs, pl[0][k], pl[1][k], pl[2][k], w1, w2, w3);
            project3(fs, pl[6][k], pl[7][k], pl[8][k], g1, g2, g3);
            p1[j] = fma(A1, w1, g1);
            m1[N - 1 - j] = fma(-A1, w1, g1);
            p2[j] = fma(A2, w2, g2);
            m2[N - 1 - j] = fma(-A2, w2, g2);
            p3[j] = fma(A3, w3, g3);
            m3[N - 1 - j] = fma(-A3, w3, g3);
          }
          h1 = pair_flux_r<R>(za_r<R, AI, P1>(p1, rp4), za_r<R, AI, P1>(m1, rp4));
          h2 = pair_flux_r<R>(za_r<R, AI, P1>(p2, rp2), za_r<R, AI, P1>(m2, rp2));
          h3 = pair_flux_r<R>(za_r<R, AI, P1>(p3, rp4), za_r<R, AI, P1>(m3, rp4));
        }
        double F0, F1, F2;
        backproject3(fs, h1, h2, h3, F0, F1, F2);
        if constexpr (R == 3) add_centre3(pl[6][kL], pl[7][kL], pl[8][kL], dd, ND, kL, F0, F1, F2);
        fl[f][0] = F0;
        fl[f][1] = F1;
        fl[f][2] = F2;
      }
    }
  }
  __syncthreads();

  // The faces hold 4 F (Euler, backproject3) or 2 F (a scalar: the split
  // without 1/2), so that factor goes with 1/dx.
  const double idx = s_idx;
  unsigned long long m3v[3] = {0ull, 0ull, 0ull};
  const bool want_alpha = (NC == 3 || a.system >= 2) && (a.mode == 0) && (a.alpha_out != nullptr);
  if (tid < T && i0 + tid < nx) {
    const long long gi = i0 + tid;
    const long long o = b * NC * nx + gi;
    double uo[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const double L = -(fl[tid + 1][q] - fl[tid][q]) * idx;
      if (a.mode == 1) {
        uo[q] = L;
      } else {
        const double uin = (NC == 1) ? pl[0][tid + R] : pl[q][tid + R];
        const double base_s = fma(dt, L, uin);
        uo[q] = (a.a_n != 0.0) ? fma(a.a_n, a.Un[o + q * nx], a.a_s * base_s) : a.a_s * base_s;
      }
      a.Uout[o + q * nx] = uo[q];
    }
    if (want_alpha && NC == 1) {  // scalar: keys of max u and max -u
      if (!(uo[0] == uo[0]) || fabs(uo[0]) > 1.7e308) record_status(a.status, 3, a.stage, b, 0, gi);
      m3v[0] = okey(uo[0]);
      m3v[1] = okey(-uo[0]);
    } else if (want_alpha) {
      const double ir = rcp_pos(uo[0]);
      const double u = uo[1] * ir;
      const double p = gm1 * (uo[NC - 1] - 0.5 * (uo[1] * u));
      if (!(pos_finite(uo[0]) && pos_finite(p))) record_status(a.status, 3, a.stage, b, 0, gi);
      const double cs = sqrt_pos(a.gamma * p * ir);
      m3v[0] = abs_bits(u - cs);
      m3v[1] = abs_bits(u);
      m3v[2] = abs_bits(u + cs);
    }
  }
  if (want_alpha) {
    const int slot[3] = {0, 1, 2};
    const int dup[3] = {-1, -1, -1};
    block_max_atomic<3>(m3v, a.alpha_out + b * 8, slot, dup);
  }
}

template <int NC, bool AI, bool P1, int PREC, int R = 3>
__global__ void __launch_bounds__(kThreads1D) k_line1d(const StageArgs a) {
  extern __shared__ double sm[];
  line1d_tile<NC, AI, P1, PREC, kT1, R>(a, blockIdx.y, blockIdx.x,
                                        blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0, sm);
}

// Latency layout of small 1D problems: 128 threads, 3 per face for Euler
// (41 cells a tile) or 2 per face for a scalar (63 cells).
__host__ __device__ constexpr int kT1Lanes(int nc) { return nc == 3 ? 41 : 63; }

template <int NC, bool AI, bool P1, int PREC>
__global__ void __launch_bounds__(kThreads1D) k_line1d_lanes(const StageArgs a) {
  extern __shared__ double sm[];
  line1d_tile<NC, AI, P1, PREC, kT1Lanes(NC), 3, (NC == 3 ? 3 : 2)>(
      a, blockIdx.y, blockIdx.x, blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0, sm);
}
