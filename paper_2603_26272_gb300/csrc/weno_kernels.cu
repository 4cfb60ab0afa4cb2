// weno_kernels.cu -- sixth-order (WENO-ZA6) stage launches, the wavespeed
// reductions of eq. (6), the serving engine's persistent stage kernel and the
// host-side launchers for GB300 (sm_103a).  The tile kernels themselves are in
// weno_tiles.cuh; the schemes of other orders are instantiated in
// weno_orders.cu.
#include <mutex>

#include "weno_tiles.cuh"

namespace weno {
namespace {

// ---------------------------------------------------------------------------
// Wavespeed maxima of a state (the GLF speeds of eq. (6)), grid-stride per
// problem (blockIdx.y).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_alpha(const AlphaArgs a) {
  const long long b = blockIdx.y;
  const long long plane = a.nx * a.ny;
  const double *Ub = a.U + b * a.nc * plane;
  if (a.system >= 2) {  // scalar: keys of max u and max -u
    unsigned long long km[2] = {0ull, 0ull};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < plane;
         k += (long long)gridDim.x * blockDim.x) {
      const double u = Ub[k];
      if (!(u == u) || fabs(u) > 1.7e308) record_status(a.status, 3, 0, b, 0, k);
      km[0] = max(km[0], okey(u));
      km[1] = max(km[1], okey(-u));
    }
    const int slot[2] = {0, 1};
    const int dup[2] = {-1, -1};
    block_max_atomic<2>(km, a.alpha_out + b * 8, slot, dup);
    return;
  }
  const double gm1 = a.gamma - 1.0;
  unsigned long long vm[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < plane;
       k += (long long)gridDim.x * blockDim.x) {
    const double rho = Ub[k];
    const double ir = rcp_pos(rho);
    const double mx = Ub[plane + k];
    const double my = (a.nc == 4) ? Ub[2 * plane + k] : 0.0;
    const double E = Ub[(a.nc - 1) * plane + k];
    const double u = mx * ir, v = my * ir;
    const double p = gm1 * (E - 0.5 * fma(mx, u, my * v));
    if (!(pos_finite(rho) && pos_finite(p)))
      record_status(a.status, 3, 0, b, k / a.nx, k % a.nx);
    const double cs = sqrt_pos(a.gamma * p * ir);
    vm[0] = max(vm[0], abs_bits(u - cs));
    vm[1] = max(vm[1], abs_bits(u));
    vm[2] = max(vm[2], abs_bits(u + cs));
    vm[3] = max(vm[3], abs_bits(v - cs));
    vm[4] = max(vm[4], abs_bits(v));
    vm[5] = max(vm[5], abs_bits(v + cs));
  }
  if (a.nc == 3) {
    const int slot[6] = {0, 1, 2, 4, 5, 7};  // 1D: fields u-c, u, u+c in slots 0..2
    const int dup[6] = {-1, -1, -1, -1, -1, -1};
    unsigned long long w[6] = {vm[0], vm[1], vm[2], 0ull, 0ull, 0ull};
    block_max_atomic<6>(w, a.alpha_out + b * 8, slot, dup);
  } else {
    const int slot[6] = {0, 1, 3, 4, 5, 7};
    const int dup[6] = {-1, 2, -1, -1, 6, -1};
    block_max_atomic<6>(vm, a.alpha_out + b * 8, slot, dup);
  }
}

__global__ void k_alpha_export(const AlphaArgs a, const unsigned long long *bits, double *alpha,
                               double *dt) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.nbatch) return;
  const unsigned long long *al = bits + b * 8;
  if (alpha) {
    for (int k = 0; k < 8; ++k) alpha[b * 8 + k] = 0.0;
    if (a.system == 0 || a.system >= 2) {
      alpha[b * 8] = scalar_alpha_of(a.system, a.adv_speed, a.ustar, al);
    } else {
      for (int k = 0; k < 8; ++k) alpha[b * 8 + k] = bits2d(al[k]);
      if (a.alpha_single)
        for (int dir = 0; dir < a.ndim; ++dir) {
          double m = 0.0;
          for (int k = 0; k < a.nc; ++k) m = fmax(m, alpha[b * 8 + dir * 4 + k]);
          for (int k = 0; k < a.nc; ++k) alpha[b * 8 + dir * 4 + k] = m;
        }
    }
  }
  if (dt) dt[b] = cfl_dt(a.system, a.ndim, a.nc, a.cfl, a.dx, a.dy, a.adv_speed, al, a.ustar);
}

__global__ void k_pack_rows(const double *U, long long nplanes, long long ny, long long nx,
                            long long j0, long long nr, double *out) {
  const long long per = nr * nx, n = nplanes * per;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const long long pl = k / per, rem = k - pl * per;
    out[k] = U[pl * ny * nx + j0 * nx + rem];
  }
}

__global__ void k_fill(double *p, long long n, double v) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    p[k] = v;
}


// ---------------------------------------------------------------------------
// Serving engine stage kernel.  A persistent grid (kEngineBlocksPerSM blocks
// of kEngineThreads per SM) takes tiles from the device-resident work list,
// from entry *first on, with an atomic counter (heaviest tiles first in the
// list; the fast slots' tiles last, so a sub-step over the fast slots only
// starts at their first entry) and runs the same tile functions as the
// single-problem kernels, on the slot's own buffers, speed slots and clock.
// The counter of the launch after next is cleared here, so consecutive
// launches never wait on the host.  Restricted to the scheme's default
// (Ai weights, p = 1); FP64 or FP32 reconstruction per slot.
// ---------------------------------------------------------------------------
__device__ __forceinline__ StageArgs slot_stage_args(const SlotDev &S, int stage) {
  StageArgs a;
  a.system = 1;
  a.ndim = S.ndim;
  a.nc = S.nc;
  a.nbatch = 1;
  a.nx = S.nx;
  a.ny = S.ny;
  a.dx = S.dx;
  a.dy = S.dy;
  a.bc_x = S.bc_x;
  a.bc_y = S.bc_y;
  a.gamma = S.gamma;
  a.cfl = S.cfl;
  a.eps = S.eps;
  a.mu0 = S.mu0;
  a.p = S.p;
  a.ai = 1;
  a.alpha_single = S.alpha_single;
  a.precision = S.precision;
  a.adv_speed = 0.0;
  const int kin = stage - 1, kout = stage % 3, kzero = (stage + 1) % 3;
  a.alpha_in = S.alpha + 8 * kin;
  a.alpha_out = S.alpha + 8 * kout;
  a.alpha_zero = S.alpha + 8 * kzero;
  a.mode = 0;
  a.stage = stage;
  a.dt_fixed = 0.0;
  a.t_final = S.t_final;
  a.halo_lo = a.halo_hi = nullptr;
  a.send_lo = a.send_hi = nullptr;
  a.use_tma = a.tma_no_copy = 0;
  a.t = S.clock;
  a.tnext = S.clock + 1;
  a.dt = S.clock + 2;
  a.steps = S.steps;
  a.status = S.status;
  if (stage == 1) {
    a.Uin = S.U; a.Un = nullptr; a.Uout = S.U1; a.a_n = 0.0; a.a_s = 1.0;
  } else if (stage == 2) {
    a.Uin = S.U1; a.Un = S.U; a.Uout = S.U2; a.a_n = 0.75; a.a_s = 0.25;
  } else {
    a.Uin = S.U2; a.Un = S.U; a.Uout = S.U; a.a_n = 1.0 / 3.0; a.a_s = 2.0 / 3.0;
  }
  return a;
}

__global__ void __launch_bounds__(kEngineThreads, kEngineBlocksPerSM) k_engine(const EngineArgs e) {
  extern __shared__ double sm[];
  __shared__ int s_w;
  const int cin = e.stage - 1, czero = (e.stage + 1) % 3;
  if (blockIdx.x == 0 && threadIdx.x == 0) e.counters[czero] = 0;
  const int ntiles = *e.ntiles, first = *e.first;
  for (;;) {
    if (threadIdx.x == 0) s_w = first + atomicAdd(&e.counters[cin], 1);
    __syncthreads();
    const int w = s_w;
    __syncthreads();
    if (w >= ntiles) break;
    const EngineTile t = e.tiles[w];
    const SlotDev &S = e.slots[t.slot];
    if (S.active) {
      const StageArgs a = slot_stage_args(S, e.stage);
      if (S.ndim == 2) {
        if (S.precision == 1)
          euler2d_tile<kEngineTX, kEngineTY, true, true, 1>(a, 0, t.tile, t.tile == 0, sm);
        else
          euler2d_tile<kEngineTX, kEngineTY, true, true, 0>(a, 0, t.tile, t.tile == 0, sm);
      } else {
        if (S.precision == 1)
          line1d_tile<3, true, true, 1, kEngine1DCells>(a, 0, t.tile, t.tile == 0, sm);
        else
          line1d_tile<3, true, true, 0, kEngine1DCells>(a, 0, t.tile, t.tile == 0, sm);
      }
    }
    __syncthreads();
  }
}

template <bool AI, bool P1>
cudaError_t launch_order(const StageArgs &a, cudaStream_t s) {
  if (a.order_r != 3) return launch_stage_orders(a, s);  // weno_orders.cu
  return launch_stage_t<AI, P1, 0, 3>(a, s);
}

}  // namespace

namespace {
// cuTensorMapEncodeTiled, looked up once through the runtime (the library
// links no driver library of its own)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}
}  // namespace

bool encode_state_map(const double *U, long long nbatch, long long ny, long long nx, int bw,
                      int bh, CUtensorMap *out) {
  if (!U || (nx & 1) || (reinterpret_cast<uintptr_t>(U) & 15) || nx < bw || ny < bh) return false;
  if (nx > (1LL << 31) || ny > (1LL << 31) || nbatch * 4 > (1LL << 31)) return false;
  EncodeTiledFn fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)(nbatch * 4)};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 8, (cuuint64_t)nx * (cuuint64_t)ny * 8};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 4};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double *>(U), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_stage(const StageArgs &a, cudaStream_t s) {
  const bool p1 = (a.p == 1.0);
  if (a.precision == 1)  // FP32 reconstruction (affine-invariant weights, order 6)
    return p1 ? launch_stage_t<true, true, 1, 3>(a, s) : launch_stage_t<true, false, 1, 3>(a, s);
  if (a.ai) return p1 ? launch_order<true, true>(a, s) : launch_order<true, false>(a, s);
  return p1 ? launch_order<false, true>(a, s) : launch_order<false, false>(a, s);
}

size_t engine_smem_bytes() {
  const size_t a = smem_euler2d<kEngineTX, kEngineTY>(), b = smem_line1d<3, kEngine1DCells>();
  return a > b ? a : b;
}

long long engine_tiles_of(int ndim, long long nx, long long ny) {
  if (ndim == 2) return ((nx + kEngineTX - 1) / kEngineTX) * ((ny + kEngineTY - 1) / kEngineTY);
  return (nx + kEngine1DCells - 1) / kEngine1DCells;
}

cudaError_t engine_prepare() {
  return cudaFuncSetAttribute(k_engine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)engine_smem_bytes());
}

cudaError_t launch_engine_stage(const EngineArgs &e, int grid, cudaStream_t s) {
  k_engine<<<grid, kEngineThreads, engine_smem_bytes(), s>>>(e);
  return cudaGetLastError();
}

cudaError_t launch_alpha(const AlphaArgs &a, cudaStream_t s) {
  if (a.system == 0) return cudaSuccess;  // linear advection: alpha = |a|, no reduction
  const long long plane = a.nx * a.ny;
  long long bx = (plane + 255) / 256;
  if (bx > 1024) bx = 1024;
  dim3 grid((unsigned)bx, (unsigned)a.nbatch, 1);
  k_alpha<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_alpha_export(const AlphaArgs &a, const unsigned long long *bits, double *alpha,
                                double *dt, cudaStream_t s) {
  const unsigned nb = (unsigned)((a.nbatch + 127) / 128);
  k_alpha_export<<<nb, 128, 0, s>>>(a, bits, alpha, dt);
  return cudaGetLastError();
}

cudaError_t launch_pack_rows(const double *U, long long nbatch, int nc, long long ny, long long nx,
                             long long j0, long long nr, double *out, cudaStream_t s) {
  const long long n = nbatch * nc * nr * nx;
  if (n <= 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_pack_rows<<<(unsigned)nb, 256, 0, s>>>(U, nbatch * nc, ny, nx, j0, nr, out);
  return cudaGetLastError();
}

cudaError_t launch_fill(double *p, long long n, double v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_fill<<<(unsigned)nb, 256, 0, s>>>(p, n, v);
  return cudaGetLastError();
}

}  // namespace weno
