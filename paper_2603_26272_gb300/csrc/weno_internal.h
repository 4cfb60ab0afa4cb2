// weno_internal.h -- launch interface between the C-ABI layer and the kernels.
#pragma once
#include <cstdint>
#include <string>
#include <cuda.h>
#include <cuda_runtime.h>

namespace weno {

// Device status word and the location of the first failure.
struct DevStatus {
  int code;      // 0 ok, 3 nonphysical
  int stage;     // kernel that recorded it (0 wavespeeds, 1..3 RK stage, 4 rhs)
  long long b, j, i;
};

// 2D tile variants of the single-problem stage kernel (see launch_stage_t).
constexpr int kTileVariants = 11;

// Everything one stage launch needs (passed by value).
struct StageArgs {
  // grid
  int system, ndim, nc;
  long long nbatch, nx, ny;
  double dx, dy;
  int bc_x, bc_y;
  double gamma;
  // scheme
  double cfl, eps, mu0, p;
  int ai, alpha_single;
  int precision;      // 0 FP64, 1 FP32 reconstruction
  int order_r;        // r: stencil half-width, scheme order 2r (3 = WENO-ZA6)
  double ustar;       // Buckley-Leverett: maximiser of f' on [0, 1]
  int tile_variant;   // 2D tile shape, 0 .. kTileVariants-1 (results identical)
  double adv_speed;
  // data
  const double *Uin;  // stage input (read with the stencil)
  const double *Un;   // base of the RK combination (read at the own cell only)
  double *Uout;       // may alias Un (last stage)
  double a_n, a_s;    // Uout = a_n Un + a_s (Uin + dt L(Uin))
  int mode;           // 0 RK stage, 1 write L(Uin)
  int stage;          // 1, 2, 3 (1 sets dt, 3 advances t) ; 0 for rhs
  double dt_fixed;    // > 0: fixed step for stage 1
  double t_final;     // clipping target of stage 1 (inf: none)
  // workspace
  const unsigned long long *alpha_in;  // [nbatch][8] bit patterns of |lambda| maxima
  unsigned long long *alpha_out;       // next stage's maxima (NULL: skip)
  unsigned long long *alpha_zero;      // slot to clear for the stage after next (NULL: skip)
  double *t, *tnext, *dt;              // [nbatch]
  long long *steps;                    // [nbatch]
  DevStatus *status;
  // 2D strip of a domain split in y (NULL when unused): the r ghost rows
  // below row 0 / above row ny-1 come from halo_lo / halo_hi ([nbatch][4][r][nx],
  // rows in increasing j) instead of the boundary condition, and the stage
  // output's first / last r rows are copied into send_lo / send_hi (same layout).
  const double *halo_lo, *halo_hi;
  double *send_lo, *send_hi;
  // set by the 2D launcher: interior tiles stage by TMA through the tensor
  // map passed beside these arguments; tma_no_copy (a test of the bounded
  // wait, WENO_TEST_TMA_NO_COPY=1 in the environment) arms the barrier but
  // issues no copy, so every TMA wait runs out and reports WENO_ERR_TIMEOUT
  int use_tma, tma_no_copy;
};

// Wavespeed reduction of U into alpha_out (which must be zero), optional dt.
struct AlphaArgs {
  int system, ndim, nc, alpha_single;
  long long nbatch, nx, ny;
  double dx, dy, gamma, cfl, adv_speed, ustar;
  const double *U;
  unsigned long long *alpha_out;
  DevStatus *status;
};

// ---------------------------------------------------------------------------
// Serving engine: many independent solves ("slots") of mixed shape and
// precision advanced together by one persistent kernel per Runge-Kutta stage.
// ---------------------------------------------------------------------------
struct SlotDev {
  int ndim, nc, bc_x, bc_y, precision, alpha_single, active, pad;
  long long nx, ny;
  double dx, dy, gamma, cfl, eps, mu0, p, t_final;
  double *U, *U1, *U2;          // state and the two stage buffers
  unsigned long long *alpha;    // [3][8] rotating speed-maxima slots
  double *clock;                // t, tnext, dt
  long long *steps;
  DevStatus *status;
};

struct EngineTile {
  int slot;
  int tile;
};

struct EngineArgs {
  const SlotDev *slots;
  const EngineTile *tiles;
  const int *ntiles;
  const int *first;             // first work-list entry of this launch (0, or
                                // the start of the fast slots' tiles)
  int *counters;                // [3] rotating work counters
  int stage;                    // 1, 2, 3
};

constexpr int kEngineThreads = 128;
constexpr int kEngineBlocksPerSM = 3;
constexpr int kEngine1DCells = kEngineThreads - 1;
constexpr int kEngineTX = 16, kEngineTY = 15;  // two x- and two y-faces per thread
size_t engine_smem_bytes();
long long engine_tiles_of(int ndim, long long nx, long long ny);
cudaError_t engine_prepare();  // kernel attributes; call before capturing
cudaError_t launch_engine_stage(const EngineArgs &e, int grid, cudaStream_t s);

// Tensor map of a 2D stage input U [nbatch][4][ny][nx] as a 3D tensor
// (x, y, plane of a problem) with a box of bw x bh x 4 doubles; false when a
// tiled copy cannot address it (nx odd: rows are not multiples of 16 bytes;
// U not 16-byte aligned; the grid smaller than the box; no encoder in the
// driver), and the launch then stages with plain loads.
bool encode_state_map(const double *U, long long nbatch, long long ny, long long nx, int bw,
                      int bh, CUtensorMap *out);

cudaError_t launch_alpha(const AlphaArgs &a, cudaStream_t s);
cudaError_t launch_stage(const StageArgs &a, cudaStream_t s);
// The same for a.order_r = 2, 4, 5 (FP64 reconstruction only).
cudaError_t launch_stage_orders(const StageArgs &a, cudaStream_t s);
// alpha bits -> doubles, and the CFL dt per problem
cudaError_t launch_alpha_export(const AlphaArgs &a, const unsigned long long *bits, double *alpha,
                                double *dt, cudaStream_t s);
cudaError_t launch_fill(double *p, long long n, double v, cudaStream_t s);
// Rows [j0, j0 + nr) of every problem and component of a 2D state
// [nbatch][nc][ny][nx] into a contiguous [nbatch][nc][nr][nx] buffer.
cudaError_t launch_pack_rows(const double *U, long long nbatch, int nc, long long ny, long long nx,
                             long long j0, long long nr, double *out, cudaStream_t s);

// Maximiser of the Buckley-Leverett speed f' on [0, 1].
double bl_speed_argmax();

// Message returned by weno_last_error() on the calling thread.
void set_last_error(const char *msg);
inline void set_last_error(const std::string &msg) { set_last_error(msg.c_str()); }

}  // namespace weno
