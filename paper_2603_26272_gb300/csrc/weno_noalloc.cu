// weno_noalloc.cu -- weno_rhs_noalloc: the right-hand side for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: a
// plug-in whose host application owns every device allocation, a control
// loop that must never enter the allocator (an allocation can synchronise the
// device or fail under memory pressure), or a caller holding a fixed memory
// budget.  They pass only their input U and their output dUdt.  The little
// scratch the right-hand side needs -- a status word and one slot of
// per-problem speed maxima -- lives here, in a file-scope device array of
// fixed size that exists on every GPU that loads this library, until the
// process exits.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current, and caches it; make
// that first call before any stream capture on that device.  Host code never
// uses the array's name as a pointer (on the host it is only a stand-in for
// the symbol).  Every call ends by synchronising its stream, to read the
// shared status word back.
//
// Sharing: every call on a device uses the same array.  Each call clears the
// parts that must start at zero; calls whose work overlaps on the GPU (on two
// streams, or from two threads) race on the array and must be serialised by
// the caller.
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/weno.h"
#include "weno_internal.h"

namespace {

constexpr size_t kScratchBytes = 64 * 1024;
constexpr size_t kStatusBytes = 256;  // weno::DevStatus, padded to the alignment
// nbatch limit: one slot of 8 u64 speed maxima per problem after the status word.
constexpr long long kMaxBatch = (long long)((kScratchBytes - kStatusBytes) / (8 * sizeof(unsigned long long)));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

weno_status say(weno_status s, const std::string &m) {
  weno::set_last_error(m);
  return s;
}

// Device address of the scratch array on the current device (set-up on first use).
weno_status scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return say(WENO_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return say(WENO_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return say(WENO_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return WENO_OK;
}

}  // namespace

extern "C" weno_status weno_rhs_noalloc(const weno_desc *d, const double *U, double *dUdt,
                                        void *stream) {
  // The descriptor and pointers are checked the same way as weno_rhs does.
  if (weno_workspace_bytes(d) == 0) return WENO_ERR_ARG;  // message set by the check
  if (!U || !dUdt) return say(WENO_ERR_ARG, "NULL array");
  if (U == dUdt) return say(WENO_ERR_ARG, "dUdt must not overlap U");
  if (d->nbatch > kMaxBatch)
    return say(WENO_ERR_ARG, "weno_rhs_noalloc: nbatch " + std::to_string(d->nbatch) +
                                 " exceeds its fixed scratch (at most " + std::to_string(kMaxBatch) +
                                 " problems); use weno_rhs with a workspace");
  void *base = nullptr;
  weno_status st = scratch_address(&base);
  if (st != WENO_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  weno::DevStatus *status = (weno::DevStatus *)base;
  unsigned long long *slot = (unsigned long long *)((char *)base + kStatusBytes);
  const size_t clear = kStatusBytes + (size_t)d->nbatch * 8 * sizeof(unsigned long long);
  cudaError_t e = cudaMemsetAsync(base, 0, clear, s);
  if (e != cudaSuccess) return say(WENO_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));

  const int nc = d->system == WENO_SYS_ADVECTION ? 1 : (d->ndim == 1 ? 3 : 4);
  const double dx = (d->x1 - d->x0) / (double)d->nx;
  const double dy = d->ndim == 2 ? (d->y1 - d->y0) / (double)d->ny : 1.0;

  weno::AlphaArgs a = {};
  a.system = d->system;
  a.ndim = d->ndim;
  a.nc = nc;
  a.alpha_single = d->alpha_mode == WENO_ALPHA_SINGLE;
  a.nbatch = d->nbatch;
  a.nx = d->nx;
  a.ny = d->ny;
  a.dx = dx;
  a.dy = dy;
  a.gamma = d->gamma;
  a.cfl = d->cfl;
  a.adv_speed = d->adv_speed;
  a.ustar = weno::bl_speed_argmax();
  a.U = U;
  a.alpha_out = slot;
  a.status = status;
  e = weno::launch_alpha(a, s);
  if (e != cudaSuccess) return say(WENO_ERR_CUDA, std::string("alpha launch: ") + cudaGetErrorString(e));

  weno::StageArgs r = {};
  r.system = d->system;
  r.ndim = d->ndim;
  r.nc = nc;
  r.nbatch = d->nbatch;
  r.nx = d->nx;
  r.ny = d->ny;
  r.dx = dx;
  r.dy = dy;
  r.bc_x = d->bc_x;
  r.bc_y = d->bc_y;
  r.gamma = d->gamma;
  r.cfl = d->cfl;
  r.eps = d->eps;
  r.mu0 = d->mu0;
  r.p = d->p;
  r.ai = d->ai;
  r.alpha_single = d->alpha_mode == WENO_ALPHA_SINGLE;
  r.precision = d->precision;
  r.order_r = d->order == 0 ? 3 : d->order / 2;
  r.ustar = weno::bl_speed_argmax();
  r.adv_speed = d->adv_speed;
  r.Uin = U;
  r.Uout = dUdt;
  r.mode = 1;
  r.stage = 4;
  r.alpha_in = slot;
  r.status = status;
  e = weno::launch_stage(r, s);
  if (e != cudaSuccess) return say(WENO_ERR_CUDA, std::string("rhs launch: ") + cudaGetErrorString(e));

  // Report a nonphysical input now: this entry point has no workspace the
  // caller could inspect later.
  weno::DevStatus h;
  e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return say(WENO_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
  if (h.code == 5) return say(WENO_ERR_TIMEOUT, "a tile's shared-memory copy did not complete");
  if (h.code != 0) {
    char buf[192];
    std::snprintf(buf, sizeof(buf), "nonphysical state in problem %lld, cell (j=%lld, i=%lld)", h.b,
                  h.j, h.i);
    return say(WENO_ERR_NONPHYSICAL, buf);
  }
  weno::set_last_error("");
  return WENO_OK;
}
