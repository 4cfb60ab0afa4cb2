// weno_orders.cu -- stage launches of the central-upwind schemes of order
// 4, 8 and 10 (r = 2, 4, 5; the tables of the Appendix, weights of eqs.
// (16)-(22)).  A translation unit of its own so it compiles in parallel with
// the sixth-order kernels; the kernels are the templates of weno_tiles.cuh.
#include "weno_tiles.cuh"

namespace weno {
namespace {

template <bool AI, bool P1>
cudaError_t launch_r(const StageArgs &a, cudaStream_t s) {
  switch (a.order_r) {
    case 2: return launch_stage_t<AI, P1, 0, 2>(a, s);
    case 4: return launch_stage_t<AI, P1, 0, 4>(a, s);
    case 5: return launch_stage_t<AI, P1, 0, 5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_stage_orders(const StageArgs &a, cudaStream_t s) {
  const bool p1 = (a.p == 1.0);
  if (a.ai) return p1 ? launch_r<true, true>(a, s) : launch_r<true, false>(a, s);
  return p1 ? launch_r<false, true>(a, s) : launch_r<false, false>(a, s);
}

}  // namespace weno
