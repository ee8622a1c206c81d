// Explicit instantiations of the 3D Jacobian operator kernels, float arithmetic.
#include "pff_launch.h"
#include "pff_op.cuh"

namespace pff {

template <int P, int SPLIT>
static cudaError_t run_jac3(const float* x, float* y, const unsigned char* flags, const Geom& g, const Tab<float>& tb,
                             const float* qp, int mode, int inmask, int outmask, cudaStream_t s) {
  constexpr size_t smem = op3d_smem<P, float>();
  static bool attr = false;
  auto kern = k_op3d<P, float, float, PWJac<3, float, SPLIT>>;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  PWJac<3, float, SPLIT> pw;
  pw.qp = qp;
  pw.qpt = g.qpt;
  pw.tstride = (long long)qp_nv(3, SPLIT) * g.qpt;
  pw.mode = mode;
  OpArgs oa{inmask, outmask};
  const dim3 blk(Tile3<P>::QPX, Tile3<P>::QPY, Tile3<P>::TZ);
  if (g.ntiles > 0) return launch_k(kern, dim3((unsigned)g.ntiles), blk, smem, s, x, y, flags, g, tb, pw, oa);
  return cudaSuccess;
}

cudaError_t launch_jac_d3(int dim, int p, int split, const float* x, float* y, const unsigned char* flags, const Geom& g,
                       const Tab<float>& tb, const float* qp, int mode, int inmask, int outmask, cudaStream_t s) {
  if (dim != 3) return cudaErrorInvalidValue;
#define PFF_CASE(PP, SS) \
  if (p == PP && split == SS) return run_jac3<PP, SS>(x, y, flags, g, tb, qp, mode, inmask, outmask, s);
  PFF_CASE(1, 0) PFF_CASE(2, 0) PFF_CASE(3, 0) PFF_CASE(4, 0)
  PFF_CASE(1, 1) PFF_CASE(2, 1) PFF_CASE(3, 1) PFF_CASE(4, 1)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace pff
