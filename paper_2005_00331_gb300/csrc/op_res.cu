// Explicit instantiations of the residual operator kernels (FP64), 2D and 3D.
#include "pff_launch.h"
#include "pff_op.cuh"

namespace pff {

template <int DIM, int P, int SPLIT>
static cudaError_t run_res(const double* U, double* r, const unsigned char* flags, const Geom& g,
                           const Tab<double>& tb, const double* st, const double* sp, double eps, double kappa,
                           int outmask, cudaStream_t s) {
  size_t smem;
  if constexpr (DIM == 2) smem = op2d_smem<P, double>();
  else smem = op3d_smem<P, double>();
  static bool attr = false;
  void (*kern)(const double*, double*, const unsigned char*, Geom, Tab<double>, PWRes<DIM, SPLIT>, OpArgs);
  if constexpr (DIM == 2) kern = k_op2d<P, double, double, PWRes<2, SPLIT>>;
  else kern = k_op3d<P, double, double, PWRes<3, SPLIT>>;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  PWRes<DIM, SPLIT> pw;
  pw.st = st;
  pw.sp = SPLIT ? sp : nullptr;
  pw.qpt = g.qpt;
  pw.tstride = (long long)ST_NV * g.qpt;
  pw.qpx = g.qpx;
  pw.qpy = g.qpy;
  pw.n = P + 1;
  for (int q = 0; q < MAXN; ++q) pw.W[q] = tb.W[q];
  pw.hd = tb.hd;
  pw.eps = eps;
  pw.kappa = kappa;
  OpArgs oa{IN_RAW, outmask};
  dim3 blk(Tile3<P>::QPX, Tile3<P>::QPY, Tile3<P>::TZ);
  if constexpr (DIM == 2) blk = dim3(Tile2<P>::QPX, Tile2<P>::TY);
  if (g.ntiles > 0) { count_launch(); kern<<<(unsigned)g.ntiles, blk, smem, s>>>(U, r, flags, g, tb, pw, oa); }
  return cudaGetLastError();
}

cudaError_t launch_res(int dim, int p, int split, const double* U, double* r, const unsigned char* flags,
                       const Geom& g, const Tab<double>& tb, const double* st, const double* sp, double eps,
                       double kappa, cudaStream_t s, int outmask) {
  if (outmask != OUT_ZERO_DIRICHLET && outmask != OUT_RAW) return cudaErrorInvalidValue;
#define PFF_CASE(DD, PP, SS)                    \
  if (dim == DD && p == PP && split == SS)      \
    return run_res<DD, PP, SS>(U, r, flags, g, tb, st, sp, eps, kappa, outmask, s);
  PFF_CASE(2, 1, 0) PFF_CASE(2, 2, 0) PFF_CASE(2, 3, 0) PFF_CASE(2, 4, 0)
  PFF_CASE(2, 1, 1) PFF_CASE(2, 2, 1) PFF_CASE(2, 3, 1) PFF_CASE(2, 4, 1)
  PFF_CASE(3, 1, 0) PFF_CASE(3, 2, 0) PFF_CASE(3, 3, 0) PFF_CASE(3, 4, 0)
  PFF_CASE(3, 1, 1) PFF_CASE(3, 2, 1) PFF_CASE(3, 3, 1) PFF_CASE(3, 4, 1)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_jac(int dim, int p, int split, const double* x, double* y, const unsigned char* flags,
                       const Geom& g, const Tab<double>& tb, const double* qp, int mode, int inmask, int outmask,
                       cudaStream_t s, const ChebEpi<double>* ce, const CgEpi<double>* cg) {
  return dim == 2 ? launch_jac_d2(dim, p, split, x, y, flags, g, tb, qp, mode, inmask, outmask, s, ce, cg)
                  : launch_jac_d3(dim, p, split, x, y, flags, g, tb, qp, mode, inmask, outmask, s);
}
cudaError_t launch_jac(int dim, int p, int split, const float* x, float* y, const unsigned char* flags,
                       const Geom& g, const Tab<float>& tb, const float* qp, int mode, int inmask, int outmask,
                       cudaStream_t s, const ChebEpi<float>* ce, const Rc32* rc, const CgEpi<float>* cg) {
  return dim == 2 ? launch_jac_d2(dim, p, split, x, y, flags, g, tb, qp, mode, inmask, outmask, s, ce, rc, cg)
                  : launch_jac_d3(dim, p, split, x, y, flags, g, tb, qp, mode, inmask, outmask, s);
}

}  // namespace pff
