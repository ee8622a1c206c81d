// Explicit instantiations of the 2D Jacobian operator kernels, double arithmetic.
#include "pff_launch.h"
#include "pff_op.cuh"

namespace pff {

template <int P, int SPLIT, int CG>
static cudaError_t run_jac2(const double* x, double* y, const unsigned char* flags, const Geom& g, const Tab<double>& tb,
                             const double* qp, int mode, int inmask, int outmask, cudaStream_t s,
                             const ChebEpi<double>& ce, const CgEpi<double>& cg) {
  constexpr size_t smem = jac2_staged_smem<P, double, double, SPLIT, 0, CG>();
  static int grid_per_sm = 0;
  auto kern = k_jac2_staged<P, double, double, SPLIT, 0, CG>;
  if (!grid_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&grid_per_sm, kern, Tile2<P>::NT, smem);
    if (e != cudaSuccess) return e;
    if (grid_per_sm < 1) grid_per_sm = 1;
  }
  int sms = 152;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  long long grid = (long long)sms * grid_per_sm;
  if (grid > g.ntiles) grid = g.ntiles;
  const OpArgs oa = op_args(inmask, outmask, grid, g.ntile[0]);
  const dim3 blk(Tile2<P>::QPX, Tile2<P>::TY);
  if (grid > 0) return launch_k(kern, dim3((unsigned)grid), blk, smem, s, x, y, flags, g, tb, qp, mode, oa, ce, MatConst32{}, cg);
  return cudaSuccess;
}

cudaError_t launch_jac_d2(int dim, int p, int split, const double* x, double* y, const unsigned char* flags, const Geom& g,
                       const Tab<double>& tb, const double* qp, int mode, int inmask, int outmask, cudaStream_t s,
                       const ChebEpi<double>* ce, const CgEpi<double>* cg) {
  ChebEpi<double> off{};
  off.on = 0;
  const ChebEpi<double>& e = ce ? *ce : off;
  const CgEpi<double> cg_off{};
  const CgEpi<double>& cgr = cg ? *cg : cg_off;
  if (dim != 2) return cudaErrorInvalidValue;
#define PFF_CASE(PP, SS) \
  if (p == PP && split == SS)                                                                               \
    return cgr.on ? run_jac2<PP, SS, 1>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, e, cgr)                         \
                  : run_jac2<PP, SS, 0>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, e, cgr);
  PFF_CASE(1, 0) PFF_CASE(2, 0) PFF_CASE(3, 0) PFF_CASE(4, 0)
  PFF_CASE(1, 1) PFF_CASE(2, 1) PFF_CASE(3, 1) PFF_CASE(4, 1)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_cheb_seam<double>(const Geom& g, double* y, const ChebEpi<double>& ce, cudaStream_t s) {
  const long long n = (long long)(g.ntile[0] - 1 + g.ntile[1] - 1) * g.n1;
  if (n <= 0) return cudaSuccess;
  return launch_k(k_cheb_seam2<double>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, g, g.tdim[0] * g.p,
                  g.tdim[1] * g.p, y, ce);
}

}  // namespace pff
