// Explicit instantiations of the 2D Jacobian operator kernels in double-word (float-float)
// arithmetic: FP64 vectors in global memory, per-point data as double-word pairs.
#include "pff_launch.h"
#include "pff_op.cuh"

namespace pff {

template <int P, int SPLIT, int CG>
static cudaError_t run_jac2_df(const double* x, double* y, const unsigned char* flags, const Geom& g, const Tab<df64>& tb,
                             const df64* qp, int mode, int inmask, int outmask, cudaStream_t s,
                             const ChebEpi<double>& ce, const CgEpi<double>& cg) {
  constexpr size_t smem = jac2_staged_smem<P, df64, double, SPLIT, 0, CG>();
  static int grid_per_sm = 0;
  auto kern = k_jac2_staged<P, df64, double, SPLIT, 0, CG>;
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

cudaError_t launch_jac_df(int dim, int p, int split, const double* x, double* y, const unsigned char* flags,
                          const Geom& g, const Tab<df64>& tb, const df64* qp, int mode, int inmask, int outmask,
                          cudaStream_t s, const ChebEpi<double>* ce, const CgEpi<double>* cg) {
  ChebEpi<double> off{};
  off.on = 0;
  const ChebEpi<double>& e = ce ? *ce : off;
  const CgEpi<double> cg_off{};
  const CgEpi<double>& cgr = cg ? *cg : cg_off;
  if (dim != 2) return cudaErrorInvalidValue;
#define PFF_CASE(PP, SS) \
  if (p == PP && split == SS)                                                                               \
    return cgr.on ? run_jac2_df<PP, SS, 1>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, e, cgr)                         \
                  : run_jac2_df<PP, SS, 0>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, e, cgr);
  PFF_CASE(1, 0) PFF_CASE(2, 0) PFF_CASE(3, 0) PFF_CASE(4, 0)
  PFF_CASE(1, 1) PFF_CASE(2, 1) PFF_CASE(3, 1) PFF_CASE(4, 1)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace pff
