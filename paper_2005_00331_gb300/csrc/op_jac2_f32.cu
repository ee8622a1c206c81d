// Explicit instantiations of the 2D Jacobian operator kernels, float arithmetic.
#include "pff_launch.h"
#include "pff_op.cuh"

namespace pff {

// CTAs of one kernel instantiation resident on the device at once (occupancy times SMs, queried once).
template <int P, int SPLIT, int RC, int CG, int ES>
static cudaError_t jac2_slots(long long* slots) {
  constexpr size_t smem = jac2_staged_smem<P, float, float, SPLIT, RC, CG, ES>();
  static int grid_per_sm = 0;
  auto kern = k_jac2_staged<P, float, float, SPLIT, RC, CG, ES>;
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
  *slots = (long long)sms * grid_per_sm;
  return cudaSuccess;
}

template <int P, int SPLIT, int RC, int CG, int ES = 0>
static cudaError_t run_jac2(const float* x, float* y, const unsigned char* flags, const Geom& g, const Tab<float>& tb,
                             const float* qp, int mode, int inmask, int outmask, cudaStream_t s,
                             const ChebEpi<float>& ce, const MatConst32& mc, const CgEpi<float>& cg) {
  constexpr size_t smem = jac2_staged_smem<P, float, float, SPLIT, RC, CG, ES>();
  long long grid = 0;
  cudaError_t e = jac2_slots<P, SPLIT, RC, CG, ES>(&grid);
  if (e != cudaSuccess) return e;
  if (grid > g.ntiles) grid = g.ntiles;
  const OpArgs oa = op_args(inmask, outmask, grid, g.ntile[0]);
  const dim3 blk(Tile2<P>::QPX, Tile2<P>::TY);
  if (grid > 0)
    return launch_k(k_jac2_staged<P, float, float, SPLIT, RC, CG, ES>, dim3((unsigned)grid), blk, smem, s, x, y, flags,
                    g, tb, qp, mode, oa, ce, mc, cg);
  return cudaSuccess;
}

// A Chebyshev step (stored tangent) on a level whose tiles fit one wave of the staged-epilogue kernel: that
// kernel (its copies also stage the step's operands) when they do, else the plain one.
template <int P, int SPLIT>
static cudaError_t run_cheb_step(const float* x, float* y, const unsigned char* flags, const Geom& g,
                                 const Tab<float>& tb, const float* qp, int mode, int inmask, int outmask, cudaStream_t s,
                                 const ChebEpi<float>& ce, const CgEpi<float>& cg) {
  long long slots = 0;
  cudaError_t e = jac2_slots<P, SPLIT, 0, 0, 1>(&slots);
  if (e != cudaSuccess) return e;
  if (g.ntiles <= slots)
    return run_jac2<P, SPLIT, 0, 0, 1>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, ce, MatConst32{}, cg);
  return run_jac2<P, SPLIT, 0, 0, 0>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, ce, MatConst32{}, cg);
}

cudaError_t launch_jac_d2(int dim, int p, int split, const float* x, float* y, const unsigned char* flags, const Geom& g,
                       const Tab<float>& tb, const float* qp, int mode, int inmask, int outmask, cudaStream_t s,
                       const ChebEpi<float>* ce, const Rc32* rc, const CgEpi<float>* cg) {
  ChebEpi<float> off{};
  off.on = 0;
  const ChebEpi<float>& e = ce ? *ce : off;
  const CgEpi<float> cg_off{};
  const CgEpi<float>& cgr = cg ? *cg : cg_off;
  if (dim != 2) return cudaErrorInvalidValue;
  // the CG-Lanczos epilogue and the recomputed tangent are separate instantiations, so that the plain
  // apply keeps its own code
  const bool cgo = cgr.on != 0;
#define PFF_CASE(PP, SS)                                                                                       \
  if (p == PP && split == SS) {                                                                                \
    if (rc && cgo) return run_jac2<PP, SS, 1, 1>(x, y, flags, g, tb, rc->state, mode, inmask, outmask, s, e, rc->mc, cgr); \
    if (rc) return run_jac2<PP, SS, 1, 0>(x, y, flags, g, tb, rc->state, mode, inmask, outmask, s, e, rc->mc, cgr);        \
    if (cgo) return run_jac2<PP, SS, 0, 1>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, e, MatConst32{}, cgr);        \
    if (e.on) return run_cheb_step<PP, SS>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, e, cgr);                     \
    return run_jac2<PP, SS, 0, 0>(x, y, flags, g, tb, qp, mode, inmask, outmask, s, e, MatConst32{}, cgr);                 \
  }
  PFF_CASE(1, 0) PFF_CASE(2, 0) PFF_CASE(3, 0) PFF_CASE(4, 0)
  PFF_CASE(1, 1) PFF_CASE(2, 1) PFF_CASE(3, 1) PFF_CASE(4, 1)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_cheb_seam<float>(const Geom& g, float* y, const ChebEpi<float>& ce, cudaStream_t s) {
  const long long n = (long long)(g.ntile[0] - 1 + g.ntile[1] - 1) * g.n1;
  if (n <= 0) return cudaSuccess;
  return launch_k(k_cheb_seam2<float>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, g, g.tdim[0] * g.p,
                  g.tdim[1] * g.p, y, ce);
}

}  // namespace pff
