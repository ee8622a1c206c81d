// pff_launch.h -- host-side launchers of the operator kernels (internal to libpff).
#pragma once
#include <cuda_runtime.h>
#include "pff_common.cuh"
#include "pff_df64.cuh"

namespace pff {

// Number of kernels launched by this library since it was loaded (all contexts).
void count_launch();
void add_launches(long long n);
long long launch_count();

#ifndef PFF_PDL
#define PFF_PDL 1
#endif
// Launch with programmatic stream serialisation (the kernel must begin with pdl_wait()); inside a
// captured graph this becomes a programmatic edge, so the launch work of the kernel overlaps the
// tail of its predecessor.
template <typename... KP, typename... A>
inline cudaError_t launch_k(void (*k)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = PFF_PDL;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KP>(args)...);
}

// y (+)= G x on one level from the stored per-point data (qp: [tile][nv][qpt]); y must be
// zeroed by the caller (seam nodes are accumulated atomically). mode: JM_*; masks: In/OutMask.
// With cg != nullptr (2D only) it is one step of the CG-Lanczos estimate (CgEpi).
// With ce != nullptr (2D only) the block-diagonal apply finishes a Chebyshev step on the nodes of a
// single tile (x and d updated in place) and accumulates only seam nodes into y; launch_cheb_seam
// then completes the step on the seam nodes.
cudaError_t launch_jac(int dim, int p, int split, const double* x, double* y, const unsigned char* flags,
                       const Geom& g, const Tab<double>& tb, const double* qp, int mode, int inmask,
                       int outmask, cudaStream_t s, const ChebEpi<double>* ce = nullptr,
                       const CgEpi<double>* cg = nullptr);
// FP32 Jacobian recomputed at the points from the nodal state (2D; see pw_jac_rc2): state = u_x, u_y,
// phi, phi~ as 4 blocks of g.nn floats, mc the material constants. Passed as `rc`, it replaces qp.
struct Rc32 {
  const float* state;
  MatConst32 mc;
};
cudaError_t launch_jac(int dim, int p, int split, const float* x, float* y, const unsigned char* flags,
                       const Geom& g, const Tab<float>& tb, const float* qp, int mode, int inmask, int outmask,
                       cudaStream_t s, const ChebEpi<float>* ce = nullptr, const Rc32* rc = nullptr,
                       const CgEpi<float>* cg = nullptr);
template <typename Store>
cudaError_t launch_cheb_seam(const Geom& g, Store* y, const ChebEpi<Store>& ce, cudaStream_t s);
cudaError_t launch_jac_d2(int dim, int p, int split, const double* x, double* y, const unsigned char* flags,
                          const Geom& g, const Tab<double>& tb, const double* qp, int mode, int inmask, int outmask,
                          cudaStream_t s, const ChebEpi<double>* ce, const CgEpi<double>* cg = nullptr);
cudaError_t launch_jac_d2(int dim, int p, int split, const float* x, float* y, const unsigned char* flags,
                          const Geom& g, const Tab<float>& tb, const float* qp, int mode, int inmask, int outmask,
                          cudaStream_t s, const ChebEpi<float>* ce, const Rc32* rc = nullptr,
                          const CgEpi<float>* cg = nullptr);
cudaError_t launch_jac_d3(int dim, int p, int split, const double* x, double* y, const unsigned char* flags,
                          const Geom& g, const Tab<double>& tb, const double* qp, int mode, int inmask, int outmask,
                          cudaStream_t s);
cudaError_t launch_jac_d3(int dim, int p, int split, const float* x, float* y, const unsigned char* flags,
                          const Geom& g, const Tab<float>& tb, const float* qp, int mode, int inmask, int outmask,
                          cudaStream_t s);
// The same Jacobian in double-word arithmetic (FP64 vectors, per-point data as df64 pairs); 2D.
cudaError_t launch_jac_df(int dim, int p, int split, const double* x, double* y, const unsigned char* flags,
                          const Geom& g, const Tab<df64>& tb, const df64* qp, int mode, int inmask, int outmask,
                          cudaStream_t s, const ChebEpi<double>* ce = nullptr, const CgEpi<double>* cg = nullptr);
cudaError_t launch_jac_df3(int dim, int p, int split, const double* x, double* y, const unsigned char* flags,
                           const Geom& g, const Tab<df64>& tb, const df64* qp, int mode, int inmask, int outmask,
                           cudaStream_t s);
// r = R(U) (FP64) from the per-point state st: [tile][4][qpt] = g(phi~), G_c, lambda, mu. With the
// Miehe split and sp != null, sigma+ and E_s+ per point are read from sp ([tile][NM + 1][qpt], the
// strain pass of the same u) instead of recomputing the eigen-decomposition. r must be zeroed by the
// caller. outmask: OUT_ZERO_DIRICHLET (Dirichlet rows 0) or OUT_RAW (every row, for reactions).
cudaError_t launch_res(int dim, int p, int split, const double* U, double* r, const unsigned char* flags,
                       const Geom& g, const Tab<double>& tb, const double* st, const double* sp, double eps,
                       double kappa, cudaStream_t s, int outmask = OUT_ZERO_DIRICHLET);

}  // namespace pff
