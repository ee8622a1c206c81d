// pff_pgrad.cu -- parameter gradients of the residual (nodal G_c, lambda, mu).
#include <cstdint>
#include <atomic>

#include "pff_kernels.h"
#include "pff_launch.h"
#include "pff_op.cuh"
#include "pff_point.cuh"

namespace pff {

// ===========================================================================================
// Parameter gradients: per point the partial derivatives of the residual's pointwise terms with
// respect to G_c, lambda, mu, contracted with the test function v; then integrated against N_a.
template <int DIM, int P, int SPLIT>
__global__ void k_pgrad_qp(const double* __restrict__ U, const double* __restrict__ v,
                           const double* __restrict__ st64, Geom g, Tab<double> tb, MatConst mc,
                           double* __restrict__ tmp) {
  constexpr int NQ = ipow<DIM>(P + 1);
  const long long ncell = DIM == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncell * NQ) return;
  CellQP<DIM, P> cq;
  cq.set(t / NQ, int(t % NQ), g);
  double gu[DIM][DIM], ph, gph[DIM], gv[DIM][DIM], vph, gvph[DIM];
  eval_state<DIM, P>(cq, U, g, tb, gu, ph, gph);
  eval_state<DIM, P>(cq, v, g, tb, gv, vph, gvph);
  const double gt = st64[cq.tile * ST_NV * g.qpt + cq.qidx];
  const double jxw = cq.jxw(tb);
  const double dgp = deg_dg(ph, mc.kappa);
  double e[DIM][DIM], tr = 0.0, divv = 0.0;
  for (int i = 0; i < DIM; ++i) {
    for (int j = 0; j < DIM; ++j) e[i][j] = 0.5 * (gu[i][j] + gu[j][i]);
    tr += e[i][i];
    divv += gv[i][i];
  }
  double gpgv = 0.0;
  for (int j = 0; j < DIM; ++j) gpgv += gph[j] * gvph[j];
  const double s_gc = -(1.0 - ph) / mc.eps * vph + mc.eps * gpgv;
  double ep[DIM][DIM];
  double trp;
  if constexpr (SPLIT == 0) {
    trp = tr;
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) ep[i][j] = e[i][j];
  } else {
    double l[DIM], V[DIM][DIM];
    eig_sym<DIM>(e, l, V);
    double trs = tr;
    snap_zero<DIM>(l, trs);
    trp = pos(trs);
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        double s = 0.0;
        for (int k = 0; k < DIM; ++k) s += pos(l[k]) * V[i][k] * V[j][k];
        ep[i][j] = s;
      }
  }
  // lambda: sigma+ = trp I, sigma- = (tr - trp) I, E+ = trp^2/2
  const double s_lam = (gt * trp + (tr - trp)) * divv + dgp * 0.5 * trp * trp * vph;
  // mu: sigma+ = 2 e+, sigma- = 2 (e - e+), E+ = e+ : e+
  double s_mu = 0.0, epep = 0.0;
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      s_mu += (gt * 2.0 * ep[i][j] + 2.0 * (e[i][j] - ep[i][j])) * gv[i][j];
      epep += ep[i][j] * ep[i][j];
    }
  s_mu += dgp * epep * vph;
  tmp[t] = s_gc * jxw;
  tmp[ncell * NQ + t] = s_lam * jxw;
  tmp[2 * ncell * NQ + t] = s_mu * jxw;
}

template <int DIM, int P>
__global__ void k_pgrad_int(const double* __restrict__ tmp, Geom g, Tab<double> tb, double* __restrict__ o0,
                            double* __restrict__ o1, double* __restrict__ o2) {
  constexpr int NA = ipow<DIM>(P + 1), NQ = NA;
  const long long ncell = DIM == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncell * NA) return;
  const long long cell = t / NA;
  const int a = int(t % NA);
  double acc[3] = {0.0, 0.0, 0.0};
  CellQP<DIM, P> cq;
  long long nd = 0;
  for (int q = 0; q < NQ; ++q) {
    cq.set(cell, q, g);
    if (q == 0) nd = cq.node(a, g);
    double N, dN[DIM];
    cq.shape(a, tb, N, dN);
    for (int k = 0; k < 3; ++k) acc[k] += N * tmp[k * ncell * NQ + cell * NQ + q];
  }
  if (o0) atomicAdd(o0 + nd, acc[0]);
  if (o1) atomicAdd(o1 + nd, acc[1]);
  if (o2) atomicAdd(o2 + nd, acc[2]);
}

cudaError_t launch_param_grad(int dim, int p, int split, const double* U, const double* v, const double* st64,
                              const Geom& g, const Tab<double>& tb, const MatConst& mc, double* tmp,
                              double* out_gc, double* out_lam, double* out_mu, cudaStream_t s) {
  for (double* o : {out_gc, out_lam, out_mu}) {
    if (o) {
      cudaError_t e = cudaMemsetAsync(o, 0, sizeof(double) * g.nn, s);
      if (e != cudaSuccess) return e;
    }
  }
  const long long ncell = dim == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long tot = ncell * (dim == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1));
  const unsigned gr = grid_for(tot, 128);
  bool done = false;
#define PFF_CASE(DD, PP, SS)                                                                  \
  if (!done && dim == DD && p == PP && split == SS) {                                        \
    count_launch(); k_pgrad_qp<DD, PP, SS><<<gr, 128, 0, s>>>(U, v, st64, g, tb, mc, tmp);                   \
    count_launch(); k_pgrad_int<DD, PP><<<gr, 128, 0, s>>>(tmp, g, tb, out_gc, out_lam, out_mu);             \
    done = true;                                                                              \
  }
  PFF_CASE(2, 1, 0) PFF_CASE(2, 2, 0) PFF_CASE(2, 3, 0) PFF_CASE(2, 4, 0)
  PFF_CASE(2, 1, 1) PFF_CASE(2, 2, 1) PFF_CASE(2, 3, 1) PFF_CASE(2, 4, 1)
  PFF_CASE(3, 1, 0) PFF_CASE(3, 2, 0) PFF_CASE(3, 3, 0) PFF_CASE(3, 4, 0)
  PFF_CASE(3, 1, 1) PFF_CASE(3, 2, 1) PFF_CASE(3, 3, 1) PFF_CASE(3, 4, 1)
#undef PFF_CASE
  return done ? cudaGetLastError() : cudaErrorInvalidValue;
}

}  // namespace pff
