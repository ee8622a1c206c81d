// pff_diag.cu -- diagonal of the block-diagonal operator and dense coarse-level assembly.
#include <cstdint>
#include <atomic>

#include "pff_kernels.h"
#include "pff_launch.h"
#include "pff_op.cuh"
#include "pff_point.cuh"

namespace pff {

// ===========================================================================================
// Diagonal of diag(G_uu, G_phiphi): for a basis function N_a e_k the quadratic form
// e(N_a e_k) : C_eff : e(N_a e_k), and c N_a^2 + k |grad N_a|^2 for the phase field.
template <int DIM, int P, int SPLIT, typename Real>
__global__ void k_diagonal(const Real* __restrict__ qp, Geom g, Tab<Real> tb, Real* __restrict__ d) {
  constexpr int NA = ipow<DIM>(P + 1), NQ = NA;
  constexpr int NM = Mandel<DIM>::NM;
  constexpr int NV = qp_nv(DIM, SPLIT);
  constexpr int OFFB = SPLIT == 0 ? 2 : NM * (NM + 1) / 2;
  constexpr Real R2 = Real(RS2);
  const long long ncell = DIM == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncell * NA) return;
  const long long cell = t / NA;
  const int a = int(t % NA);
  Real acc[DIM + 1];
  for (int f = 0; f <= DIM; ++f) acc[f] = Real(0);
  CellQP<DIM, P> cq;
  long long nd = 0;
  for (int q = 0; q < NQ; ++q) {
    cq.set(cell, q, g);
    if (q == 0) nd = cq.node(a, g);
    Real N, dN[DIM];
    cq.shape(a, tb, N, dN);
    const Real* v = qp + cq.tile * NV * g.qpt + cq.qidx;
    for (int k = 0; k < DIM; ++k) {
      Real em[NM];
      for (int m = 0; m < NM; ++m) {
        const int i = Mandel<DIM>::ia(m), j = Mandel<DIM>::ib(m);
        if (i == j) em[m] = (i == k) ? dN[k] : Real(0);
        else em[m] = (i == k ? dN[j] : (j == k ? dN[i] : Real(0))) * R2;
      }
      Real val = Real(0);
      if constexpr (SPLIT == 0) {
        Real ee = Real(0);
        for (int m = 0; m < NM; ++m) ee += em[m] * em[m];
        val = v[0] * dN[k] * dN[k] + Real(2) * v[g.qpt] * ee;
      } else {
        for (int i = 0; i < NM; ++i)
          for (int j = i; j < NM; ++j) {
            const Real cij = v[sym_index(NM, i, j) * g.qpt];
            val += (i == j ? Real(1) : Real(2)) * cij * em[i] * em[j];
          }
      }
      acc[k] += val;
    }
    Real gg = Real(0);
    for (int j = 0; j < DIM; ++j) gg += dN[j] * dN[j];
    acc[DIM] += v[(OFFB + NM) * g.qpt] * N * N + v[(OFFB + NM + 1) * g.qpt] * gg;
  }
  for (int f = 0; f <= DIM; ++f) atomicAdd(d + f * g.nn + nd, acc[f]);
}

template <typename Real>
__global__ void k_diag_finish(long long n, long long nn, const unsigned char* __restrict__ flags, Real* __restrict__ d) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int f = int(e / nn);
  if ((flags[e % nn] >> f) & 1u) d[e] = Real(1);
}

template <typename Real>
cudaError_t launch_diagonal(int dim, int p, int split, const Real* qp, const unsigned char* flags, const Geom& g,
                            const Tab<Real>& tb, Real* d, cudaStream_t s) {
  const long long n = (dim + 1) * g.nn;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(Real) * n, s);
  if (e != cudaSuccess) return e;
  const long long ncell = dim == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long tot = ncell * (dim == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1));
  const unsigned gr = grid_for(tot, 128);
  bool done = false;
#define PFF_CASE(DD, PP, SS)                                                         \
  if (!done && dim == DD && p == PP && split == SS) {                               \
    count_launch(); k_diagonal<DD, PP, SS, Real><<<gr, 128, 0, s>>>(qp, g, tb, d);  \
    done = true;                                                                     \
  }
  PFF_CASE(2, 1, 0) PFF_CASE(2, 2, 0) PFF_CASE(2, 3, 0) PFF_CASE(2, 4, 0)
  PFF_CASE(2, 1, 1) PFF_CASE(2, 2, 1) PFF_CASE(2, 3, 1) PFF_CASE(2, 4, 1)
  PFF_CASE(3, 1, 0) PFF_CASE(3, 2, 0) PFF_CASE(3, 3, 0) PFF_CASE(3, 4, 0)
  PFF_CASE(3, 1, 1) PFF_CASE(3, 2, 1) PFF_CASE(3, 3, 1) PFF_CASE(3, 4, 1)
#undef PFF_CASE
  if (!done) return cudaErrorInvalidValue;
  count_launch(); k_diag_finish<Real><<<grid_for(n), BLK, 0, s>>>(n, g.nn, flags, d);
  return cudaGetLastError();
}
template cudaError_t launch_diagonal<double>(int, int, int, const double*, const unsigned char*, const Geom&,
                                             const Tab<double>&, double*, cudaStream_t);
template cudaError_t launch_diagonal<float>(int, int, int, const float*, const unsigned char*, const Geom&,
                                            const Tab<float>&, float*, cudaStream_t);


// ===========================================================================================
// Dense coarse operator: element matrices from the stored per-point data, one thread per
// (cell, test DoF, trial DoF), accumulated into the u-u, phi-phi and phi-u blocks.
template <int DIM, int P, int SPLIT>
__global__ void k_coarse_asm(const double* __restrict__ qp64, Geom g, Tab<double> tb, double* __restrict__ Au,
                             double* __restrict__ Ap, double* __restrict__ B) {
  constexpr int NA = ipow<DIM>(P + 1), NQ = NA, NL = (DIM + 1) * NA;
  const long long ncell = DIM == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncell * NL * NL) return;
  const long long cell = t / (NL * NL);
  const int i = int((t / NL) % NL), j = int(t % NL);
  const int fi = i / NA, a = i % NA, fj = j / NA, b = j % NA;
  if (fi < DIM && fj == DIM) return;  // G_uphi = 0
  PWJac<DIM, double, SPLIT> pw;
  pw.qp = qp64;
  pw.qpt = g.qpt;
  pw.tstride = (long long)qp_nv(DIM, SPLIT) * g.qpt;
  pw.mode = JM_FULL;
  CellQP<DIM, P> cq;
  double val = 0.0;
  long long na_ = 0, nb_ = 0;
  for (int q = 0; q < NQ; ++q) {
    cq.set(cell, q, g);
    if (q == 0) {
      na_ = cq.node(a, g);
      nb_ = cq.node(b, g);
    }
    double Na, dNa[DIM], Nb, dNb[DIM];
    cq.shape(a, tb, Na, dNa);
    cq.shape(b, tb, Nb, dNb);
    QPIn<DIM, double> in;
    for (int k = 0; k < DIM; ++k)
      for (int m = 0; m < DIM; ++m) in.gu[k][m] = (k == fj) ? dNb[m] : 0.0;
    in.ph = (fj == DIM) ? Nb : 0.0;
    for (int m = 0; m < DIM; ++m) in.gph[m] = (fj == DIM) ? dNb[m] : 0.0;
    QPOut<DIM, double> o;
    pw(cq.tile, cq.qidx, in, o);
    if (fi < DIM) {
      for (int m = 0; m < DIM; ++m) val += o.cu[fi][m] * dNa[m];
    } else {
      val += o.cv * Na;
      for (int m = 0; m < DIM; ++m) val += o.cg[m] * dNa[m];
    }
  }
  const long long nn = g.nn, nu = DIM * nn;
  if (fi < DIM && fj < DIM) atomicAdd(Au + (fi * nn + na_) * nu + (fj * nn + nb_), val);
  else if (fi == DIM && fj == DIM) atomicAdd(Ap + na_ * nn + nb_, val);
  else atomicAdd(B + na_ * nu + (fj * nn + nb_), val);
}

__global__ void k_coarse_mask(int dim, long long nn, const unsigned char* __restrict__ flags, double* Au, double* Ap,
                              double* B) {
  const long long nu = dim * nn;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // rows/cols of Au
  if (t < nu * nu) {
    const long long r = t / nu, c = t % nu;
    const bool mr = (flags[r % nn] >> (r / nn)) & 1u, mc = (flags[c % nn] >> (c / nn)) & 1u;
    if (mr || mc) Au[t] = (r == c) ? 1.0 : 0.0;
  }
  if (t < nn * nn) {
    const long long r = t / nn, c = t % nn;
    const bool mr = (flags[r] >> dim) & 1u, mc = (flags[c] >> dim) & 1u;
    if (mr || mc) Ap[t] = (r == c) ? 1.0 : 0.0;
  }
  if (t < nn * nu) {
    const long long r = t / nu, c = t % nu;
    const bool mr = (flags[r] >> dim) & 1u, mc = (flags[c % nn] >> (c / nn)) & 1u;
    if (mr || mc) B[t] = 0.0;
  }
}

cudaError_t launch_coarse_assemble(int dim, int p, int split, const double* qp64, const unsigned char* flags,
                                   const Geom& g, const Tab<double>& tb, double* Au, double* Ap, double* B,
                                   cudaStream_t s) {
  const long long nn = g.nn, nu = dim * nn;
  cudaError_t e;
  if ((e = cudaMemsetAsync(Au, 0, sizeof(double) * nu * nu, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(Ap, 0, sizeof(double) * nn * nn, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(B, 0, sizeof(double) * nn * nu, s)) != cudaSuccess) return e;
  const long long ncell = dim == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const int na = dim == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1);
  const long long nl = (dim + 1) * na;
  const unsigned gr = grid_for(ncell * nl * nl, 128);
  bool done = false;
#define PFF_CASE(DD, PP, SS)                                             \
  if (!done && dim == DD && p == PP && split == SS) {                   \
    count_launch(); k_coarse_asm<DD, PP, SS><<<gr, 128, 0, s>>>(qp64, g, tb, Au, Ap, B); \
    done = true;                                                         \
  }
  PFF_CASE(2, 1, 0) PFF_CASE(2, 2, 0) PFF_CASE(2, 3, 0) PFF_CASE(2, 4, 0)
  PFF_CASE(2, 1, 1) PFF_CASE(2, 2, 1) PFF_CASE(2, 3, 1) PFF_CASE(2, 4, 1)
  PFF_CASE(3, 1, 0) PFF_CASE(3, 2, 0) PFF_CASE(3, 3, 0) PFF_CASE(3, 4, 0)
  PFF_CASE(3, 1, 1) PFF_CASE(3, 2, 1) PFF_CASE(3, 3, 1) PFF_CASE(3, 4, 1)
#undef PFF_CASE
  if (!done) return cudaErrorInvalidValue;
  count_launch(); k_coarse_mask<<<grid_for(nu * nu), BLK, 0, s>>>(dim, nn, flags, Au, Ap, B);
  return cudaGetLastError();
}

}  // namespace pff
