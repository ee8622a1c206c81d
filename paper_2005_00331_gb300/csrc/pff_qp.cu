// pff_qp.cu -- per-point tangent and residual state of the Jacobian (k_qp_setup).
#include <cstdint>
#include <atomic>

#include "pff_kernels.h"
#include "pff_launch.h"
#include "pff_op.cuh"
#include "pff_point.cuh"

namespace pff {

// ===========================================================================================
// Per-point data of the Jacobian: tangent of g(phi~) sigma^+ + sigma^- (Sec. 2.1, 3.5), the
// coupling g'(phi) sigma^+ and the phase-field coefficients, times JxW (see qp_nv).
// part QP_ALL: everything. Miehe split, in two passes: QP_STRAIN (what depends on u only: the
// eigen-decomposition, the tangent, the phase-field coefficients, and sigma+ / E_s+ into sp64 for the
// residual), then QP_PHASE (the coupling g'(phi) sigma+ from sp64 and phi, after each phi change).
// FP32 and double-word copies of a per-point value (the FP32 copy is the double-word pair's high part:
// one FP64 -> FP32 rounding fewer).
__device__ __forceinline__ void store_lower(float* qp32, df64* qpdf, long long o, double v) {
  if (qpdf) {
    const df64 d = df_from(v);
    qpdf[o] = d;
    if (qp32) qp32[o] = d.hi;
  } else if (qp32) {
    qp32[o] = (float)v;
  }
}

template <int DIM, int P, int SPLIT>
__global__ void k_qp_setup(const double* __restrict__ U, const double* __restrict__ phit,
                           const double* __restrict__ gcf, const double* __restrict__ lamf,
                           const double* __restrict__ muf, Geom g, Tab<double> tb, MatConst mc,
                           double* __restrict__ qp64, float* __restrict__ qp32, df64* __restrict__ qpdf,
                           double* __restrict__ st64, double* __restrict__ sp64, int part) {
  constexpr int NQ = ipow<DIM>(P + 1);
  constexpr int NM = Mandel<DIM>::NM;
  constexpr int NV = qp_nv(DIM, SPLIT);
  const long long ncell = DIM == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= ncell * NQ) return;
  CellQP<DIM, P> cq;
  cq.set(t / NQ, int(t % NQ), g);
  // the state passes evaluate U and phi~ together (one shape evaluation per node)
  const bool state_pass = qp64 && !(SPLIT == 1 && part == QP_PHASE);
  double gu[DIM][DIM], ph, gph[DIM], pt;
  if (state_pass) eval_state_scalar<DIM, P>(cq, U, phit, g, tb, gu, ph, gph, pt);
  else pt = eval_scalar<DIM, P>(cq, phit, g, tb);
  const double gc = gcf ? eval_scalar<DIM, P>(cq, gcf, g, tb) : mc.gc;
  const double lam = lamf ? eval_scalar<DIM, P>(cq, lamf, g, tb) : mc.lambda;
  const double mu = muf ? eval_scalar<DIM, P>(cq, muf, g, tb) : mc.mu;
  const double gt = deg_g(pt, mc.kappa);
  if (st64) {
    const long long sb = cq.tile * ST_NV * g.qpt + cq.qidx;
    st64[sb] = gt;
    st64[sb + g.qpt] = gc;
    st64[sb + 2 * g.qpt] = lam;
    st64[sb + 3 * g.qpt] = mu;
  }
  if (!qp64) return;  // residual state only (it does not depend on U)
  const double jxw = cq.jxw(tb);
  const long long base = cq.tile * NV * g.qpt + cq.qidx;
  if (SPLIT == 1 && part == QP_PHASE) {
    const double dgp = deg_dg(eval_scalar<DIM, P>(cq, U + DIM * g.nn, g, tb), mc.kappa);
    const double* sp = sp64 + cq.tile * (NM + 1) * g.qpt + cq.qidx;
    constexpr int OB = NM * (NM + 1) / 2;
    for (int m = 0; m < NM; ++m) {
      const double v = dgp * sp[m * g.qpt] * jxw;
      const long long o = base + (OB + m) * g.qpt;
      qp64[o] = v;
      store_lower(qp32, qpdf, o, v);
    }
    return;
  }
  const double dgp = deg_dg(ph, mc.kappa), ddg = deg_ddg(mc.kappa);

  double e[DIM][DIM], tr = 0.0;
  for (int i = 0; i < DIM; ++i) {
    for (int j = 0; j < DIM; ++j) e[i][j] = 0.5 * (gu[i][j] + gu[j][i]);
    tr += e[i][i];
  }
  double em[NM];
  for (int m = 0; m < NM; ++m) {
    const int i = Mandel<DIM>::ia(m), j = Mandel<DIM>::ib(m);
    em[m] = (i == j) ? e[i][i] : e[i][j] / RS2;
  }
  double vals[NV];
  if constexpr (SPLIT == 0) {
    double ee = 0.0;
    for (int m = 0; m < NM; ++m) ee += em[m] * em[m];
    const double Es = 0.5 * lam * tr * tr + mu * ee;
    vals[0] = gt * lam * jxw;
    vals[1] = gt * mu * jxw;
    for (int m = 0; m < NM; ++m) vals[2 + m] = dgp * (2.0 * mu * em[m] + (m < DIM ? lam * tr : 0.0)) * jxw;
    vals[2 + NM] = (ddg * Es + gc / mc.eps) * jxw;
    vals[3 + NM] = gc * mc.eps * jxw;
  } else {
    double Pp[NM][NM], epm[NM], H, trp, Esp;  // P+ (upper triangle), e+ (Mandel), H(tr), <tr>+, E_s+
    if constexpr (DIM == 2) {
      // Closed form in the eigen-angle t of e: (c2, s2) = (cos 2t, sin 2t), l1,2 = m +- r. With the
      // orthonormal Mandel vectors u = I / sqrt2, w = R / sqrt2, z = J / sqrt2 (R, J as in the FP32 tangent),
      // E_11 = (u + w) / sqrt2, E_22 = (u - w) / sqrt2 and E_12 = z, so
      // P+ = Hs (u u^T + w w^T) + Hd (u w^T + w u^T) + theta z z^T, Hs,d = (H(l1) +- H(l2)) / 2, and
      // e+ = Ep I + Em R, Ep,m = (<l1>+ +- <l2>+) / 2. No eigenvector and one reciprocal square root.
      const double m = 0.5 * (e[0][0] + e[1][1]), dd = 0.5 * (e[0][0] - e[1][1]), b = e[0][1];
      const double r2 = fma(dd, dd, b * b);
      double r = 0.0, c2 = 1.0, s2 = 0.0;  // a degenerate pair keeps the coordinate axes, as eig_sym2
      if (r2 > 0.0) {
        const double ir = rsqrt(r2);
        r = r2 * ir;
        c2 = dd * ir;
        s2 = b * ir;
      }
      double l[2] = {m + r, m - r};
      double trs = tr;
      snap_zero<2>(l, trs);
      H = heav(trs);
      trp = pos(trs);
      const double p1 = pos(l[0]), p2 = pos(l[1]);
      Esp = 0.5 * lam * trp * trp + mu * (p1 * p1 + p2 * p2);
      const double th = theta_dd(l[0], l[1]);
      const double Hs = 0.5 * (heav(l[0]) + heav(l[1])), Hd = 0.5 * (heav(l[0]) - heav(l[1]));
      const double cc = c2 * c2, ss = s2 * s2, cs = c2 * s2;
      Pp[0][0] = 0.5 * Hs * (1.0 + cc) + Hd * c2 + 0.5 * th * ss;
      Pp[0][1] = 0.5 * Hs * (1.0 - cc) - 0.5 * th * ss;
      Pp[0][2] = RS2 * (Hs * cs + Hd * s2 - th * cs);
      Pp[1][1] = 0.5 * Hs * (1.0 + cc) - Hd * c2 + 0.5 * th * ss;
      Pp[1][2] = RS2 * (Hd * s2 + th * cs - Hs * cs);
      Pp[2][2] = Hs * ss + th * cc;
      const double Ep = 0.5 * (p1 + p2), Em = 0.5 * (p1 - p2);
      epm[0] = Ep + Em * c2;
      epm[1] = Ep - Em * c2;
      epm[2] = 1.4142135623730951 * Em * s2;
    } else {
      double l[DIM], V[DIM][DIM];
      eig_sym<DIM>(e, l, V);
      double trs = tr;
      snap_zero<DIM>(l, trs);
      H = heav(trs);
      trp = pos(trs);
      double sl2 = 0.0;
      for (int t2 = 0; t2 < DIM; ++t2) sl2 += pos(l[t2]) * pos(l[t2]);
      Esp = 0.5 * lam * trp * trp + mu * sl2;
      // P+ = sum_i H(l_i) E_ii E_ii^T + sum_{i<j} theta_ij E_ij E_ij^T (orthonormal Mandel basis)
      for (int a = 0; a < NM; ++a)
        for (int b = 0; b < NM; ++b) Pp[a][b] = 0.0;
      for (int mm = 0; mm < NM; ++mm) epm[mm] = 0.0;
      for (int i = 0; i < DIM; ++i) {
        for (int j = i; j < DIM; ++j) {
          double vi[DIM], vj[DIM], Em[NM];
          for (int k = 0; k < DIM; ++k) {
            vi[k] = V[k][i];
            vj[k] = V[k][j];
          }
          mandel_dyad<DIM>(vi, vj, i == j, Em);
          const double th = (i == j) ? heav(l[i]) : theta_dd(l[i], l[j]);
          for (int a = 0; a < NM; ++a)  // upper triangle (the tangent below reads b >= a)
            for (int b = a; b < NM; ++b) Pp[a][b] += th * Em[a] * Em[b];
          if (i == j)
            for (int mm = 0; mm < NM; ++mm) epm[mm] += pos(l[i]) * Em[mm];
        }
      }
    }
    const double aH = gt * H + 1.0 - H;
    int o = 0;
    for (int a = 0; a < NM; ++a)
      for (int b = a; b < NM; ++b) {
        double Cab = 2.0 * mu * ((a == b ? 1.0 : 0.0) + (gt - 1.0) * Pp[a][b]);
        if (a < DIM && b < DIM) Cab += lam * aH;
        vals[o++] = Cab * jxw;
      }
    for (int m = 0; m < NM; ++m) {
      const double spm = 2.0 * mu * epm[m] + (m < DIM ? lam * trp : 0.0);
      vals[o + m] = dgp * spm * jxw;
      if (part == QP_STRAIN) sp64[cq.tile * (NM + 1) * g.qpt + m * g.qpt + cq.qidx] = spm;
    }
    vals[o + NM] = (ddg * Esp + gc / mc.eps) * jxw;
    vals[o + NM + 1] = gc * mc.eps * jxw;
    if (part == QP_STRAIN) sp64[cq.tile * (NM + 1) * g.qpt + NM * g.qpt + cq.qidx] = Esp;
  }
  // QP_STRAIN leaves the coupling entries to the phase pass
  constexpr int OB = SPLIT == 1 ? NM * (NM + 1) / 2 : 2;
  for (int v = 0; v < NV; ++v) {
    if (SPLIT == 1 && part == QP_STRAIN && v >= OB && v < OB + NM) continue;
    qp64[base + v * g.qpt] = vals[v];
    store_lower(qp32, qpdf, base + v * g.qpt, vals[v]);
  }
}

cudaError_t launch_qp_setup(int dim, int p, int split, const double* U, const double* phit, const double* gcf,
                            const double* lamf, const double* muf, const Geom& g, const Tab<double>& tb,
                            const MatConst& mc, double* qp64, float* qp32, df64* qpdf, double* st64, cudaStream_t s,
                            double* sp64, int part) {
  const long long ncell = dim == 2 ? (long long)g.N * g.N : (long long)g.N * g.N * g.N;
  const long long tot = ncell * (dim == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1));
  const unsigned gr = grid_for(tot, 128);
#define PFF_CASE(DD, PP, SS)                                                                          \
  if (dim == DD && p == PP && split == SS) {                                                          \
    count_launch(); k_qp_setup<DD, PP, SS><<<gr, 128, 0, s>>>(U, phit, gcf, lamf, muf, g, tb, mc, qp64, qp32, qpdf, st64, sp64, part); \
    return cudaGetLastError();                                                                        \
  }
  PFF_CASE(2, 1, 0) PFF_CASE(2, 2, 0) PFF_CASE(2, 3, 0) PFF_CASE(2, 4, 0)
  PFF_CASE(2, 1, 1) PFF_CASE(2, 2, 1) PFF_CASE(2, 3, 1) PFF_CASE(2, 4, 1)
  PFF_CASE(3, 1, 0) PFF_CASE(3, 2, 0) PFF_CASE(3, 3, 0) PFF_CASE(3, 4, 0)
  PFF_CASE(3, 1, 1) PFF_CASE(3, 2, 1) PFF_CASE(3, 3, 1) PFF_CASE(3, 4, 1)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

}  // namespace pff
