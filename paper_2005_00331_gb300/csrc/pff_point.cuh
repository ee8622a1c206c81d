// pff_point.cuh -- bookkeeping shared by the one-thread-per-point kernels of libpff (internal):
// launch shape helpers, the cell / Gauss point / tile index of a point, shape functions and the
// evaluation of nodal fields at a point.
#pragma once
#include "pff_common.cuh"
#include "pff_kernels.h"

namespace pff {

namespace {

constexpr int BLK = 256;
constexpr double RS2 = 0.70710678118654752440;

inline unsigned grid_for(long long n, int blk = BLK) {
  long long g = (n + blk - 1) / blk;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int DIM>
__host__ __device__ constexpr int ipow(int b) { return DIM == 2 ? b * b : b * b * b; }

// Cell, quadrature-point and tile bookkeeping shared by the direct (one thread per point) kernels.
template <int DIM, int P>
struct CellQP {
  int c[3], q[3];
  long long tile, qidx;
  __device__ void set(long long cell, int qq, const Geom& g) {
    constexpr int n = P + 1;
    c[0] = int(cell % g.N);
    c[1] = int((cell / g.N) % g.N);
    c[2] = DIM == 3 ? int(cell / ((long long)g.N * g.N)) : 0;
    q[0] = qq % n;
    q[1] = (qq / n) % n;
    q[2] = DIM == 3 ? qq / (n * n) : 0;
    const int TX = TileCfg<DIM, P>::TX, TY = TileCfg<DIM, P>::TY, TZ = TileCfg<DIM, P>::TZ;
    const int tx = c[0] / TX, ty = c[1] / TY, tz = c[2] / TZ;
    const int lx = c[0] % TX, ly = c[1] % TY, lz = c[2] % TZ;
    tile = tx + (long long)g.ntile[0] * (ty + (long long)g.ntile[1] * tz);
    qidx = ((long long)(lz * n + q[2]) * g.qpy + (ly * n + q[1])) * g.qpx + (lx * n + q[0]);
  }
  __device__ long long node(int a, const Geom& g) const {
    constexpr int n = P + 1;
    const int ax = a % n, ay = (a / n) % n, az = DIM == 3 ? a / (n * n) : 0;
    const int gx = c[0] * P + ax;
    // a cell just below a cut slit uses the copies of the slit's nodes (its top face, x < 1/2)
    if (g.cut && (DIM == 2 ? (c[1] * P + ay == g.cut_row && ay == P) : (c[2] * P + az == g.cut_row && az == P)) &&
        gx < g.cut_x)
      return cut_copy(g, gx, DIM == 3 ? c[1] * P + ay : 0);
    long long nd = gx + (long long)g.n1 * (c[1] * P + ay);
    if (DIM == 3) nd += (long long)g.n1 * g.n1 * (c[2] * P + az);
    return nd;
  }
  // N_a and grad N_a at this point
  template <typename Real>
  __device__ void shape(int a, const Tab<Real>& tb, Real& N, Real dN[DIM]) const {
    constexpr int n = P + 1;
    const int aa[3] = {a % n, (a / n) % n, DIM == 3 ? a / (n * n) : 0};
    N = Real(1);
    for (int t = 0; t < DIM; ++t) dN[t] = Real(1);
    for (int s = 0; s < DIM; ++s) {
      const Real Sv = tb.S[q[s]][aa[s]], Dv = tb.D[q[s]][aa[s]];
      N *= Sv;
      for (int t = 0; t < DIM; ++t) dN[t] *= (t == s ? Dv : Sv);
    }
  }
  __device__ double jxw(const Tab<double>& tb) const {
    double w = tb.hd;
    for (int s = 0; s < DIM; ++s) w *= tb.W[q[s]];
    return w;
  }
};

// Evaluates a DoF vector (u, phi) at the point: grad u, phi, grad phi.
template <int DIM, int P>
__device__ void eval_state(const CellQP<DIM, P>& cq, const double* U, const Geom& g, const Tab<double>& tb,
                           double gu[DIM][DIM], double& ph, double gph[DIM]) {
  constexpr int NA = ipow<DIM>(P + 1);
  for (int k = 0; k < DIM; ++k)
    for (int j = 0; j < DIM; ++j) gu[k][j] = 0.0;
  ph = 0.0;
  for (int j = 0; j < DIM; ++j) gph[j] = 0.0;
  for (int a = 0; a < NA; ++a) {
    double N, dN[DIM];
    cq.shape(a, tb, N, dN);
    const long long nd = cq.node(a, g);
    for (int k = 0; k < DIM; ++k) {
      const double uk = U[k * g.nn + nd];
      for (int j = 0; j < DIM; ++j) gu[k][j] += uk * dN[j];
    }
    const double pv = U[DIM * g.nn + nd];
    ph += pv * N;
    for (int j = 0; j < DIM; ++j) gph[j] += pv * dN[j];
  }
}

// eval_state and the value of a scalar nodal field f at the point. In 2D the cell's node rows are first
// contracted along x (value and x-derivative weights of the point), then along y: 7 (p+1)^2 + 8 (p+1)
// FMAs instead of 9 (p+1)^2 FMAs and 3 (p+1)^2 shape products; in 3D one shape evaluation per node.
template <int DIM, int P>
__device__ void eval_state_scalar(const CellQP<DIM, P>& cq, const double* U, const double* f, const Geom& g,
                                  const Tab<double>& tb, double gu[DIM][DIM], double& ph, double gph[DIM],
                                  double& fv) {
  if constexpr (DIM == 2) {
    constexpr int n = P + 1;
    const int qx = cq.q[0], qy = cq.q[1];
    double u0s[n], u0d[n], u1s[n], u1d[n], ps[n], pd[n], fs[n];
    for (int ay = 0; ay < n; ++ay) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0, a5 = 0.0, a6 = 0.0;
      for (int ax = 0; ax < n; ++ax) {
        const long long nd = cq.node(ax + n * ay, g);
        const double Sv = tb.S[qx][ax], Dv = tb.D[qx][ax];
        const double v0 = U[nd], v1 = U[g.nn + nd], v2 = U[2 * g.nn + nd];
        a0 = fma(Sv, v0, a0);
        a1 = fma(Dv, v0, a1);
        a2 = fma(Sv, v1, a2);
        a3 = fma(Dv, v1, a3);
        a4 = fma(Sv, v2, a4);
        a5 = fma(Dv, v2, a5);
        a6 = fma(Sv, f[nd], a6);
      }
      u0s[ay] = a0; u0d[ay] = a1; u1s[ay] = a2; u1d[ay] = a3; ps[ay] = a4; pd[ay] = a5; fs[ay] = a6;
    }
    gu[0][0] = gu[0][1] = gu[1][0] = gu[1][1] = 0.0;
    ph = gph[0] = gph[1] = fv = 0.0;
    for (int ay = 0; ay < n; ++ay) {
      const double Sv = tb.S[qy][ay], Dv = tb.D[qy][ay];
      gu[0][0] = fma(Sv, u0d[ay], gu[0][0]);
      gu[0][1] = fma(Dv, u0s[ay], gu[0][1]);
      gu[1][0] = fma(Sv, u1d[ay], gu[1][0]);
      gu[1][1] = fma(Dv, u1s[ay], gu[1][1]);
      ph = fma(Sv, ps[ay], ph);
      gph[0] = fma(Sv, pd[ay], gph[0]);
      gph[1] = fma(Dv, ps[ay], gph[1]);
      fv = fma(Sv, fs[ay], fv);
    }
    return;
  }
  constexpr int NA = ipow<DIM>(P + 1);
  for (int k = 0; k < DIM; ++k)
    for (int j = 0; j < DIM; ++j) gu[k][j] = 0.0;
  ph = 0.0;
  fv = 0.0;
  for (int j = 0; j < DIM; ++j) gph[j] = 0.0;
  for (int a = 0; a < NA; ++a) {
    double N, dN[DIM];
    cq.shape(a, tb, N, dN);
    const long long nd = cq.node(a, g);
    for (int k = 0; k < DIM; ++k) {
      const double uk = U[k * g.nn + nd];
      for (int j = 0; j < DIM; ++j) gu[k][j] += uk * dN[j];
    }
    const double pv = U[DIM * g.nn + nd];
    ph += pv * N;
    for (int j = 0; j < DIM; ++j) gph[j] += pv * dN[j];
    fv += f[nd] * N;
  }
}

template <int DIM, int P>
__device__ double eval_scalar(const CellQP<DIM, P>& cq, const double* f, const Geom& g, const Tab<double>& tb) {
  if constexpr (DIM == 2) {  // contracted along x, then y
    constexpr int n = P + 1;
    double v = 0.0;
    for (int ay = 0; ay < n; ++ay) {
      double a = 0.0;
      for (int ax = 0; ax < n; ++ax) a = fma(tb.S[cq.q[0]][ax], f[cq.node(ax + n * ay, g)], a);
      v = fma(tb.S[cq.q[1]][ay], a, v);
    }
    return v;
  }
  constexpr int NA = ipow<DIM>(P + 1);
  double v = 0.0;
  for (int a = 0; a < NA; ++a) {
    double N, dN[DIM];
    cq.shape(a, tb, N, dN);
    v += f[cq.node(a, g)] * N;
  }
  return v;
}

}  // namespace

}  // namespace pff
