// pff_op.cuh -- cell-batched, sum-factorised operator kernels (2D and 3D).
//
// One CTA owns a tile of TX x TY (x TZ) cells. It stages the tile's node patch of every field
// in shared memory and evaluates the fields at all Gauss points of the tile with patch-wide 1D
// contractions (sum factorisation, Sec. 3.4 and its reference KrKo12): a node row shared by
// two cells is contracted once. A pointwise functor turns the evaluated source (gradients of
// the displacement components, phase-field value and gradient) into test coefficients; the
// transposed contractions integrate them back to the node patch. Nodes strictly inside the
// tile are written with plain stores; nodes on a seam between tiles are accumulated with
// atomics into an output the caller has zeroed. Rows masked on output (Dirichlet DoFs, the
// active set) are written once, by the tile that owns the node.
#pragma once
#include <type_traits>

#include "pff_common.cuh"
#include "pff_df64.cuh"

namespace pff {

// Gradient/value bundle handed to the pointwise functors.
template <int DIM, typename Real>
struct QPIn {
  Real gu[DIM][DIM];  // gu[k][j] = d u_k / d x_j
  Real ph;            // phase field value
  Real gph[DIM];      // phase field gradient
};
template <int DIM, typename Real>
struct QPOut {
  Real cu[DIM][DIM];  // coefficient of d w_k / d x_j in the u-test
  Real cv;            // coefficient of psi
  Real cg[DIM];       // coefficient of d psi / d x_j
};

// -------------------------------------------------------------------------------------------
// Pointwise Jacobian of Eq. (G) from stored per-point data (already multiplied by JxW).
// Full mode: u-test  tau = C_eff[e(du)],  phi-test  b : e(du) + c dphi,  k grad dphi;
// block-diagonal mode drops b : e(du); transpose mode moves the coupling to the u-test,
// tau += b dphi.
template <int DIM, typename Real, int SPLIT>
struct PWJac {
  const Real* qp;   // [tile][nv][qpt]
  long long tstride;
  long long qpt;
  int mode;
  __device__ __forceinline__ void operator()(long long tile, long long qi, const QPIn<DIM, Real>& in,
                                             QPOut<DIM, Real>& out) const {
    constexpr int NM = Mandel<DIM>::NM;
    constexpr Real RS2 = rconst<Real>(0.70710678118654752440);
    constexpr Real TWO = rconst<Real>(2.0);
    const Real* a = qp + tile * tstride + qi;
    Real em[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const int i = Mandel<DIM>::ia(m), j = Mandel<DIM>::ib(m);
      em[m] = (i == j) ? in.gu[i][i] : (in.gu[i][j] + in.gu[j][i]) * RS2;
    }
    Real tau[NM];
    int off;
    if constexpr (SPLIT == 0) {
      const Real gl = a[0], gm2 = TWO * a[qpt];
      Real tr = em[0];
#pragma unroll
      for (int t = 1; t < DIM; ++t) tr = tr + em[t];
      const Real gltr = gl * tr;
#pragma unroll
      for (int m = 0; m < NM; ++m) tau[m] = (m < DIM) ? fmac(gm2, em[m], gltr) : gm2 * em[m];
      off = 2;
    } else {
#pragma unroll
      for (int m = 0; m < NM; ++m) tau[m] = Real(0);
#pragma unroll
      for (int i = 0; i < NM; ++i) {
#pragma unroll
        for (int j = i; j < NM; ++j) {
          const Real cij = a[sym_index(NM, i, j) * qpt];
          tau[i] = fmac(cij, em[j], tau[i]);
          if (j != i) tau[j] = fmac(cij, em[i], tau[j]);
        }
      }
      off = NM * (NM + 1) / 2;
    }
    const Real c = a[(off + NM) * qpt], k = a[(off + NM + 1) * qpt];
    Real cv = c * in.ph;
    if (mode == JM_FULL) {
#pragma unroll
      for (int m = 0; m < NM; ++m) cv = fmac(a[(off + m) * qpt], em[m], cv);
    } else if (mode == JM_TRANSPOSE) {
#pragma unroll
      for (int m = 0; m < NM; ++m) tau[m] = fmac(a[(off + m) * qpt], in.ph, tau[m]);
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const int i = Mandel<DIM>::ia(m), j = Mandel<DIM>::ib(m);
      if (i == j) out.cu[i][i] = tau[m];
      else out.cu[i][j] = out.cu[j][i] = tau[m] * RS2;
    }
    out.cv = cv;
#pragma unroll
    for (int j = 0; j < DIM; ++j) out.cg[j] = k * in.gph[j];
  }
};

// -------------------------------------------------------------------------------------------
// Pointwise Jacobian of Eq. (G) in FP32, 2D, recomputed at the point from the nodal state instead of
// read from stored per-point data: st = (d u_x/dx, d u_x/dy, d u_y/dx, d u_y/dy, phi, phi~) at the
// point. With the eigenvalues l1 >= l2 of e = e(u) and the eigenvector angle t, R = v1 v1^T - v2 v2^T
// = [[cos 2t, sin 2t], [sin 2t, -cos 2t]] and J = v1 v2^T + v2 v1^T = [[-sin 2t, cos 2t], [cos 2t,
// sin 2t]]; a strain direction is e(du) = a I + b R + c J (a = tr/2, b = e(du):R/2, c = e(du):J/2) and
// the derivative of e+ (Alg. 2 in its divided-difference form) is diagonal in that basis:
//   de+[e(du)] = (H1 + H2)/2 (a I + b R) + (H1 - H2)/2 (b I + a R) + theta c J,
// theta = (l1+ - l2+)/(l1 - l2), H(l1) when l1 = l2. Then tau = lambda (g H(tr) + 1 - H(tr)) tr(e(du)) I
// + 2 mu (e(du) + (g(phi~) - 1) de+[e(du)]), the coupling g'(phi) sigma+ : e(du) with sigma+ =
// lambda <tr>+ I + 2 mu e+, and c = g'' E_s+ + G_c/eps, k = G_c eps, all times JxW. Eigenvalues and the
// trace within 1e-6 of the largest eigenvalue magnitude count as 0 (their sign is FP32 rounding).
// Split none: tau = g(phi~) (lambda tr(e(du)) I + 2 mu e(du)), sigma+ = sigma, E_s+ = E_s.
template <int SPLIT>
__device__ __forceinline__ void pw_jac_rc2(const float st[6], float jxw, const MatConst32& mc, int mode,
                                           const QPIn<2, float>& in, QPOut<2, float>& out) {
  const float exx = st[0], eyy = st[3], exy = 0.5f * (st[1] + st[2]);
  const float g = fmaf(mc.omk * st[5], st[5], mc.kappa), dg = 2.0f * mc.omk * st[4], ddg = 2.0f * mc.omk;
  const float dxx = in.gu[0][0], dyy = in.gu[1][1], dxy = 0.5f * (in.gu[0][1] + in.gu[1][0]);
  const float dtr = dxx + dyy;
  float txx, tyy, txy, sxx, syy, sxy, Esp;
  if constexpr (SPLIT == 0) {
    const float tr = exx + eyy;
    txx = g * fmaf(mc.lam, dtr, 2.0f * mc.mu * dxx);
    tyy = g * fmaf(mc.lam, dtr, 2.0f * mc.mu * dyy);
    txy = g * 2.0f * mc.mu * dxy;
    sxx = fmaf(mc.lam, tr, 2.0f * mc.mu * exx);
    syy = fmaf(mc.lam, tr, 2.0f * mc.mu * eyy);
    sxy = 2.0f * mc.mu * exy;
    Esp = 0.5f * mc.lam * tr * tr + mc.mu * (exx * exx + eyy * eyy + 2.0f * exy * exy);
  } else {
    float tr = exx + eyy;
    // half the eigenvalue gap r and its reciprocal from one rsqrt (no division): l1 - l2 = 2 r
    const float dd = 0.5f * (exx - eyy), r2 = fmaf(dd, dd, exy * exy);
    const float ir = r2 > 0.0f ? rsqrtf(r2) : 0.0f, r = r2 * ir;
    float l1 = 0.5f * tr + r, l2 = 0.5f * tr - r;
    const float tol = 1e-6f * fmaxf(fabsf(l1), fabsf(l2));
    if (fabsf(l1) <= tol) l1 = 0.0f;
    if (fabsf(l2) <= tol) l2 = 0.0f;
    if (fabsf(tr) <= tol) tr = 0.0f;
    const float c2 = r2 > 0.0f ? dd * ir : 1.0f, s2 = exy * ir;
    const float H1 = l1 >= 0.0f ? 1.0f : 0.0f, H2 = l2 >= 0.0f ? 1.0f : 0.0f, Ht = tr >= 0.0f ? 1.0f : 0.0f;
    const float p1 = fmaxf(l1, 0.0f), p2 = fmaxf(l2, 0.0f), trp = fmaxf(tr, 0.0f);
    // divided difference (p1 - p2) / (l1 - l2) with l1 - l2 = 2 r (a snapped eigenvalue moves it by at
    // most the snapping tolerance); H(l1) when the snapped eigenvalues coincide
    const float theta = l1 == l2 ? H1 : (p1 - p2) * (0.5f * ir);
    const float dm = dxx - dyy;
    const float a = 0.5f * dtr, b = 0.5f * fmaf(c2, dm, 2.0f * s2 * dxy), cj = 0.5f * fmaf(-s2, dm, 2.0f * c2 * dxy);
    const float Hs = 0.5f * (H1 + H2), Hd = 0.5f * (H1 - H2);
    const float A = fmaf(Hs, a, Hd * b), B = fmaf(Hd, a, Hs * b), T = theta * cj;
    const float pxx = A + B * c2 - T * s2, pyy = A - B * c2 + T * s2, pxy = fmaf(B, s2, T * c2);
    const float gm1 = g - 1.0f, m2 = 2.0f * mc.mu, lt = mc.lam * fmaf(g, Ht, 1.0f - Ht) * dtr;
    txx = lt + m2 * fmaf(gm1, pxx, dxx);
    tyy = lt + m2 * fmaf(gm1, pyy, dyy);
    txy = m2 * fmaf(gm1, pxy, dxy);
    const float Ep = 0.5f * (p1 + p2), Em = 0.5f * (p1 - p2), lp = mc.lam * trp;
    sxx = lp + m2 * fmaf(Em, c2, Ep);
    syy = lp + m2 * fmaf(-Em, c2, Ep);
    sxy = m2 * Em * s2;
    Esp = fmaf(0.5f * mc.lam * trp, trp, mc.mu * fmaf(p1, p1, p2 * p2));
  }
  const float cc = fmaf(ddg, Esp, mc.gc_over_eps) * jxw, kk = mc.gc_eps * jxw, dgj = dg * jxw;
  out.cu[0][0] = txx * jxw;
  out.cu[1][1] = tyy * jxw;
  out.cu[0][1] = out.cu[1][0] = txy * jxw;
  float cv = cc * in.ph;
  if (mode == JM_FULL) {
    cv = fmaf(dgj, fmaf(sxx, dxx, fmaf(syy, dyy, 2.0f * sxy * dxy)), cv);
  } else if (mode == JM_TRANSPOSE) {
    const float w = dgj * in.ph;
    out.cu[0][0] = fmaf(w, sxx, out.cu[0][0]);
    out.cu[1][1] = fmaf(w, syy, out.cu[1][1]);
    out.cu[0][1] = out.cu[1][0] = fmaf(w, sxy, out.cu[0][1]);
  }
  out.cv = cv;
  out.cg[0] = kk * in.gph[0];
  out.cg[1] = kk * in.gph[1];
}

// -------------------------------------------------------------------------------------------
// Pointwise residual of Eq. (residual) from the evaluated state (FP64):
// u-test  g(phi~) sigma^+ + sigma^-,  phi-test  g'(phi) E_s^+ - (G_c/eps)(1 - phi),
// grad-test G_c eps grad phi. Stored per point: g(phi~), G_c, lambda, mu.
template <int DIM, int SPLIT>
struct PWRes {
  const double* st;  // [tile][4][qpt]
  const double* sp;  // Miehe split: [tile][NM + 1][qpt] sigma+ (Mandel) and E_s+ of the current u, or null
  long long tstride, qpt;
  int qpx, qpy, n;
  double W[MAXN], hd, eps, kappa;
  __device__ __forceinline__ void operator()(long long tile, long long qi, const QPIn<DIM, double>& in,
                                             QPOut<DIM, double>& out) const {
    const double* a = st + tile * tstride + qi;
    const double gt = a[0], gc = a[qpt], lam = a[2 * qpt], mu = a[3 * qpt];
    const int qx = int(qi % qpx) % n;
    const int qy = int((qi / qpx) % qpy) % n;
    double jxw = hd * W[qx] * W[qy];
    if constexpr (DIM == 3) jxw *= W[int(qi / ((long long)qpx * qpy)) % n];
    double e[DIM][DIM];
    double tr = 0.0;
    for (int i = 0; i < DIM; ++i) {
      for (int j = 0; j < DIM; ++j) e[i][j] = 0.5 * (in.gu[i][j] + in.gu[j][i]);
      tr += e[i][i];
    }
    double sp[DIM][DIM], Esp;
    if constexpr (SPLIT == 0) {
      double ee = 0.0;
      for (int i = 0; i < DIM; ++i)
        for (int j = 0; j < DIM; ++j) {
          sp[i][j] = 2.0 * mu * e[i][j] + (i == j ? lam * tr : 0.0);
          ee += e[i][j] * e[i][j];
        }
      Esp = 0.5 * lam * tr * tr + mu * ee;
    } else if (this->sp) {
      // sigma+ and E_s+ of this u, computed with the tangent (one eigen-decomposition per u)
      constexpr int NM = Mandel<DIM>::NM;
      const double* c = this->sp + tile * (long long)(NM + 1) * qpt + qi;
      for (int m = 0; m < NM; ++m) {
        const int i = Mandel<DIM>::ia(m), j = Mandel<DIM>::ib(m);
        const double v = c[m * qpt];
        if (i == j) sp[i][i] = v;
        else sp[i][j] = sp[j][i] = v * 0.70710678118654752440;  // 1 / sqrt(2)
      }
      Esp = c[NM * qpt];
    } else {
      double l[DIM], V[DIM][DIM];
      eig_sym<DIM>(e, l, V);
      double trs = tr;
      snap_zero<DIM>(l, trs);
      const double trp = pos(trs);
      double sl2 = 0.0;
      for (int t = 0; t < DIM; ++t) sl2 += pos(l[t]) * pos(l[t]);
      Esp = 0.5 * lam * trp * trp + mu * sl2;
      for (int i = 0; i < DIM; ++i)
        for (int j = 0; j < DIM; ++j) {
          double epij = 0.0;
          for (int t = 0; t < DIM; ++t) epij += pos(l[t]) * V[i][t] * V[j][t];
          sp[i][j] = 2.0 * mu * epij + (i == j ? lam * trp : 0.0);
        }
    }
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        const double sig = 2.0 * mu * e[i][j] + (i == j ? lam * tr : 0.0);
        out.cu[i][j] = jxw * (gt * sp[i][j] + (sig - sp[i][j]));
      }
    out.cv = jxw * (deg_dg(in.ph, kappa) * Esp - gc / eps * (1.0 - in.ph));
    for (int j = 0; j < DIM; ++j) out.cg[j] = jxw * gc * eps * in.gph[j];
  }
};

// -------------------------------------------------------------------------------------------
struct OpArgs {
  int inmask, outmask;
  // persistent 2D kernels: gridDim.x tiles = step_y tile rows + step_x tiles (step_x < tiles per row)
  int step_x = 0, step_y = 0;
};
inline OpArgs op_args(int inmask, int outmask, long long grid, int ntile_x) {
  OpArgs a{inmask, outmask};
  a.step_x = int(grid % ntile_x);
  a.step_y = int(grid / ntile_x);
  return a;
}

__device__ __forceinline__ unsigned char dirichlet_bits(int dim) { return (unsigned char)((1u << dim) - 1u); }

// Store of one node value of the output patch (see the file comment for the seam rule).
template <typename Real>
__device__ __forceinline__ void store_node(Real* __restrict__ dst, const Real* __restrict__ src,
                                           const unsigned char* __restrict__ flags, long long node,
                                           long long gi, int f, int dim, Real v, bool low_seam,
                                           bool high_seam, int outmask) {
  bool masked = false;
  if (outmask != OUT_RAW) {
    const unsigned char fl = flags[node];
    const unsigned char m = outmask == OUT_IDENTITY ? fl : (unsigned char)(fl & dirichlet_bits(dim));
    masked = (m >> f) & 1u;
  }
  if (masked) {
    if (!low_seam) dst[gi] = outmask == OUT_IDENTITY ? src[gi] : Real(0);
  } else if (low_seam || high_seam) {
    atomicAdd(dst + gi, v);
  } else {
    dst[gi] = v;
  }
}

template <typename Real>
__device__ __forceinline__ Real load_node(const Real* __restrict__ src, const unsigned char* __restrict__ flags,
                                          long long node, long long gi, int f, int dim, int inmask) {
  Real v = src[gi];
  if (inmask != IN_RAW) {
    const unsigned char fl = flags[node];
    const unsigned char m = inmask == IN_ALL ? fl : (unsigned char)(fl & dirichlet_bits(dim));
    if ((m >> f) & 1u) v = Real(0);
  }
  return v;
}

// Range of cells (within a tile of T cells) containing local node index r (0..T*P).
template <int P>
__device__ __forceinline__ void cells_of_node(int r, int T, int& lo, int& hi) {
  lo = r == 0 ? 0 : (r - 1) / P;
  hi = r / P;
  if (hi > T - 1) hi = T - 1;
}

// ===========================================================================================
// 2D operator kernel. Thread (tx, ty) of a (TX (p+1)) x TY block owns Gauss column tx of cell row
// ty: it contracts the node rows of its cell in x, then in y, applies the pointwise functor at its
// p+1 points and contracts back in y, all in registers; a second pass sums the transposed x
// contractions of the cells sharing each node of the patch.
template <int P>
struct Tile2 {
  static constexpr int TX = TileCfg<2, P>::TX, TY = TileCfg<2, P>::TY;
  static constexpr int n = P + 1, NPX = TX * P + 1, NPY = TY * P + 1, QPX = TX * n, QPY = TY * n;
  static constexpr int NT = QPX * TY;
};

template <int P, typename Real, typename Store, class PW>
__global__ void __launch_bounds__(Tile2<P>::NT)
k_op2d(const Store* __restrict__ src, Store* __restrict__ dst, const unsigned char* __restrict__ flags,
       Geom g, Tab<Real> tb, PW pw, OpArgs oa) {
  using T = Tile2<P>;
  constexpr int TX = T::TX, TY = T::TY, n = T::n, NF = 3;
  constexpr int NPX = T::NPX, NPY = T::NPY, QPX = T::QPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* X = reinterpret_cast<Real*>(smem_raw);  // [NF][NPY][NPX], then the output patch
  Real* UB = X + NF * NPY * NPX;                 // [NF][TY][n][QPX]
  Real* UD = UB + NF * TY * n * QPX;
  Real* sS = UD + NF * TY * n * QPX;             // [n][n]
  Real* sD = sS + n * n;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * QPX + tx;
  const long long tile = blockIdx.x;
  const int tix = int(tile % g.ntile[0]), tiy = int(tile / g.ntile[0]);
  const int x0 = tix * TX * P, y0 = tiy * TY * P;
  if (tid < n * n) {
    sS[tid] = tb.S[tid / n][tid % n];
    sD[tid] = tb.D[tid / n][tid % n];
  }
  // node patch of every field (masked on input)
  for (int r = ty; r < NPY; r += TY) {
    const int gy = y0 + r;
    for (int s = tx; s < NPX; s += QPX) {
      const int gx = x0 + s;
      Real v[NF] = {Real(0), Real(0), Real(0)};
      if (gx < g.n1 && gy < g.n1) {
        const long long node = cut_below(g, tiy, r, NPY, gx) ? cut_copy(g, gx, 0) : gx + (long long)g.n1 * gy;
        unsigned char m = 0;
        if (oa.inmask != IN_RAW) {
          m = flags[node];
          if (oa.inmask == IN_DIRICHLET) m &= dirichlet_bits(2);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = ((m >> f) & 1u) ? Real(0) : cvt<Real>(src[f * g.nn + node]);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) X[(f * NPY + r) * NPX + s] = v[f];
    }
  }
  const int cx = tx / n, qi = tx % n;
  const bool inside = (tix * TX + cx < g.N) && (tiy * TY + ty < g.N);
  Real Sq[n], Dq[n];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < n; ++k) {
    Sq[k] = sS[qi * n + k];
    Dq[k] = sD[qi * n + k];
  }
  // x-contraction of the n node rows of this cell at Gauss column qi
  Real xb[NF][n], xd[NF][n];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int l = 0; l < n; ++l) {
      const Real* row = X + (f * NPY + ty * P + l) * NPX + cx * P;
      Real b = Sq[0] * row[0], d = Dq[0] * row[0];
#pragma unroll
      for (int k = 1; k < n; ++k) {
        b = fmac(Sq[k], row[k], b);
        d = fmac(Dq[k], row[k], d);
      }
      xb[f][l] = b;
      xd[f][l] = d;
    }
  Real ub[NF][n], ud[NF][n];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int l = 0; l < n; ++l) {
      ub[f][l] = Real(0);
      ud[f][l] = Real(0);
    }
  if (inside) {
#pragma unroll
    for (int qj = 0; qj < n; ++qj) {
      Real sj[n], dj[n];
#pragma unroll
      for (int l = 0; l < n; ++l) {
        sj[l] = sS[qj * n + l];
        dj[l] = sD[qj * n + l];
      }
      QPIn<2, Real> in;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        Real gx = sj[0] * xd[k][0], gy = dj[0] * xb[k][0];
#pragma unroll
        for (int l = 1; l < n; ++l) {
          gx = fmac(sj[l], xd[k][l], gx);
          gy = fmac(dj[l], xb[k][l], gy);
        }
        in.gu[k][0] = gx;
        in.gu[k][1] = gy;
      }
      {
        Real v = sj[0] * xb[2][0], gx = sj[0] * xd[2][0], gy = dj[0] * xb[2][0];
#pragma unroll
        for (int l = 1; l < n; ++l) {
          v = fmac(sj[l], xb[2][l], v);
          gx = fmac(sj[l], xd[2][l], gx);
          gy = fmac(dj[l], xb[2][l], gy);
        }
        in.ph = v;
        in.gph[0] = gx;
        in.gph[1] = gy;
      }
      QPOut<2, Real> o;
      pw(tile, (long long)(ty * n + qj) * QPX + tx, in, o);
#pragma unroll
      for (int l = 0; l < n; ++l) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          ub[k][l] = fmac(dj[l], o.cu[k][1], ub[k][l]);
          ud[k][l] = fmac(sj[l], o.cu[k][0], ud[k][l]);
        }
        ub[2][l] = fmac(sj[l], o.cv, fmac(dj[l], o.cg[1], ub[2][l]));
        ud[2][l] = fmac(sj[l], o.cg[0], ud[2][l]);
      }
    }
  }
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int l = 0; l < n; ++l) {
      UB[((f * TY + ty) * n + l) * QPX + tx] = ub[f][l];
      UD[((f * TY + ty) * n + l) * QPX + tx] = ud[f][l];
    }
  __syncthreads();
  // transposed x-contraction: each node of the patch sums the cells that share it, then stores
  for (int r = ty; r < NPY; r += TY) {
    const int gy = y0 + r;
    const int ylo = r == 0 ? 0 : (r - 1) / P, yhi = r / P < TY - 1 ? r / P : TY - 1;
    for (int s = tx; s < NPX; s += QPX) {
      const int gx = x0 + s;
      if (gx >= g.n1 || gy >= g.n1) continue;
      const int xlo = s == 0 ? 0 : (s - 1) / P, xhi = s / P < TX - 1 ? s / P : TX - 1;
      Real acc[NF] = {Real(0), Real(0), Real(0)};
      for (int cy = ylo; cy <= yhi; ++cy) {
        const int l = r - cy * P;
        for (int cxx = xlo; cxx <= xhi; ++cxx) {
          const int k = s - cxx * P;
#pragma unroll
          for (int q = 0; q < n; ++q) {
            const Real sk = sS[q * n + k], dk = sD[q * n + k];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              const int o = ((f * TY + cy) * n + l) * QPX + cxx * n + q;
              acc[f] = fmac(sk, UB[o], fmac(dk, UD[o], acc[f]));
            }
          }
        }
      }
      // a cut slit separates the tile rows above and below it: its nodes are shared only along x
      const bool below = cut_below(g, tiy, r, NPY, gx);
      const long long node = below ? cut_copy(g, gx, 0) : gx + (long long)g.n1 * gy;
      const bool low = (s == 0 && tix > 0) || (r == 0 && tiy > 0 && !cut_above(g, tiy, r, gx));
      const bool high = (s == NPX - 1 && tix < g.ntile[0] - 1) || (r == NPY - 1 && tiy < g.ntile[1] - 1 && !below);
      unsigned char m = 0;
      if (oa.outmask != OUT_RAW) {
        m = flags[node];
        if (oa.outmask == OUT_ZERO_DIRICHLET) m &= dirichlet_bits(2);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const long long gi = f * g.nn + node;
        if ((m >> f) & 1u) {
          if (!low) dst[gi] = oa.outmask == OUT_IDENTITY ? src[gi] : Store(0);
        } else if (low || high) {
          atomicAdd(dst + gi, cvt<Store>(acc[f]));
        } else {
          dst[gi] = cvt<Store>(acc[f]);
        }
      }
    }
  }
}

template <int P, typename Real>
constexpr size_t op2d_smem() {
  using T = Tile2<P>;
  return sizeof(Real) * (size_t)(3 * T::NPY * T::NPX + 2 * 3 * T::TY * T::n * T::QPX + 2 * T::n * T::n);
}

// ===========================================================================================
// 2D Jacobian kernel, persistent and staged: each CTA walks tiles blockIdx.x, +gridDim.x, ... and
// copies the next tile's node patch and per-point data into shared memory with cp.async (with
// NSTAGE = 2 under the whole computation of the current tile; with NSTAGE = 1 under its store phase,
// which halves the shared memory per CTA: on GB300 the extra resident CTAs hide more latency than
// the second stage, 0.199 vs 0.244 ms for the FP32 2D Q2 apply at 1024^2 cells). The arithmetic is
// that of k_op2d.
__device__ __forceinline__ void cp_async_bytes(void* smem, const void* gmem, bool valid, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Sum of v over the CTA (threads numbered tid < nt, nt a multiple of 32); valid in tid 0.
__device__ __forceinline__ double block_sum_lin(double v, int tid, int nt, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (tid < 32) {
    r = tid < nt / 32 ? sh[tid] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

template <int P, typename Real>
struct Stage2 {
  static constexpr int NSTAGE = 1;  // kept as a parameter: the kernel supports 2
};

// Whether the 2D Jacobian kernel masks its staged node patch in place (the raw copy is already in the
// compute type, and nothing reads the masked patch after the next tile's copies have started: the
// CG-Lanczos epilogue does, so it keeps a separate buffer). Saves 3.5 KB per CTA for FP32 Q2, which
// makes room for a fifth CTA per SM.
template <int P, typename Real, typename Store, int CG>
constexpr bool jac2_x_inplace() {
  return std::is_same<Real, Store>::value && CG == 0 && Stage2<P, Real>::NSTAGE == 1;
}

// The same smoothing update on the seam nodes of the 2D tile grid, once their y is complete; y is
// reset to 0 there, so y is all zero again afterwards (the fused applies write no other entry).
// Seam index t enumerates the vertical seam lines, then the horizontal ones (crossings once).
template <typename Store>
__device__ __forceinline__ void cheb_seam_node(const Geom& g, int tpx, int tpy, Store* y, const ChebEpi<Store>& ce,
                                               int t, Store c1, const Store c2[2]) {
  // 32-bit index arithmetic (node counts fit in 32 bits, checked at setup)
  const unsigned n1 = (unsigned)g.n1;
  const int nv = (g.ntile[0] - 1) * g.n1;
  int gx, gy;
  if (t < nv) {
    gx = int((unsigned)t / n1 + 1) * tpx;
    gy = int((unsigned)t % n1);
  } else {
    const unsigned u = (unsigned)(t - nv);
    gy = int(u / n1 + 1) * tpy;
    gx = int(u % n1);
    if (gx % tpx == 0 && gx > 0 && gx < g.n1 - 1) return;  // already done on a vertical seam line
    // a cut slit's nodes are shared along x only: the tiles finished them, except on vertical seams
    if (g.cut && gy == g.cut_row && gx < g.cut_x) return;
  }
  const bool both = g.cut && gy == g.cut_row && gx < g.cut_x;  // a vertical seam crossing a cut slit
  Store* const x_out = ce.x_out ? ce.x_out : ce.x;
  Store* const d_out = ce.d_out ? ce.d_out : ce.d;
  for (int k = 0; k < (both ? 2 : 1); ++k) {
    const long long node = k ? cut_copy(g, gx, 0) : gx + (long long)g.n1 * gy;
    // all loads before the stores (the compiler cannot tell that the arrays do not alias)
    Store yv[3], dv[3], iv[3], fv[3], xv[3], av[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const long long gi = f * g.nn + node;
      yv[f] = y[gi];
      dv[f] = ce.d[gi];
      iv[f] = ce.dinv[gi];
      fv[f] = ce.f[gi];
      xv[f] = ce.x[gi];
      av[f] = ce.acc ? ce.acc[gi] : Store(0);
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const long long gi = f * g.nn + node;
      const Store dn = c1 * dv[f] + c2[f < 2 ? 0 : 1] * (iv[f] * (fv[f] - yv[f]));
      d_out[gi] = dn;
      if (ce.acc) ce.acc[gi] = av[f] + (xv[f] + dn);
      else x_out[gi] = xv[f] + dn;
      y[gi] = Store(0);
      if (ce.tz) ce.tz[gi] = Store(0);  // the previous step's seam sums (two-buffer scheme)
    }
  }
}

// Register budget per thread that keeps the CTAs resident which fit in shared memory (FP32 Q2: five
// per SM; double-word Q2 to Q4: two): FP32 64 up to Q2 and 96 above (64 would spill there), double-word
// 80 for Q1 and 168 above (unconstrained, Q4 took 255 registers and ran one CTA of 5 warps per SM; at
// 168 it spills 8 to 16 bytes); native FP64 unconstrained.
// The recomputed FP32 tangent (RC) keeps the state's contractions live: 96 up to Q2 (80 spilled), 128 above.
// The CG-Lanczos epilogue (CG) keeps its dot products and a separate masked patch: FP32 80 up to Q2 (64
// spilled 60 bytes; shared memory holds it at four CTAs per SM, which 80 keeps), 128 above; double-word Q4
// unconstrained (one CTA per SM by shared memory; 168 spilled 200 bytes).
template <int P, typename Real, int RC = 0, int CG = 0>
constexpr int jac2_reg_budget() {
  return std::is_same<Real, float>::value
             ? (RC ? (P <= 2 ? 96 : 128) : (P <= 2 ? (CG ? 80 : 64) : (CG ? 128 : 96)))
         : std::is_same<Real, df64>::value ? (P == 1 ? 80 : (CG && P == 4) ? 0 : 168)
                                           : 0;
}
template <int P, typename Real, int RC = 0, int CG = 0>
constexpr int jac2_min_blocks() {
  return jac2_reg_budget<P, Real, RC, CG>() ? 65536 / (Tile2<P>::NT * jac2_reg_budget<P, Real, RC, CG>()) : 1;
}

// RC = 1 (FP32 only): the pointwise Jacobian is recomputed from the nodal state (u_x, u_y, phi, phi~;
// qpg then points to those 4 fields of n_nodes floats each) by pw_jac_rc2 instead of read from stored
// per-point data: the tile stages 4 state values per node instead of NV values per Gauss point.
// ES = 1 (for grids with at most one tile per CTA, where nothing hides a global round trip): the tile's
// copies also stage the Chebyshev step's operands d, D^{-1}, f, x of the patch into shared memory, which the
// store phase then reads instead of global memory.
template <int P, typename Real, typename Store, int SPLIT, int RC, int CG, int ES = 0>
__global__ void __launch_bounds__(Tile2<P>::NT, ES ? 1 : jac2_min_blocks<P, Real, RC, CG>())
k_jac2_staged(const Store* src, Store* __restrict__ dst, const unsigned char* __restrict__ flags,
              Geom g, Tab<Real> tb, const Real* __restrict__ qpg, int mode, OpArgs oa, ChebEpi<Store> ce,
              MatConst32 mc, CgEpi<Store> cg) {
  pdl_wait();
  using T = Tile2<P>;
  constexpr int TX = T::TX, TY = T::TY, n = T::n, NF = 3;
  constexpr int NPX = T::NPX, NPY = T::NPY, QPX = T::QPX;
  constexpr int QPT = T::QPX * T::QPY;
  constexpr int NV = RC ? 0 : qp_nv(2, SPLIT);
  constexpr int NSF = RC ? 4 : 0;  // staged state fields
  constexpr int NS = Stage2<P, Real>::NSTAGE;
  constexpr int NT = T::NT;
  constexpr int XS = NF * NPY * NPX;
  constexpr int NNODE = NPY * NPX, NIT = (NNODE + NT - 1) / NT;
  static_assert(!RC || std::is_same<Real, float>::value, "the recomputed tangent is FP32 only");
  constexpr bool XIN = jac2_x_inplace<P, Real, Store, CG>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* QPs = reinterpret_cast<Real*>(smem_raw);                  // [NS][NV][QPT]
  Store* Xs = reinterpret_cast<Store*>(QPs + NS * NV * QPT);      // [NS][NF][NPY][NPX] raw copies
  Store* Ss = Xs + NS * XS;                                       // [NS][NSF][NPY][NPX] state (RC)
  constexpr int NES = ES ? 4 : 0;                                 // staged epilogue arrays
  Store* Es = Ss + NS * NSF * NNODE;                              // [NS][NES][NF][NPY][NPX] d, dinv, f, x
  Real* Xc = reinterpret_cast<Real*>(Es + NS * NES * XS);
  Real* X = XIN ? reinterpret_cast<Real*>(Xs) : Xc;               // [NF][NPY][NPX] masked, compute type
  Real* UB = XIN ? Xc : Xc + XS;                                  // [NF][TY][n][QPX]
  Real* UD = UB + NF * TY * n * QPX;
  Real* sS = UD + NF * TY * n * QPX;
  Real* sD = sS + n * n;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * QPX + tx;
  if (tid < n * n) {
    sS[tid] = tb.S[tid / n][tid % n];
    sD[tid] = tb.D[tid / n][tid % n];
  }
  // Chebyshev coefficients per block (field < 2: u block), in the storage precision
  Store ch_c1 = Store(0), ch_c2[2] = {Store(0), Store(0)};
  Store pc1 = Store(0), pc2[2] = {Store(0), Store(0)};  // the previous step's (seam completion)
  if (ce.on) {
    ch_c2[0] = Store(ce.c2s) * ce.inv_lam[0];
    ch_c2[1] = Store(ce.c2s) * ce.inv_lam[1];
    ch_c1 = Store(ce.c1);
    if (ce.pp) {
      pc2[0] = Store(ce.c2sp) * ce.inv_lam[0];
      pc2[1] = Store(ce.c2sp) * ce.inv_lam[1];
      pc1 = Store(ce.c1p);
    }
  }
  Store* const x_out = ce.x_out ? ce.x_out : ce.x;
  Store* const d_out = ce.d_out ? ce.d_out : ce.d;
  Store cg_beta[2] = {Store(0), Store(0)};
  double cg_dot[2] = {0.0, 0.0};  // this thread's share of <p, A p>, per block
  if constexpr (CG != 0) {
    cg_beta[0] = Store(cg.scal[6]);
    cg_beta[1] = Store(cg.scal[7]);
  }
  // DoF indices fit in 32 bits (checked at setup); tile coordinates step by gridDim.x tiles without a
  // division (oa.step_x along x with a carry into y, oa.step_y rows)
  const int ntiles = int(g.ntiles), ntx = g.ntile[0], nn = int(g.nn), n1 = g.n1, ngrid = int(g.ngrid);
  auto next_tile = [&](int& ax, int& ay) {
    ax += oa.step_x;
    ay += oa.step_y;
    if (ax >= ntx) {
      ax -= ntx;
      ++ay;
    }
  };
  // node phases (copy, masking, store): this thread handles patch nodes tid + k NT, all fields
  auto prefetch = [&](int tile, int tix, int tiy, int st) {
    const int x0 = tix * TX * P, y0 = tiy * TY * P;
    Store* xs = Xs + st * XS;
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
      const int rs = tid + k * NT;
      if (rs >= NNODE) break;
      const int r = rs / NPX, s = rs - r * NPX;
      const int gx = x0 + s, gy = y0 + r;
      const bool ok = gx < n1 && gy < n1;
      const int node = cut_below(g, tiy, r, NPY, gx) ? ngrid + gx : gx + n1 * gy;
      const Store* sp = src + (ok ? node : 0);
      Store* dp = xs + rs;
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async_bytes(dp + f * NNODE, sp + (ok ? f * nn : 0), ok, (int)sizeof(Store));
      if constexpr (ES != 0) {
        if (ce.on) {
          const Store* ea[4] = {ce.d, ce.dinv, ce.f, ce.x};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int f = 0; f < NF; ++f)
              cp_async_bytes(Es + ((st * NES + a) * NF + f) * NNODE + rs, ea[a] + (ok ? f * nn + node : 0), ok,
                             (int)sizeof(Store));
        }
      }
      if constexpr (RC != 0) {
        const Store* stp = reinterpret_cast<const Store*>(qpg) + (ok ? node : 0);
        Store* sdp = Ss + st * NSF * NNODE + rs;
#pragma unroll
        for (int f = 0; f < NSF; ++f)
          cp_async_bytes(sdp + f * NNODE, stp + (ok ? f * nn : 0), ok, (int)sizeof(Store));
      }
    }
    if constexpr (RC == 0) {
      const char* qsrc = reinterpret_cast<const char*>(qpg + (long long)tile * (NV * QPT));
      char* qdst = reinterpret_cast<char*>(QPs + st * NV * QPT);
      constexpr int NCH = NV * QPT * (int)sizeof(Real) / 16;
      for (int i = tid; i < NCH; i += NT) cp_async16(qdst + 16 * i, qsrc + 16 * i);
    }
  };

  int it = 0;
  int tix = int(blockIdx.x % (unsigned)ntx), tiy = int(blockIdx.x / (unsigned)ntx);
  if ((int)blockIdx.x < ntiles) prefetch(blockIdx.x, tix, tiy, 0);
  cp_async_commit();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it, next_tile(tix, tiy)) {
    const int st = NS == 2 ? (it & 1) : 0;
    if constexpr (NS == 2) {
      const int nxt = tile + gridDim.x;
      int nx = tix, ny = tiy;
      next_tile(nx, ny);
      if (nxt < ntiles) prefetch(nxt, nx, ny, st ^ 1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int x0 = tix * TX * P, y0 = tiy * TY * P;
    // masked compute-type node patch
    const Store* xs = Xs + st * XS;
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
      const int rs = tid + k * NT;
      if (rs >= NNODE) break;
      const int r = rs / NPX, s = rs - r * NPX;
      const int gx = x0 + s, gy = y0 + r;
      const int node = cut_below(g, tiy, r, NPY, gx) ? ngrid + gx : gx + n1 * gy;
      unsigned char m = 0;
      if (oa.inmask != IN_RAW && gx < n1 && gy < n1) {
        m = flags[node];
        if (oa.inmask == IN_DIRICHLET) m &= dirichlet_bits(2);
      }
      Store xv[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) xv[f] = xs[f * NNODE + rs];
      // a node shared with a neighbouring tile (as in the store phase), and whether this tile owns it
      bool low = false, high = false;
      if (CG != 0 || (ce.on && ce.pp)) {
        low = (s == 0 && tix > 0) || (r == 0 && tiy > 0 && !cut_above(g, tiy, r, gx));
        high = (s == NPX - 1 && tix < g.ntile[0] - 1) ||
               (r == NPY - 1 && tiy < g.ntile[1] - 1 && !cut_below(g, tiy, r, NPY, gx));
      }
      // (Below, every field's loads come before the stores: the compiler cannot tell that the output
      // arrays do not alias the inputs, and would otherwise wait for one round trip per field.)
      if (CG != 0 && gx < n1 && gy < n1) {
        // CG-Lanczos: the apply's input p = z + beta p_old (z is the staged src)
        Store po[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) po[f] = cg.p_old[f * nn + node];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          xv[f] = xv[f] + cg_beta[f < 2 ? 0 : 1] * po[f];
          if (!low) cg.p_out[f * nn + node] = xv[f];
        }
      }
      if (ce.on && ce.pp && gx < n1 && gy < n1) {
        // a seam node of the previous step: finish that step here from its complete seam sums
        if (low || high) {
          Store dO[NF], dI[NF], fF[NF], tP[NF], xO[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const int gi = f * nn + node;
            dO[f] = d_out[gi];
            dI[f] = ce.dinv[gi];
            fF[f] = ce.f[gi];
            tP[f] = ce.tp[gi];
            xO[f] = x_out[gi];
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            const int gi = f * nn + node;
            const Store dk = pc1 * dO[f] + pc2[f < 2 ? 0 : 1] * (dI[f] * (fF[f] - tP[f]));
            xv[f] = xO[f] + dk;
            if (!low) {  // the owning tile writes the finished step back
              ce.d[gi] = dk;
              ce.x[gi] = xv[f];
              if (ce.tz) ce.tz[gi] = Store(0);
            }
          }
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int i = f * NNODE + rs;
        X[i] = ((m >> f) & 1u) ? Real(0) : cvt<Real>(xv[f]);
      }
    }
    __syncthreads();
    const int cx = tx / n, qi = tx % n;
    const bool inside = (tix * TX + cx < g.N) && (tiy * TY + ty < g.N);
    Real Sq[n], Dq[n];
#pragma unroll
    for (int k = 0; k < n; ++k) {
      Sq[k] = sS[qi * n + k];
      Dq[k] = sD[qi * n + k];
    }
    Real xb[NF][n], xd[NF][n];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const Real* row = X + (f * NPY + ty * P + l) * NPX + cx * P;
        Real b = Sq[0] * row[0], d = Dq[0] * row[0];
#pragma unroll
        for (int k = 1; k < n; ++k) {
          b = fmac(Sq[k], row[k], b);
          d = fmac(Dq[k], row[k], d);
        }
        xb[f][l] = b;
        xd[f][l] = d;
      }
    Real ub[NF][n], ud[NF][n];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int l = 0; l < n; ++l) {
        ub[f][l] = Real(0);
        ud[f][l] = Real(0);
      }
    // RC: x-contractions of the nodal state (u_x, u_y with their x-derivatives, phi and phi~)
    Real sb[RC ? 4 : 1][n], sd[RC ? 2 : 1][n];
    if constexpr (RC != 0) {
      const Store* ss = Ss + st * NSF * NNODE;
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int l = 0; l < n; ++l) {
          const Store* row = ss + (f * NPY + ty * P + l) * NPX + cx * P;
          Real b = Sq[0] * row[0], d = Dq[0] * row[0];
#pragma unroll
          for (int k = 1; k < n; ++k) {
            b = fmac(Sq[k], row[k], b);
            if (f < 2) d = fmac(Dq[k], row[k], d);
          }
          sb[f][l] = b;
          if (f < 2) sd[f][l] = d;
        }
    }
    if (inside) {
      PWJac<2, Real, SPLIT> pw;
      pw.qp = QPs + st * NV * QPT;
      pw.tstride = 0;
      pw.qpt = QPT;
      pw.mode = mode;
#pragma unroll
      for (int qj = 0; qj < n; ++qj) {
        Real sj[n], dj[n];
#pragma unroll
        for (int l = 0; l < n; ++l) {
          sj[l] = sS[qj * n + l];
          dj[l] = sD[qj * n + l];
        }
        QPIn<2, Real> in;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          Real gx = sj[0] * xd[k][0], gy = dj[0] * xb[k][0];
#pragma unroll
          for (int l = 1; l < n; ++l) {
            gx = fmac(sj[l], xd[k][l], gx);
            gy = fmac(dj[l], xb[k][l], gy);
          }
          in.gu[k][0] = gx;
          in.gu[k][1] = gy;
        }
        {
          Real v = sj[0] * xb[2][0], gx = sj[0] * xd[2][0], gy = dj[0] * xb[2][0];
#pragma unroll
          for (int l = 1; l < n; ++l) {
            v = fmac(sj[l], xb[2][l], v);
            gx = fmac(sj[l], xd[2][l], gx);
            gy = fmac(dj[l], xb[2][l], gy);
          }
          in.ph = v;
          in.gph[0] = gx;
          in.gph[1] = gy;
        }
        QPOut<2, Real> o;
        if constexpr (RC != 0) {
          float pst[6];
          pst[0] = sj[0] * sd[0][0];
          pst[1] = dj[0] * sb[0][0];
          pst[2] = sj[0] * sd[1][0];
          pst[3] = dj[0] * sb[1][0];
          pst[4] = sj[0] * sb[2][0];
          pst[5] = sj[0] * sb[3][0];
#pragma unroll
          for (int l = 1; l < n; ++l) {
            pst[0] = fmac(sj[l], sd[0][l], pst[0]);
            pst[1] = fmac(dj[l], sb[0][l], pst[1]);
            pst[2] = fmac(sj[l], sd[1][l], pst[2]);
            pst[3] = fmac(dj[l], sb[1][l], pst[3]);
            pst[4] = fmac(sj[l], sb[2][l], pst[4]);
            pst[5] = fmac(sj[l], sb[3][l], pst[5]);
          }
          pw_jac_rc2<SPLIT>(pst, tb.hd * tb.W[qi] * tb.W[qj], mc, mode, in, o);
        } else {
          pw(0, (long long)(ty * n + qj) * QPX + tx, in, o);
        }
#pragma unroll
        for (int l = 0; l < n; ++l) {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            ub[k][l] = fmac(dj[l], o.cu[k][1], ub[k][l]);
            ud[k][l] = fmac(sj[l], o.cu[k][0], ud[k][l]);
          }
          ub[2][l] = fmac(sj[l], o.cv, fmac(dj[l], o.cg[1], ub[2][l]));
          ud[2][l] = fmac(sj[l], o.cg[0], ud[2][l]);
        }
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int l = 0; l < n; ++l) {
        UB[((f * TY + ty) * n + l) * QPX + tx] = ub[f][l];
        UD[((f * TY + ty) * n + l) * QPX + tx] = ud[f][l];
      }
    __syncthreads();
    if constexpr (NS == 1 && ES == 0) {
      // the staging buffers are free: start the next tile's copies under the store phase
      const int nxt = tile + gridDim.x;
      int nx = tix, ny = tiy;
      next_tile(nx, ny);
      if (nxt < ntiles) prefetch(nxt, nx, ny, 0);
      cp_async_commit();
    }
    // Transposed x contraction, one node column per thread: thread (cx, qi) sums the n Gauss columns of
    // its cell into the cell's node column k = qi, for every field and node row of the cell. The cell's
    // node values then go to four arrays (in the UB buffer), by whether the node row / column is the
    // cell's last, i.e. shared with the next cell: E00 [NF][TY P][TX P], E10 [NF][TY][TX P],
    // E01 [NF][TY P][TX], E11 [NF][TY][TX]; each patch node sums at most one entry of each.
    constexpr int TXP = TX * P, TYP = TY * P;
    {
      Real v[NF][n];
      Real Sk[n], Dk[n];
#pragma unroll
      for (int q = 0; q < n; ++q) {
        Sk[q] = sS[q * n + qi];
        Dk[q] = sD[q * n + qi];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int l = 0; l < n; ++l) {
          const Real* ubp = UB + ((f * TY + ty) * n + l) * QPX + cx * n;
          const Real* udp = UD + ((f * TY + ty) * n + l) * QPX + cx * n;
          Real a = fmac(Dk[0], udp[0], Sk[0] * ubp[0]);
#pragma unroll
          for (int q = 1; q < n; ++q) a = fmac(Sk[q], ubp[q], fmac(Dk[q], udp[q], a));
          v[f][l] = a;
        }
      __syncthreads();  // every thread has read its cell's columns of UB and UD
      Real* E00 = UB;
      Real* E10 = E00 + NF * TYP * TXP;
      Real* E01 = E10 + NF * TY * TXP;
      Real* E11 = E01 + NF * TYP * TX;
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int l = 0; l < n; ++l) {
          Real* e;
          if (l < P)
            e = qi < P ? E00 + (f * TYP + ty * P + l) * TXP + cx * P + qi : E01 + (f * TYP + ty * P + l) * TX + cx;
          else
            e = qi < P ? E10 + (f * TY + ty) * TXP + cx * P + qi : E11 + (f * TY + ty) * TX + cx;
          *e = v[f][l];
        }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < NIT; ++kk) {
      const int rs = tid + kk * NT;
      if (rs >= NNODE) break;
      const int r = rs / NPX, s = rs - r * NPX;
      const int gx = x0 + s, gy = y0 + r;
      if (gx >= n1 || gy >= n1) continue;
      Real acc[NF];
      {
        const Real* E00 = UB;
        const Real* E10 = E00 + NF * TYP * TXP;
        const Real* E01 = E10 + NF * TY * TXP;
        const Real* E11 = E01 + NF * TYP * TX;
        const bool ra = r < TYP, sa = s < TXP;                    // the node row / column starts a cell
        const bool re = r > 0 && r % P == 0, se = s > 0 && s % P == 0;  // ... or ends one
        const int rb = r / P - 1, sb = s / P - 1;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          Real a = (ra && sa) ? E00[(f * TYP + r) * TXP + s] : Real(0);
          if (re && sa) a = a + E10[(f * TY + rb) * TXP + s];
          if (se && ra) a = a + E01[(f * TYP + r) * TX + sb];
          if (re && se) a = a + E11[(f * TY + rb) * TX + sb];
          acc[f] = a;
        }
      }
      const bool below = cut_below(g, tiy, r, NPY, gx);
      const int node = below ? ngrid + gx : gx + n1 * gy;
      const bool low = (s == 0 && tix > 0) || (r == 0 && tiy > 0 && !cut_above(g, tiy, r, gx));
      const bool high = (s == NPX - 1 && tix < g.ntile[0] - 1) || (r == NPY - 1 && tiy < g.ntile[1] - 1 && !below);
      unsigned char m = 0;
      if (oa.outmask != OUT_RAW) {
        m = flags[node];
        if (oa.outmask == OUT_ZERO_DIRICHLET) m &= dirichlet_bits(2);
      }
      if constexpr (CG != 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          if (!((m >> f) & 1u)) cg_dot[f < 2 ? 0 : 1] += cvt<double>(X[f * NNODE + rs]) * cvt<double>(acc[f]);
      }
      if (ce.on && !low && !high) {
        // node of this tile only: finish the smoothing step here (all loads first, as above)
        Store cD[NF], cI[NF], cF[NF], cX[NF], cY[NF], cA[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const int gi = f * nn + node;
          if constexpr (ES != 0) {  // staged with the tile's copies
            const Store* e = Es + st * NES * XS + f * NNODE + rs;
            cD[f] = e[0];
            cI[f] = e[XS];
            cF[f] = e[2 * XS];
            cX[f] = e[3 * XS];
          } else {
            cD[f] = ce.d[gi];
            cI[f] = ce.dinv[gi];
            cF[f] = ce.f[gi];
            cX[f] = ce.x[gi];
          }
          cY[f] = ((m >> f) & 1u) ? (oa.outmask == OUT_IDENTITY ? src[gi] : Store(0)) : cvt<Store>(acc[f]);
          cA[f] = ce.acc ? ce.acc[gi] : Store(0);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const int gi = f * nn + node;
          const Store dn = ch_c1 * cD[f] + ch_c2[f < 2 ? 0 : 1] * (cI[f] * (cF[f] - cY[f]));
          d_out[gi] = dn;
          if (ce.acc) ce.acc[gi] = cA[f] + (cX[f] + dn);
          else x_out[gi] = cX[f] + dn;
        }
      } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const int gi = f * nn + node;
          if ((m >> f) & 1u) {
            if (!low) dst[gi] = oa.outmask == OUT_IDENTITY ? src[gi] : Store(0);
          } else if (low || high) {
            atomicAdd(dst + gi, cvt<Store>(acc[f]));
          } else {
            dst[gi] = cvt<Store>(acc[f]);
          }
        }
      }
    }
    if constexpr (NS == 1 && ES != 0) {
      // the next tile's copies, once the store phase has read the staged operands
      __syncthreads();
      const int nxt = tile + gridDim.x;
      int nx = tix, ny = tiy;
      next_tile(nx, ny);
      if (nxt < ntiles) prefetch(nxt, nx, ny, 0);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  if constexpr (CG != 0) {
    // per-CTA partial of <p, A p>; the last CTA adds the partials in CTA order and takes alpha
    __shared__ double sh[32];
    __shared__ int last;
    const double r0 = block_sum_lin(cg_dot[0], tid, NT, sh), r1 = block_sum_lin(cg_dot[1], tid, NT, sh);
    unsigned* cnt = reinterpret_cast<unsigned*>(cg.scal + 12);
    if (tid == 0) {
      cg.part[2 * blockIdx.x] = r0;
      cg.part[2 * blockIdx.x + 1] = r1;
      __threadfence();
      last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double t0 = 0.0, t1 = 0.0;
      for (int b = tid; b < (int)gridDim.x; b += NT) {
        t0 += __ldcg(cg.part + 2 * b);
        t1 += __ldcg(cg.part + 2 * b + 1);
      }
      const double s0 = block_sum_lin(t0, tid, NT, sh), s1 = block_sum_lin(t1, tid, NT, sh);
      if (tid == 0) {
        *cnt = 0u;
        cg_take_alpha(cg.scal, cg.ah, cg.it, cg.iters, s0, s1);
      }
    }
  }
}

template <typename Store>
__global__ void k_cheb_seam2(Geom g, int tpx, int tpy, Store* __restrict__ y, ChebEpi<Store> ce) {
  pdl_wait();
  const int nseam = (g.ntile[0] - 1 + g.ntile[1] - 1) * g.n1;
  const int t = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (t >= nseam) return;
  const Store c2[2] = {Store(ce.c2s) * ce.inv_lam[0], Store(ce.c2s) * ce.inv_lam[1]};
  cheb_seam_node<Store>(g, tpx, tpy, y, ce, t, Store(ce.c1), c2);
}

template <int P, typename Real, typename Store, int SPLIT, int RC = 0, int CG = 0, int ES = 0>
constexpr size_t jac2_staged_smem() {
  using T = Tile2<P>;
  constexpr int NS = Stage2<P, Real>::NSTAGE;
  constexpr int XS = 3 * T::NPY * T::NPX;
  constexpr int NV = RC ? 0 : qp_nv(2, SPLIT), NSF = RC ? 4 : 0, NES = ES ? 4 : 0;
  constexpr int XC = jac2_x_inplace<P, Real, Store, CG>() ? 0 : XS;
  return sizeof(Real) * (size_t)NS * NV * T::QPX * T::QPY +
         sizeof(Store) * (size_t)NS * (XS + NSF * T::NPY * T::NPX + NES * XS) +
         sizeof(Real) * (size_t)(XC + 2 * 3 * T::TY * T::n * T::QPX + 2 * T::n * T::n);
}

// ===========================================================================================
// 3D operator kernel. Block (TX (p+1), TY (p+1), TZ): x- and y-contractions run as passes over the
// tile's node patch in shared memory (a node row shared by two cells is contracted once); thread
// (tx, ty, tz) then owns the Gauss pencil (tx, ty) of cell layer tz, contracts in z, applies the
// pointwise functor at its p+1 points and accumulates the transposed z-contraction; transposed y-
// and x-passes return to the nodes, whose seam copies are accumulated atomically.
template <int P>
struct Tile3 {
  static constexpr int TX = TileCfg<3, P>::TX, TY = TileCfg<3, P>::TY, TZ = TileCfg<3, P>::TZ;
  static constexpr int n = P + 1, NPX = TX * P + 1, NPY = TY * P + 1, NPZ = TZ * P + 1;
  static constexpr int QPX = TX * n, QPY = TY * n, NT = QPX * QPY * TZ;
};

template <int P, typename Real, typename Store, class PW>
__global__ void __launch_bounds__(Tile3<P>::NT)
k_op3d(const Store* __restrict__ src, Store* __restrict__ dst, const unsigned char* __restrict__ flags,
       Geom g, Tab<Real> tb, PW pw, OpArgs oa) {
  pdl_wait();
  using T = Tile3<P>;
  constexpr int TX = T::TX, TY = T::TY, TZ = T::TZ, n = T::n, NF = 4;
  constexpr int NPX = T::NPX, NPY = T::NPY, NPZ = T::NPZ, QPX = T::QPX, QPY = T::QPY;
  constexpr int PLANE = QPY * QPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* X = reinterpret_cast<Real*>(smem_raw);   // [NF][NPZ][NPY][NPX], later the output patch
  Real* XB = X + NF * NPZ * NPY * NPX;            // [NF][NPZ][NPY][QPX], later WB
  Real* XD = XB + NF * NPZ * NPY * QPX;           // later WD
  Real* YB = XD + NF * NPZ * NPY * QPX;           // [NF][NPZ][QPY][QPX]
  Real* YX = YB + NF * NPZ * PLANE;
  Real* YY = YX + NF * NPZ * PLANE;
  Real* ZB = YY + NF * NPZ * PLANE;               // [NF][TZ][n][QPY][QPX]
  Real* ZX = ZB + NF * TZ * n * PLANE;
  Real* ZY = ZX + NF * TZ * n * PLANE;
  Real* sS = ZY + NF * TZ * n * PLANE;
  Real* sD = sS + n * n;

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = (tz * QPY + ty) * QPX + tx;
  const long long tile = blockIdx.x;
  const int tix = int(tile % g.ntile[0]);
  const int tiy = int((tile / g.ntile[0]) % g.ntile[1]);
  const int tiz = int(tile / ((long long)g.ntile[0] * g.ntile[1]));
  const int x0 = tix * TX * P, y0 = tiy * TY * P, z0 = tiz * TZ * P;
  const long long n1 = g.n1, n1sq = n1 * n1;
  if (tid < n * n) {
    sS[tid] = tb.S[tid / n][tid % n];
    sD[tid] = tb.D[tid / n][tid % n];
  }
  for (int t = tz; t < NPZ; t += TZ)
    for (int r = ty; r < NPY; r += QPY)
      for (int s = tx; s < NPX; s += QPX) {
        const int gx = x0 + s, gy = y0 + r, gz = z0 + t;
        Real v[NF] = {Real(0), Real(0), Real(0), Real(0)};
        if (gx < g.n1 && gy < g.n1 && gz < g.n1) {
          const long long node = cut_below(g, tiz, t, NPZ, gx) ? cut_copy(g, gx, gy) : gx + n1 * gy + n1sq * gz;
          unsigned char m = 0;
          if (oa.inmask != IN_RAW) {
            m = flags[node];
            if (oa.inmask == IN_DIRICHLET) m &= dirichlet_bits(3);
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) v[f] = ((m >> f) & 1u) ? Real(0) : cvt<Real>(src[f * g.nn + node]);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) X[((f * NPZ + t) * NPY + r) * NPX + s] = v[f];
      }
  __syncthreads();
  {  // x-pass at Gauss column tx
    const int cx = tx / n, qi = tx % n;
    Real Sq[n], Dq[n];
#pragma unroll
    for (int k = 0; k < n; ++k) {
      Sq[k] = sS[qi * n + k];
      Dq[k] = sD[qi * n + k];
    }
    for (int t = tz; t < NPZ; t += TZ)
      for (int r = ty; r < NPY; r += QPY)
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const Real* row = X + ((f * NPZ + t) * NPY + r) * NPX + cx * P;
          Real b = Sq[0] * row[0], d = Dq[0] * row[0];
#pragma unroll
          for (int k = 1; k < n; ++k) {
            b = fmac(Sq[k], row[k], b);
            d = fmac(Dq[k], row[k], d);
          }
          const int o = ((f * NPZ + t) * NPY + r) * QPX + tx;
          XB[o] = b;
          XD[o] = d;
        }
  }
  __syncthreads();
  {  // y-pass at Gauss row ty
    const int cy = ty / n, qj = ty % n;
    Real Sj[n], Dj[n];
#pragma unroll
    for (int l = 0; l < n; ++l) {
      Sj[l] = sS[qj * n + l];
      Dj[l] = sD[qj * n + l];
    }
    for (int t = tz; t < NPZ; t += TZ)
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int base = ((f * NPZ + t) * NPY + cy * P) * QPX + tx;
        Real b = Sj[0] * XB[base], dx = Sj[0] * XD[base], dy = Dj[0] * XB[base];
#pragma unroll
        for (int l = 1; l < n; ++l) {
          const int o = base + l * QPX;
          b = fmac(Sj[l], XB[o], b);
          dx = fmac(Sj[l], XD[o], dx);
          dy = fmac(Dj[l], XB[o], dy);
        }
        const int o = (f * NPZ + t) * PLANE + ty * QPX + tx;
        YB[o] = b;
        YX[o] = dx;
        YY[o] = dy;
      }
  }
  __syncthreads();
  {  // z-pass, pointwise, transposed z-pass: pencil (tx, ty) of cell layer tz
    const int col = ty * QPX + tx;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const int o = ((f * TZ + tz) * n + l) * PLANE + col;
        ZB[o] = Real(0);
        ZX[o] = Real(0);
        ZY[o] = Real(0);
      }
    const bool inside = (tix * TX + tx / n < g.N) && (tiy * TY + ty / n < g.N) && (tiz * TZ + tz < g.N);
    if (inside) {
      for (int qk = 0; qk < n; ++qk) {
        Real sk[n], dk[n];
#pragma unroll
        for (int l = 0; l < n; ++l) {
          sk[l] = sS[qk * n + l];
          dk[l] = sD[qk * n + l];
        }
        QPIn<3, Real> in;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const int base = (f * NPZ + tz * P) * PLANE + col;
          Real b = sk[0] * YB[base], dx = sk[0] * YX[base], dy = sk[0] * YY[base], dz = dk[0] * YB[base];
#pragma unroll
          for (int l = 1; l < n; ++l) {
            const int o = base + l * PLANE;
            b = fmac(sk[l], YB[o], b);
            dx = fmac(sk[l], YX[o], dx);
            dy = fmac(sk[l], YY[o], dy);
            dz = fmac(dk[l], YB[o], dz);
          }
          if (f < 3) {
            in.gu[f][0] = dx;
            in.gu[f][1] = dy;
            in.gu[f][2] = dz;
          } else {
            in.ph = b;
            in.gph[0] = dx;
            in.gph[1] = dy;
            in.gph[2] = dz;
          }
        }
        QPOut<3, Real> o;
        pw(tile, (long long)(tz * n + qk) * PLANE + col, in, o);
#pragma unroll
        for (int l = 0; l < n; ++l) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int oi = ((k * TZ + tz) * n + l) * PLANE + col;
            ZB[oi] = fmac(dk[l], o.cu[k][2], ZB[oi]);
            ZX[oi] = fmac(sk[l], o.cu[k][0], ZX[oi]);
            ZY[oi] = fmac(sk[l], o.cu[k][1], ZY[oi]);
          }
          const int oi = ((3 * TZ + tz) * n + l) * PLANE + col;
          ZB[oi] = fmac(sk[l], o.cv, fmac(dk[l], o.cg[2], ZB[oi]));
          ZX[oi] = fmac(sk[l], o.cg[0], ZX[oi]);
          ZY[oi] = fmac(sk[l], o.cg[1], ZY[oi]);
        }
      }
    }
  }
  __syncthreads();
  // transposed y-pass into WB, WD [NF][NPZ][NPY][QPX] (reusing XB, XD): node row r of plane t
  Real* WB = XB;
  Real* WD = XD;
  for (int t = tz; t < NPZ; t += TZ) {
    const int zlo = t == 0 ? 0 : (t - 1) / P, zhi = t / P < TZ - 1 ? t / P : TZ - 1;
    for (int r = ty; r < NPY; r += QPY) {
      const int ylo = r == 0 ? 0 : (r - 1) / P, yhi = r / P < TY - 1 ? r / P : TY - 1;
      Real wb[NF], wd[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        wb[f] = Real(0);
        wd[f] = Real(0);
      }
      for (int cz = zlo; cz <= zhi; ++cz) {
        const int lz = t - cz * P;
        for (int cy = ylo; cy <= yhi; ++cy) {
          const int ly = r - cy * P;
#pragma unroll
          for (int qj = 0; qj < n; ++qj) {
            const Real s = sS[qj * n + ly], d = sD[qj * n + ly];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              const int o = ((f * TZ + cz) * n + lz) * PLANE + (cy * n + qj) * QPX + tx;
              wb[f] = fmac(s, ZB[o], fmac(d, ZY[o], wb[f]));
              wd[f] = fmac(s, ZX[o], wd[f]);
            }
          }
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int o = ((f * NPZ + t) * NPY + r) * QPX + tx;
        WB[o] = wb[f];
        WD[o] = wd[f];
      }
    }
  }
  __syncthreads();
  // transposed x-pass and store
  for (int t = tz; t < NPZ; t += TZ)
    for (int r = ty; r < NPY; r += QPY)
      for (int s = tx; s < NPX; s += QPX) {
        const int gx = x0 + s, gy = y0 + r, gz = z0 + t;
        if (gx >= g.n1 || gy >= g.n1 || gz >= g.n1) continue;
        const int xlo = s == 0 ? 0 : (s - 1) / P, xhi = s / P < TX - 1 ? s / P : TX - 1;
        Real acc[NF] = {Real(0), Real(0), Real(0), Real(0)};
        for (int cx = xlo; cx <= xhi; ++cx) {
          const int k = s - cx * P;
#pragma unroll
          for (int qi = 0; qi < n; ++qi) {
            const Real sv = sS[qi * n + k], dv = sD[qi * n + k];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              const int o = ((f * NPZ + t) * NPY + r) * QPX + cx * n + qi;
              acc[f] = fmac(sv, WB[o], fmac(dv, WD[o], acc[f]));
            }
          }
        }
        const bool below = cut_below(g, tiz, t, NPZ, gx);
        const long long node = below ? cut_copy(g, gx, gy) : gx + n1 * gy + n1sq * gz;
        const bool low = (s == 0 && tix > 0) || (r == 0 && tiy > 0) || (t == 0 && tiz > 0 && !cut_above(g, tiz, t, gx));
        const bool high = (s == NPX - 1 && tix < g.ntile[0] - 1) || (r == NPY - 1 && tiy < g.ntile[1] - 1) ||
                          (t == NPZ - 1 && tiz < g.ntile[2] - 1 && !below);
        unsigned char m = 0;
        if (oa.outmask != OUT_RAW) {
          m = flags[node];
          if (oa.outmask == OUT_ZERO_DIRICHLET) m &= dirichlet_bits(3);
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const long long gi = f * g.nn + node;
          if ((m >> f) & 1u) {
            if (!low) dst[gi] = oa.outmask == OUT_IDENTITY ? src[gi] : Store(0);
          } else if (low || high) {
            atomicAdd(dst + gi, cvt<Store>(acc[f]));
          } else {
            dst[gi] = cvt<Store>(acc[f]);
          }
        }
      }
}

template <int P, typename Real>
constexpr size_t op3d_smem() {
  using T = Tile3<P>;
  constexpr int NF = 4, PLANE = T::QPX * T::QPY;
  return sizeof(Real) * (size_t)(NF * T::NPZ * T::NPY * T::NPX + 2 * NF * T::NPZ * T::NPY * T::QPX +
                                 3 * NF * T::NPZ * PLANE + 3 * NF * T::TZ * T::n * PLANE + 2 * T::n * T::n);
}

}  // namespace pff
