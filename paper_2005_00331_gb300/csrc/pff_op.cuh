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
// Pointwise residual of Eq. (residual) from the evaluated state (FP64):
// u-test  g(phi~) sigma^+ + sigma^-,  phi-test  g'(phi) E_s^+ - (G_c/eps)(1 - phi),
// grad-test G_c eps grad phi. Stored per point: g(phi~), G_c, lambda, mu.
template <int DIM, int SPLIT>
struct PWRes {
  const double* st;  // [tile][4][qpt]
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
};

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
  static constexpr int TX = 8, TY = (P == 1 ? 16 : (P == 2 ? 8 : 4));
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
        const long long node = gx + (long long)g.n1 * gy;
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
      const long long node = gx + (long long)g.n1 * gy;
      const bool low = (s == 0 && tix > 0) || (r == 0 && tiy > 0);
      const bool high = (s == NPX - 1 && tix < g.ntile[0] - 1) || (r == NPY - 1 && tiy < g.ntile[1] - 1);
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
// copies the next tile's node patch and per-point data into shared memory with cp.async while it
// computes the current tile (NSTAGE = 2; with NSTAGE = 1 the copy for the next tile overlaps the
// store phase only). The arithmetic is that of k_op2d.
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

template <int P, typename Real>
struct Stage2 {
  static constexpr int NSTAGE = sizeof(Real) == 4 ? 2 : 1;
};

template <int P, typename Real, typename Store, int SPLIT>
__global__ void __launch_bounds__(Tile2<P>::NT)
k_jac2_staged(const Store* __restrict__ src, Store* __restrict__ dst, const unsigned char* __restrict__ flags,
              Geom g, Tab<Real> tb, const Real* __restrict__ qpg, int mode, OpArgs oa) {
  using T = Tile2<P>;
  constexpr int TX = T::TX, TY = T::TY, n = T::n, NF = 3;
  constexpr int NPX = T::NPX, NPY = T::NPY, QPX = T::QPX;
  constexpr int QPT = T::QPX * T::QPY;
  constexpr int NV = qp_nv(2, SPLIT);
  constexpr int NS = Stage2<P, Real>::NSTAGE;
  constexpr int NT = T::NT;
  constexpr int XS = NF * NPY * NPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* QPs = reinterpret_cast<Real*>(smem_raw);                  // [NS][NV][QPT]
  Store* Xs = reinterpret_cast<Store*>(QPs + NS * NV * QPT);      // [NS][NF][NPY][NPX] raw copies
  Real* X = reinterpret_cast<Real*>(Xs + NS * XS);                // [NF][NPY][NPX] masked, compute type
  Real* UB = X + XS;                                              // [NF][TY][n][QPX]
  Real* UD = UB + NF * TY * n * QPX;
  Real* sS = UD + NF * TY * n * QPX;
  Real* sD = sS + n * n;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * QPX + tx;
  if (tid < n * n) {
    sS[tid] = tb.S[tid / n][tid % n];
    sD[tid] = tb.D[tid / n][tid % n];
  }
  const long long ntiles = g.ntiles;
  auto prefetch = [&](long long tile, int st) {
    const int tix = int(tile % g.ntile[0]), tiy = int(tile / g.ntile[0]);
    const int x0 = tix * TX * P, y0 = tiy * TY * P;
    Store* xs = Xs + st * XS;
    for (int i = tid; i < XS; i += NT) {
      const int s = i % NPX, r = (i / NPX) % NPY, f = i / (NPX * NPY);
      const int gx = x0 + s, gy = y0 + r;
      const bool ok = gx < g.n1 && gy < g.n1;
      const long long gi = ok ? f * g.nn + gx + (long long)g.n1 * gy : 0;
      cp_async_bytes(xs + i, src + gi, ok, (int)sizeof(Store));
    }
    const char* qsrc = reinterpret_cast<const char*>(qpg + tile * (long long)NV * QPT);
    char* qdst = reinterpret_cast<char*>(QPs + st * NV * QPT);
    constexpr int NCH = NV * QPT * (int)sizeof(Real) / 16;
    for (int i = tid; i < NCH; i += NT) cp_async16(qdst + 16 * i, qsrc + 16 * i);
  };

  int it = 0;
  if ((long long)blockIdx.x < ntiles) prefetch(blockIdx.x, 0);
  cp_async_commit();
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int st = NS == 2 ? (it & 1) : 0;
    if constexpr (NS == 2) {
      const long long nxt = tile + gridDim.x;
      if (nxt < ntiles) prefetch(nxt, st ^ 1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int tix = int(tile % g.ntile[0]), tiy = int(tile / g.ntile[0]);
    const int x0 = tix * TX * P, y0 = tiy * TY * P;
    // masked compute-type node patch
    const Store* xs = Xs + st * XS;
    for (int rs = tid; rs < NPY * NPX; rs += NT) {
      const int s = rs % NPX, r = rs / NPX;
      const int gx = x0 + s, gy = y0 + r;
      unsigned char m = 0;
      if (oa.inmask != IN_RAW && gx < g.n1 && gy < g.n1) {
        m = flags[gx + (long long)g.n1 * gy];
        if (oa.inmask == IN_DIRICHLET) m &= dirichlet_bits(2);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int i = f * NPY * NPX + rs;
        X[i] = ((m >> f) & 1u) ? Real(0) : cvt<Real>(xs[i]);
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
        pw(0, (long long)(ty * n + qj) * QPX + tx, in, o);
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
    if constexpr (NS == 1) {
      // the staging buffers are free: start the next tile's copies under the store phase
      const long long nxt = tile + gridDim.x;
      if (nxt < ntiles) prefetch(nxt, 0);
      cp_async_commit();
    }
    for (int rs = tid; rs < NPY * NPX; rs += NT) {
      const int s = rs % NPX, r = rs / NPX;
      const int gx = x0 + s, gy = y0 + r;
      if (gx >= g.n1 || gy >= g.n1) continue;
      const int ylo = r == 0 ? 0 : (r - 1) / P, yhi = r / P < TY - 1 ? r / P : TY - 1;
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
      const long long node = gx + (long long)g.n1 * gy;
      const bool low = (s == 0 && tix > 0) || (r == 0 && tiy > 0);
      const bool high = (s == NPX - 1 && tix < g.ntile[0] - 1) || (r == NPY - 1 && tiy < g.ntile[1] - 1);
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
  cp_async_wait<0>();
}

template <int P, typename Real, typename Store, int SPLIT>
constexpr size_t jac2_staged_smem() {
  using T = Tile2<P>;
  constexpr int NS = Stage2<P, Real>::NSTAGE;
  constexpr int XS = 3 * T::NPY * T::NPX;
  return sizeof(Real) * (size_t)NS * qp_nv(2, SPLIT) * T::QPX * T::QPY + sizeof(Store) * (size_t)NS * XS +
         sizeof(Real) * (size_t)(XS + 2 * 3 * T::TY * T::n * T::QPX + 2 * T::n * T::n);
}

// ===========================================================================================
// 3D operator kernel.
template <int P, typename Real, class PW>
__global__ void __launch_bounds__(256)
k_op3d(const Real* __restrict__ src, Real* __restrict__ dst, const unsigned char* __restrict__ flags,
       Geom g, Tab<Real> tb, PW pw, OpArgs oa) {
  constexpr int TX = TileCfg<3, P>::TX, TY = TileCfg<3, P>::TY, TZ = TileCfg<3, P>::TZ;
  constexpr int n = P + 1, NF = 4;
  constexpr int NPX = TX * P + 1, NPY = TY * P + 1, NPZ = TZ * P + 1;
  constexpr int QPX = TX * n, QPY = TY * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* X = reinterpret_cast<Real*>(smem_raw);          // [NF][NPZ][NPY][NPX]; later W* and output
  Real* XB = X + NF * NPZ * NPY * NPX;                   // [NF][NPZ][NPY][QPX]
  Real* XD = XB + NF * NPZ * NPY * QPX;
  Real* YB = XD + NF * NPZ * NPY * QPX;                  // [NF][NPZ][QPY][QPX]
  Real* YX = YB + NF * NPZ * QPY * QPX;
  Real* YY = YX + NF * NPZ * QPY * QPX;
  Real* ZB = YY + NF * NPZ * QPY * QPX;                  // [NF][TZ][n][QPY][QPX]
  Real* ZX = ZB + NF * TZ * n * QPY * QPX;
  Real* ZY = ZX + NF * TZ * n * QPY * QPX;

  const long long tile = blockIdx.x;
  const int tx = int(tile % g.ntile[0]);
  const int ty = int((tile / g.ntile[0]) % g.ntile[1]);
  const int tz = int(tile / ((long long)g.ntile[0] * g.ntile[1]));
  const int x0 = tx * TX * P, y0 = ty * TY * P, z0 = tz * TZ * P;
  const int cx0 = tx * TX, cy0 = ty * TY, cz0 = tz * TZ;
  const long long n1 = g.n1, n1sq = n1 * n1;

  for (int i = threadIdx.x; i < NF * NPZ * NPY * NPX; i += blockDim.x) {
    const int s = i % NPX, r = (i / NPX) % NPY, t = (i / (NPX * NPY)) % NPZ, f = i / (NPX * NPY * NPZ);
    const int gx = x0 + s, gy = y0 + r, gz = z0 + t;
    Real v = 0;
    if (gx < g.n1 && gy < g.n1 && gz < g.n1) {
      const long long node = gx + n1 * gy + n1sq * gz;
      v = load_node(src, flags, node, f * g.nn + node, f, 3, oa.inmask);
    }
    X[i] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NF * NPZ * NPY * QPX; i += blockDim.x) {
    const int c = i % QPX, row = i / QPX;
    const int cx = c / n, qi = c % n;
    const Real* xr = X + row * NPX + cx * P;
    Real b = 0, d = 0;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      b += tb.S[qi][k] * xr[k];
      d += tb.D[qi][k] * xr[k];
    }
    XB[i] = b;
    XD[i] = d;
  }
  __syncthreads();
  // y-pass: YB = S_y XB, YX = S_y XD, YY = D_y XB
  for (int i = threadIdx.x; i < NF * NPZ * QPY * QPX; i += blockDim.x) {
    const int c = i % QPX, qyc = (i / QPX) % QPY, ft = i / (QPX * QPY);  // ft = f*NPZ + t
    const int cy = qyc / n, qj = qyc % n;
    Real b = 0, dx = 0, dy = 0;
#pragma unroll
    for (int l = 0; l < n; ++l) {
      const int idx = (ft * NPY + cy * P + l) * QPX + c;
      b += tb.S[qj][l] * XB[idx];
      dx += tb.S[qj][l] * XD[idx];
      dy += tb.D[qj][l] * XB[idx];
    }
    YB[i] = b;
    YX[i] = dx;
    YY[i] = dy;
  }
  __syncthreads();
  // z-pass, pointwise, transposed z-pass: one thread per (cell layer, Gauss column)
  constexpr int PLANE = QPY * QPX;
  for (int i = threadIdx.x; i < TZ * PLANE; i += blockDim.x) {
    const int c = i % QPX, qyc = (i / QPX) % QPY, cz = i / PLANE;
    const int col = qyc * QPX + c;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const int o = ((f * TZ + cz) * n + l) * PLANE + col;
        ZB[o] = 0;
        ZX[o] = 0;
        ZY[o] = 0;
      }
    const bool inside = (cx0 + c / n < g.N) && (cy0 + qyc / n < g.N) && (cz0 + cz < g.N);
    if (!inside) continue;
    for (int qk = 0; qk < n; ++qk) {
      Real vb[NF], vx[NF], vy[NF], vz[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        Real b = 0, dx = 0, dy = 0, dz = 0;
#pragma unroll
        for (int l = 0; l < n; ++l) {
          const int idx = (f * NPZ + cz * P + l) * PLANE + col;
          const Real s = tb.S[qk][l];
          b += s * YB[idx];
          dx += s * YX[idx];
          dy += s * YY[idx];
          dz += tb.D[qk][l] * YB[idx];
        }
        vb[f] = b;
        vx[f] = dx;
        vy[f] = dy;
        vz[f] = dz;
      }
      QPIn<3, Real> in;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        in.gu[k][0] = vx[k];
        in.gu[k][1] = vy[k];
        in.gu[k][2] = vz[k];
      }
      in.ph = vb[3];
      in.gph[0] = vx[3];
      in.gph[1] = vy[3];
      in.gph[2] = vz[3];
      QPOut<3, Real> o;
      pw(tile, (long long)(cz * n + qk) * PLANE + col, in, o);
#pragma unroll
      for (int l = 0; l < n; ++l) {
        const Real s = tb.S[qk][l], d = tb.D[qk][l];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int oi = ((k * TZ + cz) * n + l) * PLANE + col;
          ZB[oi] += d * o.cu[k][2];
          ZX[oi] += s * o.cu[k][0];
          ZY[oi] += s * o.cu[k][1];
        }
        const int oi = ((3 * TZ + cz) * n + l) * PLANE + col;
        ZB[oi] += s * o.cv + d * o.cg[2];
        ZX[oi] += s * o.cg[0];
        ZY[oi] += s * o.cg[1];
      }
    }
  }
  __syncthreads();
  // transposed y-pass into WB, WD [NF][NPZ][NPY][QPX] (reusing XB, XD)
  Real* WB = XB;
  Real* WD = XD;
  for (int i = threadIdx.x; i < NF * NPZ * NPY * QPX; i += blockDim.x) {
    const int c = i % QPX, r = (i / QPX) % NPY, t = (i / (QPX * NPY)) % NPZ, f = i / (QPX * NPY * NPZ);
    int zlo, zhi, ylo, yhi;
    cells_of_node<P>(t, TZ, zlo, zhi);
    cells_of_node<P>(r, TY, ylo, yhi);
    Real wb = 0, wd = 0;
    for (int cz = zlo; cz <= zhi; ++cz) {
      const int lz = t - cz * P;
      for (int cy = ylo; cy <= yhi; ++cy) {
        const int ly = r - cy * P;
        const int base = ((f * TZ + cz) * n + lz) * PLANE + (cy * n) * QPX + c;
#pragma unroll
        for (int qj = 0; qj < n; ++qj) {
          const int o = base + qj * QPX;
          wb += tb.S[qj][ly] * ZB[o] + tb.D[qj][ly] * ZY[o];
          wd += tb.S[qj][ly] * ZX[o];
        }
      }
    }
    WB[i] = wb;
    WD[i] = wd;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NF * NPZ * NPY * NPX; i += blockDim.x) {
    const int s = i % NPX, row = i / NPX;
    int xlo, xhi;
    cells_of_node<P>(s, TX, xlo, xhi);
    Real acc = 0;
    for (int cx = xlo; cx <= xhi; ++cx) {
      const int k = s - cx * P;
      const Real* wb = WB + row * QPX + cx * n;
      const Real* wd = WD + row * QPX + cx * n;
#pragma unroll
      for (int qi = 0; qi < n; ++qi) acc += tb.S[qi][k] * wb[qi] + tb.D[qi][k] * wd[qi];
    }
    X[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NF * NPZ * NPY * NPX; i += blockDim.x) {
    const int s = i % NPX, r = (i / NPX) % NPY, t = (i / (NPX * NPY)) % NPZ, f = i / (NPX * NPY * NPZ);
    const int gx = x0 + s, gy = y0 + r, gz = z0 + t;
    if (gx >= g.n1 || gy >= g.n1 || gz >= g.n1) continue;
    const long long node = gx + n1 * gy + n1sq * gz;
    const bool low = (s == 0 && tx > 0) || (r == 0 && ty > 0) || (t == 0 && tz > 0);
    const bool high = (s == NPX - 1 && tx < g.ntile[0] - 1) || (r == NPY - 1 && ty < g.ntile[1] - 1) ||
                      (t == NPZ - 1 && tz < g.ntile[2] - 1);
    store_node(dst, src, flags, node, f * g.nn + node, f, 3, X[i], low, high, oa.outmask);
  }
}

template <int P, typename Real>
constexpr size_t op3d_smem() {
  constexpr int TX = TileCfg<3, P>::TX, TY = TileCfg<3, P>::TY, TZ = TileCfg<3, P>::TZ;
  constexpr int n = P + 1, NF = 4, NPX = TX * P + 1, NPY = TY * P + 1, NPZ = TZ * P + 1;
  constexpr int QPX = TX * n, QPY = TY * n;
  return sizeof(Real) * (size_t)(NF * NPZ * NPY * NPX + 2 * NF * NPZ * NPY * QPX + 3 * NF * NPZ * QPY * QPX +
                                 3 * NF * TZ * n * QPY * QPX);
}

}  // namespace pff
