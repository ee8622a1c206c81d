// pff_kernels.cu -- launch counter, dense coarse inverses, transfers, vector, Chebyshev,
// CG-Lanczos and Newton-step kernels of libpff (per-point setup, diagonal, parameter gradient and
// coarse assembly live in pff_qp.cu, pff_diag.cu and pff_pgrad.cu).
#include <cstdint>
#include <atomic>

#include "pff_kernels.h"
#include "pff_launch.h"
#include "pff_op.cuh"
#include "pff_point.cuh"

namespace pff {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }


// In-place Gauss-Jordan inversion without pivoting, blocked by GJB pivots. One block step with
// pivot block K (rows/columns k0 .. k0+bk-1) and P = A_KK^{-1} performs
//   A_ij -= A_iK P A_Kj (i, j outside K),  A_Kj = P A_Kj,  A_iK = -A_iK P,  A_KK = P,
// which is bk consecutive pointwise Gauss-Jordan steps at once. Three launches per step: the
// pivot block inverse (one CTA), the panels W = P A_K* and C = A_*K, and the rank-bk update.
constexpr int GJB = 32;

template <typename Real>
__global__ void __launch_bounds__(GJB * GJB) k_gj_pivot(const Real* __restrict__ A, int n, int k0, int bk,
                                                         Real* __restrict__ P) {
  __shared__ Real s[GJB][GJB + 1];
  const int i = threadIdx.y, j = threadIdx.x;
  const bool in = i < bk && j < bk;
  s[i][j] = in ? A[(long long)(k0 + i) * n + k0 + j] : Real(0);
  __syncthreads();
  __shared__ Real inv;
  for (int m = 0; m < bk; ++m) {
    // one division per step (FP64 division is slow on this part): the other threads multiply
    if (i == 0 && j == 0) inv = Real(1) / s[m][m];
    __syncthreads();
    const Real r = inv, aim = s[i][m], amj = s[m][j], aij = s[i][j];
    __syncthreads();
    Real v;
    if (i == m) v = (j == m) ? r : amj * r;
    else if (j == m) v = -aim * r;
    else v = aij - aim * (amj * r);
    if (in) s[i][j] = v;
    __syncthreads();
  }
  if (in) P[i * GJB + j] = s[i][j];
}

// W[m][j] = (P A_K*)[m][j] for j outside K and P[m][j - k0] inside; C[i][m] = A[i][k0 + m].
template <typename Real>
__global__ void k_gj_panels(const Real* __restrict__ A, int n, int k0, int bk, const Real* __restrict__ P,
                            Real* __restrict__ W, Real* __restrict__ C) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < (long long)bk * n) {
    const int m = int(t / n), j = int(t % n);
    Real v;
    if (j >= k0 && j < k0 + bk) {
      v = P[m * GJB + (j - k0)];
    } else {
      v = Real(0);
      for (int l = 0; l < bk; ++l) v = fmac(P[m * GJB + l], A[(long long)(k0 + l) * n + j], v);
    }
    W[(long long)m * n + j] = v;
  } else if (t < 2LL * bk * n) {
    const long long u = t - (long long)bk * n;
    const int i = int(u / bk), m = int(u % bk);
    C[(long long)i * GJB + m] = A[(long long)i * n + k0 + m];
  }
}

// Rank-bk update on 16 x 16 tiles of A.
template <typename Real>
__global__ void __launch_bounds__(256) k_gj_rank(Real* __restrict__ A, int n, int k0, int bk,
                                                 const Real* __restrict__ W, const Real* __restrict__ C) {
  __shared__ Real cs[16][GJB + 1];
  __shared__ Real ws[GJB][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  const int tid = ty * 16 + tx;
  for (int e = tid; e < 16 * GJB; e += 256) {
    const int r = e / GJB, m = e % GJB;
    cs[r][m] = (i0 + r < n && m < bk) ? C[(long long)(i0 + r) * GJB + m] : Real(0);
    const int mm = e / 16, cc = e % 16;
    ws[mm][cc] = (j0 + cc < n && mm < bk) ? W[(long long)mm * n + j0 + cc] : Real(0);
  }
  __syncthreads();
  const int i = i0 + ty, j = j0 + tx;
  if (i >= n || j >= n) return;
  Real* aij = A + (long long)i * n + j;
  if (i >= k0 && i < k0 + bk) {
    *aij = ws[i - k0][tx];
    return;
  }
  Real sum = Real(0);
  for (int m = 0; m < bk; ++m) sum = fmac(cs[ty][m], ws[m][tx], sum);
  *aij = (j >= k0 && j < k0 + bk) ? -sum : *aij - sum;
}

long long gj_buffer_size(int n) { return (long long)GJB * GJB + 2LL * GJB * n; }

template <typename Real>
cudaError_t launch_gj_inverse(Real* A, int n, Real* buf, cudaStream_t s) {
  Real* P = buf;
  Real* W = buf + GJB * GJB;
  Real* C = W + (long long)GJB * n;
  const dim3 tile(16, 16), grid((n + 15) / 16, (n + 15) / 16);
  for (int k0 = 0; k0 < n; k0 += GJB) {
    const int bk = n - k0 < GJB ? n - k0 : GJB;
    count_launch(); k_gj_pivot<Real><<<1, dim3(GJB, GJB), 0, s>>>(A, n, k0, bk, P);
    count_launch(); k_gj_panels<Real><<<grid_for(2LL * bk * n, 64), 64, 0, s>>>(A, n, k0, bk, P, W, C);
    count_launch(); k_gj_rank<Real><<<grid, tile, 0, s>>>(A, n, k0, bk, W, C);
  }
  return cudaGetLastError();
}
template cudaError_t launch_gj_inverse<double>(double*, int, double*, cudaStream_t);
template cudaError_t launch_gj_inverse<float>(float*, int, float*, cudaStream_t);

template <typename Real>
__global__ void k_gemv(const Real* __restrict__ A, int n, int m, const Real* __restrict__ x, Real* __restrict__ y,
                       double alpha, double beta) {
  pdl_wait();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const Real* row = A + (long long)warp * m;
  Real s = Real(0);
  for (int j = lane; j < m; j += 32) s = fmac(row[j], x[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[warp] = (beta == 0.0 ? Real(0) : Real(beta) * y[warp]) + Real(alpha) * s;
}

template <typename Real>
cudaError_t launch_gemv(const Real* A, int n, int m, const Real* x, Real* y, double alpha, double beta,
                        cudaStream_t s) {
  return launch_k(k_gemv<Real>, dim3(grid_for((long long)n * 32)), dim3(BLK), 0, s, A, n, m, x, y, alpha, beta);
}
template cudaError_t launch_gemv<double>(const double*, int, int, const double*, double*, double, double,
                                         cudaStream_t);
template cudaError_t launch_gemv<float>(const float*, int, int, const float*, float*, double, double, cudaStream_t);

// ===========================================================================================
// Transfers between a coarse level (Nc cells) and its fine level (2 Nc cells), same degree.
// The 1D tables live in shared memory in the vector precision: indexed per thread (the fine offset and
// the coarse local node differ across a warp), they would be divergent constant-bank reads as kernel
// parameters, and double entries would need conversions on the FP64 pipe.
template <int DIM, int P, typename Real>
__global__ void k_prolong(const Real* __restrict__ xc, Real* __restrict__ yf, const unsigned char* __restrict__ flf,
                          Geom gc, Geom gf, XferTab xt, int accumulate) {
  constexpr int NO = 2 * P + 1, NK = P + 1;
  __shared__ Real E[NO][NK];
  for (int i = threadIdx.x; i < NO * NK; i += blockDim.x) E[i / NK][i % NK] = Real(xt.E[i / NK][i % NK]);
  pdl_wait();
  __syncthreads();
  // 32-bit index arithmetic (node counts fit in 32 bits, checked at setup)
  const int nd = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (nd >= gf.nn) return;
  const unsigned n1 = (unsigned)gf.n1;
  unsigned rem = (unsigned)nd;
  if (nd >= gf.ngrid) {  // copy of a cut slit node: the coarse function's value at its grid point
    const unsigned k = unsigned(nd - gf.ngrid);
    const unsigned x = k % (unsigned)gf.cut_x, y = k / (unsigned)gf.cut_x;
    rem = x + n1 * (DIM == 2 ? (unsigned)gf.cut_row : y + n1 * (unsigned)gf.cut_row);
  }
  int C[3] = {0, 0, 0}, o[3] = {0, 0, 0};
#pragma unroll
  for (int t = 0; t < DIM; ++t) {
    const int i = int(rem % n1);
    rem /= n1;
    int c = i / (2 * P);
    if (c > gc.N - 1) c = gc.N - 1;
    C[t] = c;
    o[t] = i - 2 * P * c;
  }
  Real wx[NK], wy[NK], wz[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    wx[k] = E[o[0]][k];
    wy[k] = E[o[1]][k];
    wz[k] = DIM == 3 ? E[o[2]][k] : Real(1);
  }
  const unsigned char fl = flf[nd];
  const long long cbase = (long long)C[0] * P + (long long)gc.n1 * (C[1] * P + (DIM == 3 ? (long long)gc.n1 * C[2] * P : 0));
  // the coarse values are loaded whatever the fine node's mask (applied below), so that the loads do not
  // wait for the flag byte
#pragma unroll
  for (int f = 0; f <= DIM; ++f) {
    Real v = Real(0);
    {
      const Real* xb = xc + f * gc.nn + cbase;
#pragma unroll
      for (int kz = 0; kz < (DIM == 3 ? NK : 1); ++kz)
#pragma unroll
        for (int ky = 0; ky < NK; ++ky) {
          const Real* row = xb + (long long)ky * gc.n1 + (DIM == 3 ? (long long)kz * gc.n1 * gc.n1 : 0);
          Real sx = Real(0);
#pragma unroll
          for (int kx = 0; kx < NK; ++kx) sx += wx[kx] * row[kx];
          v += wz[kz] * wy[ky] * sx;
        }
    }
    if ((fl >> f) & 1u) v = Real(0);
    Real* y = yf + f * gf.nn + nd;
    *y = accumulate ? *y + v : v;
  }
}

// Restriction = transpose of the prolongation. Per direction, the fine nodes that see coarse node J
// (J = P c + k, 0 <= k < P) lie at fine offsets o in [-2P, 2P] from the first fine node 2P c of coarse
// cell c, with weight W[k][o + 2P]: E[o][k] for o >= 0 and, for a vertex (k = 0), E[o + 2P][P] from
// the cell on the left for o < 0.
template <int DIM, int P, typename Real>
__global__ void k_restrict(const Real* __restrict__ xf, Real* __restrict__ yc, const unsigned char* __restrict__ flf,
                           const unsigned char* __restrict__ flc, Geom gf, Geom gc, XferTab xt, int mask_fine,
                           ChebStart<Real> cs) {
  constexpr int NW = 4 * P + 1;
  __shared__ Real W[P][NW];
  for (int i = threadIdx.x; i < P * NW; i += blockDim.x) {
    const int k = i / NW, o = i % NW - 2 * P;
    W[k][i % NW] = o >= 0 ? Real(xt.E[o][k]) : (k == 0 ? Real(xt.E[o + 2 * P][P]) : Real(0));
  }
  pdl_wait();
  __syncthreads();
  const long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (nd >= gc.nn) return;
  long long rem = nd;
  int b[3] = {0, 0, 0}, kk[3] = {0, 0, 0};
#pragma unroll
  for (int t = 0; t < DIM; ++t) {
    const int J = int(rem % gc.n1);
    rem /= gc.n1;
    const int c = J / P;
    kk[t] = J - P * c;
    b[t] = 2 * P * c;
  }
  const unsigned char fc = flc[nd];
  Real acc[DIM + 1];
#pragma unroll
  for (int f = 0; f <= DIM; ++f) acc[f] = Real(0);
  // in 3D only the innermost direction is unrolled: the (4p+1)^3 stencil unrolled whole made this
  // file take minutes to compile (2D unrolls the whole (4p+1)^2 stencil as before)
#pragma unroll 1
  for (int oz = 0; oz < (DIM == 3 ? NW : 1); ++oz) {
    const int iz = DIM == 3 ? b[2] + oz - 2 * P : 0;
    if (DIM == 3 && (iz < 0 || iz >= gf.n1)) continue;
    const Real w3 = DIM == 3 ? W[kk[2]][oz] : Real(1);
    if (w3 == Real(0)) continue;
#pragma unroll(DIM == 2 ? NW : 1)
    for (int oy = 0; oy < NW; ++oy) {
      const int iy = b[1] + oy - 2 * P;
      if (iy < 0 || iy >= gf.n1) continue;
      const Real w2 = w3 * W[kk[1]][oy];
      if (w2 == Real(0)) continue;
      const long long rowb = (long long)gf.n1 * (iy + (DIM == 3 ? (long long)gf.n1 * iz : 0));
#pragma unroll
      for (int ox = 0; ox < NW; ++ox) {
        const int ix = b[0] + ox - 2 * P;
        if (ix < 0 || ix >= gf.n1) continue;
        const Real w = w2 * W[kk[0]][ox];
        if (w == Real(0)) continue;
        const long long fn = rowb + ix;
        const unsigned char ff = mask_fine ? flf[fn] : 0;
#pragma unroll
        for (int f = 0; f <= DIM; ++f)
          if (!((ff >> f) & 1u)) acc[f] += w * xf[f * gf.nn + fn];
        if (gf.cut && (DIM == 2 ? iy : iz) == gf.cut_row && ix < gf.cut_x) {
          // a cut slit node: its copy sees the same coarse functions (restriction = transpose)
          const long long fc = cut_copy(gf, ix, DIM == 3 ? iy : 0);
          const unsigned char fcm = mask_fine ? flf[fc] : 0;
#pragma unroll
          for (int f = 0; f <= DIM; ++f)
            if (!((fcm >> f) & 1u)) acc[f] += w * xf[f * gf.nn + fc];
        }
      }
    }
  }
  Real a0 = Real(0), a1 = Real(0);
  if (cs.on) {
    a0 = Real(cs.c0s) * cs.inv_lam[0];
    a1 = Real(cs.c0s) * cs.inv_lam[1];
  }
  Real di[DIM + 1];  // loaded before the stores below, which the compiler cannot tell apart from them
#pragma unroll
  for (int f = 0; f <= DIM; ++f) di[f] = cs.on ? cs.dinv[f * gc.nn + nd] : Real(0);
#pragma unroll
  for (int f = 0; f <= DIM; ++f) {
    const long long gi = f * gc.nn + nd;
    const Real v = ((fc >> f) & 1u) ? Real(0) : acc[f];
    yc[gi] = v;
    if (cs.on) {
      const Real de = (f < DIM ? a0 : a1) * (di[f] * v);
      cs.d[gi] = de;
      cs.x[gi] = de;
    }
  }
}

// 2D restriction by tiles of coarse nodes (RCX x RCY coarse cells' nodes per CTA): the fine window that
// the tile's coarse functions touch is staged in shared memory (masked; a cut slit's copy is added to its
// grid node, which carries the same coarse weights), then contracted along x and along y. The restriction
// is the transpose of the tensor-product prolongation, so each coarse value takes 2 (4p+1) products
// instead of (4p+1)^2 gathers, and the CTA's loads are coalesced and independent of one another.
template <int P>
struct RTile2 {
  static constexpr int CXC = P == 1 ? 16 : P == 2 ? 8 : 4, CYC = P == 1 ? 8 : P == 2 ? 4 : P == 3 ? 3 : 2;
  static constexpr int CX = CXC * P, CY = CYC * P;                        // coarse nodes per CTA
  static constexpr int FX = 2 * CX + 4 * P - 1, FY = 2 * CY + 4 * P - 1;  // fine window
};
constexpr int RT_THREADS = 128;

template <int P, typename Real>
__global__ void __launch_bounds__(RT_THREADS)
k_restrict2(const Real* __restrict__ xf, Real* __restrict__ yc, const unsigned char* __restrict__ flf,
            const unsigned char* __restrict__ flc, Geom gf, Geom gc, XferTab xt, int mask_fine, ChebStart<Real> cs) {
  using T = RTile2<P>;
  constexpr int NW = 4 * P + 1, CX = T::CX, CY = T::CY, FX = T::FX, FY = T::FY;
  __shared__ Real W[P][NW];
  __shared__ Real F[3][FY][FX];   // masked fine window
  __shared__ Real Tx[3][FY][CX];  // the window contracted along x
  for (int i = threadIdx.x; i < P * NW; i += blockDim.x) {
    const int k = i / NW, o = i % NW - 2 * P;
    W[k][i % NW] = o >= 0 ? Real(xt.E[o][k]) : (k == 0 ? Real(xt.E[o + 2 * P][P]) : Real(0));
  }
  pdl_wait();
  const int ntx = (gc.n1 + CX - 1) / CX;
  const int J0 = int(blockIdx.x % (unsigned)ntx) * CX, I0 = int(blockIdx.x / (unsigned)ntx) * CY;
  const int fx0 = 2 * J0 - 2 * P, fy0 = 2 * I0 - 2 * P;  // window origin on the fine grid
  for (int i = threadIdx.x; i < FX * FY; i += blockDim.x) {
    const int wy = i / FX, wx = i - wy * FX;
    const int ix = fx0 + wx, iy = fy0 + wy;
    Real v[3] = {Real(0), Real(0), Real(0)};
    if (ix >= 0 && iy >= 0 && ix < gf.n1 && iy < gf.n1) {
      const long long fn = ix + (long long)gf.n1 * iy;
      const unsigned char ff = mask_fine ? flf[fn] : 0;
      Real x3[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) x3[f] = xf[f * gf.nn + fn];
#pragma unroll
      for (int f = 0; f < 3; ++f) v[f] = ((ff >> f) & 1u) ? Real(0) : x3[f];
      if (gf.cut && iy == gf.cut_row && ix < gf.cut_x) {
        const long long fcp = cut_copy(gf, ix, 0);
        const unsigned char fcm = mask_fine ? flf[fcp] : 0;
#pragma unroll
        for (int f = 0; f < 3; ++f)
          if (!((fcm >> f) & 1u)) v[f] += xf[f * gf.nn + fcp];
      }
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) F[f][wy][wx] = v[f];
  }
  __syncthreads();
  // coarse column jc (node J0 + jc, local basis k = jc mod P since J0 is a multiple of P) sees the fine
  // window columns 2P (jc / P) + o, o in [0, 4P]
  for (int i = threadIdx.x; i < FY * CX; i += blockDim.x) {
    const int wy = i / CX, jc = i - wy * CX;
    const int k = jc % P, wb = 2 * P * (jc / P);
    Real a[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int o = 0; o < NW; ++o) {
      const Real w = W[k][o];
#pragma unroll
      for (int f = 0; f < 3; ++f) a[f] += w * F[f][wy][wb + o];
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) Tx[f][wy][jc] = a[f];
  }
  __syncthreads();
  Real a0 = Real(0), a1 = Real(0);
  if (cs.on) {
    a0 = Real(cs.c0s) * cs.inv_lam[0];
    a1 = Real(cs.c0s) * cs.inv_lam[1];
  }
  for (int i = threadIdx.x; i < CY * CX; i += blockDim.x) {
    const int ic = i / CX, jc = i - ic * CX;
    const int J = J0 + jc, I = I0 + ic;
    if (J >= gc.n1 || I >= gc.n1) continue;
    const int k = ic % P, wb = 2 * P * (ic / P);
    Real acc[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int o = 0; o < NW; ++o) {
      const Real w = W[k][o];
#pragma unroll
      for (int f = 0; f < 3; ++f) acc[f] += w * Tx[f][wb + o][jc];
    }
    const long long nd = J + (long long)gc.n1 * I;
    const unsigned char fc = flc[nd];
    Real di[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) di[f] = cs.on ? cs.dinv[f * gc.nn + nd] : Real(0);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const long long gi = f * gc.nn + nd;
      const Real v = ((fc >> f) & 1u) ? Real(0) : acc[f];
      yc[gi] = v;
      if (cs.on) {
        const Real de = (f < 2 ? a0 : a1) * (di[f] * v);
        cs.d[gi] = de;
        cs.x[gi] = de;
      }
    }
  }
}

template <typename Real>
cudaError_t launch_prolong(int dim, int p, const Real* xc, Real* yf, const unsigned char* flags_f, const Geom& gc,
                           const Geom& gf, const XferTab& xt, bool accumulate, cudaStream_t s) {
  const unsigned gr = grid_for(gf.nn);
#define PFF_CASE(DD, PP)                                                                                 \
  if (dim == DD && p == PP)                                                                              \
    return launch_k(k_prolong<DD, PP, Real>, dim3(gr), dim3(BLK), 0, s, xc, yf, flags_f, gc, gf, xt,     \
                    accumulate ? 1 : 0);
  PFF_CASE(2, 1) PFF_CASE(2, 2) PFF_CASE(2, 3) PFF_CASE(2, 4)
  PFF_CASE(3, 1) PFF_CASE(3, 2) PFF_CASE(3, 3) PFF_CASE(3, 4)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t launch_restrict(int dim, int p, const Real* xf, Real* yc, const unsigned char* flags_f,
                            const unsigned char* flags_c, const Geom& gf, const Geom& gc, const XferTab& xt,
                            cudaStream_t s, bool mask_fine, const ChebStart<Real>* cs) {
  const unsigned gr = grid_for(gc.nn, 128);
  ChebStart<Real> off{};
  off.on = 0;
  const ChebStart<Real>& st = cs ? *cs : off;
  if (dim == 2 && !gc.cut) {  // coarse levels carry no slit copies
#define PFF_CASE2(PP)                                                                                    \
  if (p == PP) {                                                                                         \
    using T = RTile2<PP>;                                                                                \
    const unsigned g2 = (unsigned)(((gc.n1 + T::CX - 1) / T::CX) * ((gc.n1 + T::CY - 1) / T::CY));       \
    return launch_k(k_restrict2<PP, Real>, dim3(g2), dim3(RT_THREADS), 0, s, xf, yc, flags_f, flags_c, gf, \
                    gc, xt, mask_fine ? 1 : 0, st);                                                      \
  }
    PFF_CASE2(1) PFF_CASE2(2) PFF_CASE2(3) PFF_CASE2(4)
#undef PFF_CASE2
  }
#define PFF_CASE(DD, PP)                                                                                 \
  if (dim == DD && p == PP)                                                                              \
    return launch_k(k_restrict<DD, PP, Real>, dim3(gr), dim3(128), 0, s, xf, yc, flags_f, flags_c, gf, gc, \
                    xt, mask_fine ? 1 : 0, st);
  PFF_CASE(2, 1) PFF_CASE(2, 2) PFF_CASE(2, 3) PFF_CASE(2, 4)
  PFF_CASE(3, 1) PFF_CASE(3, 2) PFF_CASE(3, 3) PFF_CASE(3, 4)
#undef PFF_CASE
  return cudaErrorInvalidValue;
}

template cudaError_t launch_prolong<double>(int, int, const double*, double*, const unsigned char*, const Geom&,
                                            const Geom&, const XferTab&, bool, cudaStream_t);
template cudaError_t launch_prolong<float>(int, int, const float*, float*, const unsigned char*, const Geom&,
                                           const Geom&, const XferTab&, bool, cudaStream_t);
template cudaError_t launch_restrict<double>(int, int, const double*, double*, const unsigned char*,
                                             const unsigned char*, const Geom&, const Geom&, const XferTab&,
                                             cudaStream_t, bool, const ChebStart<double>*);
template cudaError_t launch_restrict<float>(int, int, const float*, float*, const unsigned char*,
                                            const unsigned char*, const Geom&, const Geom&, const XferTab&,
                                            cudaStream_t, bool, const ChebStart<float>*);

// Fine FE function evaluated at the coarse nodes (carries the state to coarse levels).
__global__ void k_state_interp(int dim, int p, const double* __restrict__ xf, double* __restrict__ yc, int nfields,
                               Geom gf, Geom gc, XferTab xt) {
  const long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (nd >= gc.nn) return;
  int base[3] = {0, 0, 0}, k[3] = {0, 0, 0};
  long long rem = nd;
  for (int t = 0; t < dim; ++t) {
    const int J = int(rem % gc.n1);
    rem /= gc.n1;
    int c = J / p;
    if (c > gc.N - 1) c = gc.N - 1;
    k[t] = J - c * p;
    base[t] = (2 * c + xt.FC[k[t]]) * p;  // first fine node of the fine cell holding the coarse node
  }
  for (int f = 0; f < nfields; ++f) {
    const double* x = xf + (long long)f * gf.nn;
    double v = 0.0;
    const int mz = dim == 3 ? p : 0;
    for (int cz = 0; cz <= mz; ++cz) {
      const double wz = dim == 3 ? xt.F[k[2]][cz] : 1.0;
      if (wz == 0.0) continue;
      for (int cy = 0; cy <= p; ++cy) {
        const double wy = xt.F[k[1]][cy];
        if (wy == 0.0) continue;
        for (int cx = 0; cx <= p; ++cx) {
          const double wx = xt.F[k[0]][cx];
          if (wx == 0.0) continue;
          long long fn = (base[0] + cx) + (long long)gf.n1 * (base[1] + cy);
          if (dim == 3) fn += (long long)gf.n1 * gf.n1 * (base[2] + cz);
          v += wz * wy * wx * x[fn];
        }
      }
    }
    yc[(long long)f * gc.nn + nd] = v;
  }
}

cudaError_t launch_state_interp(int dim, int p, const double* xf, double* yc, int nfields, const Geom& gf,
                                const Geom& gc, const XferTab& xt, cudaStream_t s) {
  count_launch(); k_state_interp<<<grid_for(gc.nn), BLK, 0, s>>>(dim, p, xf, yc, nfields, gf, gc, xt);
  return cudaGetLastError();
}

__global__ void k_coarse_active(int dim, int p, const unsigned char* __restrict__ flf, unsigned char* __restrict__ flc,
                                Geom gf, Geom gc, XferTab xt) {
  const long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (nd >= gc.nn) return;
  long long rem = nd, fn = 0, stride = 1;
  bool col = true;
  for (int t = 0; t < dim; ++t) {
    const int J = int(rem % gc.n1);
    rem /= gc.n1;
    int c = J / p;
    if (c > gc.N - 1) c = gc.N - 1;
    const int k = J - c * p;
    if (xt.COL[k] < 0) col = false;
    else fn += stride * (2 * p * c + xt.COL[k]);
    stride *= gf.n1;
  }
  const unsigned char bit = (unsigned char)(1u << dim);
  unsigned char fl = flc[nd] & (unsigned char)~bit;
  if (col && (flf[fn] & bit)) fl |= bit;
  flc[nd] = fl;
}

cudaError_t launch_coarse_active(int dim, int p, const unsigned char* flags_f, unsigned char* flags_c,
                                 const Geom& gf, const Geom& gc, const XferTab& xt, cudaStream_t s) {
  count_launch(); k_coarse_active<<<grid_for(gc.nn), BLK, 0, s>>>(dim, p, flags_f, flags_c, gf, gc, xt);
  return cudaGetLastError();
}

// ===========================================================================================
// Vector kernels.
template <typename Real>
__global__ void k_axpby(long long n, double a, const Real* __restrict__ x, double b, Real* __restrict__ y) {
  pdl_wait();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = Real(a * (double)x[e] + (b == 0.0 ? 0.0 : b * (double)y[e]));
}
template <>
__global__ void k_axpby<float>(long long n, double a, const float* __restrict__ x, double b, float* __restrict__ y) {
  pdl_wait();
  const float af = (float)a, bf = (float)b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = af * x[e] + (bf == 0.0f ? 0.0f : bf * y[e]);
}

template <typename Real>
cudaError_t launch_axpby(long long n, double a, const Real* x, double b, Real* y, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return launch_k(k_axpby<Real>, dim3((unsigned)g), dim3(BLK), 0, s, n, a, x, b, y);
}
template cudaError_t launch_axpby<double>(long long, double, const double*, double, double*, cudaStream_t);
template cudaError_t launch_axpby<float>(long long, double, const float*, double, float*, cudaStream_t);

// res = r - t, then t = 0 (the V-cycle's residual; leaves the apply buffer zeroed for the next apply);
// with cs.on also the first smoothing step of res.
template <typename Real>
__global__ void k_res_update(long long n, const Real* __restrict__ r, Real* __restrict__ t, Real* __restrict__ res,
                             ChebStart<Real> cs) {
  pdl_wait();
  Real a0 = Real(0), a1 = Real(0);
  if (cs.on) {
    a0 = Real(cs.c0s) * cs.inv_lam[0];
    a1 = Real(cs.c0s) * cs.inv_lam[1];
  }
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const Real v = r[e] - t[e];
    res[e] = v;
    t[e] = Real(0);
    if (cs.on) {
      const Real de = (e < cs.nu ? a0 : a1) * (cs.dinv[e] * v);
      cs.d[e] = de;
      cs.x[e] = de;
    }
  }
}
template <typename Real>
cudaError_t launch_res_update(long long n, const Real* r, Real* t, Real* res, const ChebStart<Real>& cs,
                              cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return launch_k(k_res_update<Real>, dim3((unsigned)g), dim3(BLK), 0, s, n, r, t, res, cs);
}
template cudaError_t launch_res_update<double>(long long, const double*, double*, double*, const ChebStart<double>&,
                                               cudaStream_t);
template cudaError_t launch_res_update<float>(long long, const float*, float*, float*, const ChebStart<float>&,
                                              cudaStream_t);

template <typename Ti, typename To>
__global__ void k_cast(long long n, const Ti* __restrict__ x, To* __restrict__ y) {
  pdl_wait();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = To(x[e]);
}
template <typename Ti, typename To>
cudaError_t launch_cast(long long n, const Ti* x, To* y, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return launch_k(k_cast<Ti, To>, dim3((unsigned)g), dim3(BLK), 0, s, n, x, y);
}
template cudaError_t launch_cast<double, float>(long long, const double*, float*, cudaStream_t);
template cudaError_t launch_cast<float, double>(long long, const float*, double*, cudaStream_t);

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// Grid of the reduction kernels: two CTAs of BLK threads per SM, fewer for short vectors (measured on
// the 2D Q2 256^2 Newton step: eight per SM made the CG-Lanczos update slower, 24 vs 19 us).
constexpr int RED_GRID_MAX = 152 * 2;
inline unsigned red_grid(long long n) {
  long long g = (n + BLK - 1) / BLK;
  if (g > RED_GRID_MAX) g = RED_GRID_MAX;
  return (unsigned)(g < 1 ? 1 : g);
}

template <typename Real>
__global__ void k_dot2_part(long long n, long long nu, const Real* __restrict__ x, const Real* __restrict__ y,
                            double* __restrict__ part) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = (double)x[e] * (double)y[e];
    if (e < nu) s0 += v;
    else s1 += v;
  }
  const double r0 = block_sum(s0, sh);
  const double r1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r0;
    part[2 * blockIdx.x + 1] = r1;
  }
}
__global__ void k_dot2_final(int nb, const double* __restrict__ part, double* __restrict__ res) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    s0 += part[2 * b];
    s1 += part[2 * b + 1];
  }
  const double r0 = block_sum(s0, sh);
  const double r1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    res[0] = r0;
    res[1] = r1;
  }
}

template <typename Real>
cudaError_t launch_dot2(long long n, long long nu, const Real* x, const Real* y, double* partial, double* res,
                        cudaStream_t s) {
  const unsigned g = red_grid(n);
  count_launch(); k_dot2_part<Real><<<g, BLK, 0, s>>>(n, nu, x, y, partial);
  count_launch(); k_dot2_final<<<1, BLK, 0, s>>>((int)g, partial, res);
  return cudaGetLastError();
}
template cudaError_t launch_dot2<double>(long long, long long, const double*, const double*, double*, double*,
                                         cudaStream_t);
template cudaError_t launch_dot2<float>(long long, long long, const float*, const float*, double*, double*,
                                        cudaStream_t);

// Multi-dot h_i = <V_i, w>: blockIdx.y selects a group of 4 basis vectors.
__global__ void k_mdot_part(long long n, int k, const double* __restrict__ V, const double* __restrict__ w,
                            double* __restrict__ part) {
  __shared__ double sh[32];
  const int i0 = blockIdx.y * 4;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double we = w[e];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i0 + j < k) s[j] += V[(long long)(i0 + j) * n + e] * we;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double r = block_sum(s[j], sh);
    if (threadIdx.x == 0 && i0 + j < k) part[(long long)(i0 + j) * gridDim.x + blockIdx.x] = r;
  }
}
__global__ void k_mdot_final(int nb, const double* __restrict__ part, double* __restrict__ h) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(long long)blockIdx.x * nb + b];
  const double r = block_sum(s, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = r;
}

cudaError_t launch_mdot(long long n, int k, const double* V, const double* w, double* partial, double* h,
                        cudaStream_t s) {
  const int nb = 152;
  dim3 grd(nb, (k + 3) / 4);
  count_launch(); k_mdot_part<<<grd, BLK, 0, s>>>(n, k, V, w, partial);
  count_launch(); k_mdot_final<<<k, BLK, 0, s>>>(nb, partial, h);
  return cudaGetLastError();
}

__global__ void k_maxpy(long long n, int k, const double* __restrict__ V, const double* __restrict__ h,
                        double* __restrict__ w, double sign) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += V[(long long)i * n + e] * h[i];
    w[e] += sign * acc;
  }
}

cudaError_t launch_maxpy(long long n, int k, const double* V, const double* h, double* w, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 8) g = 152 * 8;
  count_launch(); k_maxpy<<<(unsigned)g, BLK, 0, s>>>(n, k, V, h, w, -1.0);
  return cudaGetLastError();
}
cudaError_t launch_zupdate(long long n, int k, const double* Z, const double* y, double* x, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 8) g = 152 * 8;
  count_launch(); k_maxpy<<<(unsigned)g, BLK, 0, s>>>(n, k, Z, y, x, 1.0);
  return cudaGetLastError();
}

__global__ void k_normalize(long long n, const double* __restrict__ x, const double* __restrict__ inv,
                            double* __restrict__ y, float* __restrict__ y32) {
  const double a = inv[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e] * a;
    y[e] = v;
    if (y32) y32[e] = (float)v;
  }
}
cudaError_t launch_normalize(long long n, const double* x, const double* inv, double* y, float* y32,
                             cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  count_launch(); k_normalize<<<(unsigned)g, BLK, 0, s>>>(n, x, inv, y, y32);
  return cudaGetLastError();
}

// ===========================================================================================
// Classical Gram-Schmidt with reorthogonalisation (CGS2) of a new FGMRES direction w against the basis
// V_0 .. V_{k-1} (one instantiation per k <= CGS_KMAX), in three passes over the vectors:
//   MODE 0: h_i = <V_i, w>;
//   MODE 1: w -= sum_i V_i h_i, then h'_i = <V_i, w> of the updated w;
//   MODE 2: w -= sum_i V_i h_i, then out = (<w, w>, 0, 1 / |w|) of the updated w (1 / |w| = 0 for w = 0).
// Per element the update and the products are those of the separate passes. Each CTA leaves its partial
// sums in part; the last CTA to finish (counted in cnt, which it resets) adds them in CTA order, one warp
// per basis vector, so the results do not depend on timing.
constexpr int CGS_GRID = CGS_GRID_MAX;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int K, int MODE>
__global__ void __launch_bounds__(BLK) k_cgs_pass(long long n, const double* __restrict__ V,
                                                  const double* __restrict__ h, double* __restrict__ w,
                                                  double* __restrict__ part, double* __restrict__ out,
                                                  unsigned* __restrict__ cnt) {
  constexpr int NS = MODE == 2 ? 1 : K;  // sums per thread
  constexpr int KA = K > 0 ? K : 1;
  constexpr int NW = BLK / 32;
  __shared__ double sh[NS > 0 ? NS : 1][NW];
  __shared__ double shh[KA];
  __shared__ int last;
  if constexpr (MODE != 0 && K > 0)
    if ((int)threadIdx.x < K) shh[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double s[NS > 0 ? NS : 1];
#pragma unroll
  for (int i = 0; i < NS; ++i) s[i] = 0.0;
  // one element: the update (MODE 1, 2), then this thread's products
  auto element = [&](const double* vv, double we) -> double {
    if constexpr (MODE != 0) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < K; ++i) acc += vv[i] * shh[i];
      we -= acc;
    }
    if constexpr (MODE == 2) {
      s[0] += we * we;
    } else {
#pragma unroll
      for (int i = 0; i < K; ++i) s[i] += vv[i] * we;
    }
    return we;
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // two elements per iteration, their loads issued before the arithmetic; the products are added in
  // element order, as one element per iteration would
  for (; e + stride < n; e += 2 * stride) {
    double v0[KA], v1[KA];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      v0[i] = V[(long long)i * n + e];
      v1[i] = V[(long long)i * n + e + stride];
    }
    const double w0 = w[e], w1 = w[e + stride];
    const double u0 = element(v0, w0);
    const double u1 = element(v1, w1);
    if constexpr (MODE != 0) {
      w[e] = u0;
      w[e + stride] = u1;
    }
  }
  if (e < n) {
    double v0[KA];
#pragma unroll
    for (int i = 0; i < K; ++i) v0[i] = V[(long long)i * n + e];
    const double u0 = element(v0, w[e]);
    if constexpr (MODE != 0) w[e] = u0;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const double v = warp_sum(s[i]);
    if (lane == 0) sh[i][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < NW; ++q) t += sh[threadIdx.x][q];
    part[(long long)threadIdx.x * gridDim.x + blockIdx.x] = t;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = wid; i < NS; i += NW) {
    double t = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(part + (long long)i * gridDim.x + b);
    t = warp_sum(t);
    if (lane == 0) {
      if constexpr (MODE == 2) {
        out[0] = t;
        out[1] = 0.0;
        out[2] = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
      } else {
        out[i] = t;
      }
    }
  }
  if (threadIdx.x == 0) *cnt = 0u;
}

static unsigned cgs_grid(long long n) {
  long long g = (n + BLK - 1) / BLK;
  if (g > CGS_GRID) g = CGS_GRID;
  if (g < 1) g = 1;
  return (unsigned)g;
}

template <int K>
static cudaError_t cgs_passes(long long n, const double* V, double* w, double* part, double* h1, double* h2,
                              double* nrm, unsigned* cnt, cudaStream_t s) {
  const unsigned g = cgs_grid(n);
  count_launch(); k_cgs_pass<K, 0><<<g, BLK, 0, s>>>(n, V, nullptr, w, part, h1, cnt);
  count_launch(); k_cgs_pass<K, 1><<<g, BLK, 0, s>>>(n, V, h1, w, part, h2, cnt);
  count_launch(); k_cgs_pass<K, 2><<<g, BLK, 0, s>>>(n, V, h2, w, part, nrm, cnt);
  return cudaGetLastError();
}

cudaError_t launch_cgs2(long long n, int k, const double* V, double* w, double* part, double* h1, double* h2,
                        double* nrm, unsigned* cnt, cudaStream_t s) {
  switch (k) {
#define PFF_CASE(K) \
  case K: return cgs_passes<K>(n, V, w, part, h1, h2, nrm, cnt, s);
    PFF_CASE(1) PFF_CASE(2) PFF_CASE(3) PFF_CASE(4) PFF_CASE(5) PFF_CASE(6) PFF_CASE(7) PFF_CASE(8)
    PFF_CASE(9) PFF_CASE(10) PFF_CASE(11) PFF_CASE(12) PFF_CASE(13) PFF_CASE(14) PFF_CASE(15) PFF_CASE(16)
#undef PFF_CASE
    default: break;
  }
  static_assert(CGS_KMAX == 16, "one instantiation per basis size up to CGS_KMAX");
  // larger bases: the separate multi-dot and update passes, then the norm pass with no basis vector
  cudaError_t e = launch_mdot(n, k, V, w, part, h1, s);
  if (e == cudaSuccess) e = launch_maxpy(n, k, V, h1, w, s);
  if (e == cudaSuccess) e = launch_mdot(n, k, V, w, part, h2, s);
  if (e == cudaSuccess) e = launch_maxpy(n, k, V, h2, w, s);
  if (e != cudaSuccess) return e;
  count_launch(); k_cgs_pass<0, 2><<<cgs_grid(n), BLK, 0, s>>>(n, V, h2, w, part, nrm, cnt);
  return cudaGetLastError();
}

// ===========================================================================================
// Chebyshev-Jacobi step on the two diagonal blocks (Sec. 3.3), interval [lo, hi] * lambda_max.
template <typename Real>
__global__ void k_cheb(int step, long long n, long long nu, const Real* __restrict__ f, const Real* __restrict__ Ax,
                       const Real* __restrict__ dinv, Real* __restrict__ d, Real* __restrict__ x,
                       const Real* __restrict__ inv_lam, double c0s, double c1, double c2s) {
  pdl_wait();
  // step 0: d = dinv f / theta_b, 1 / theta_b = c0s / lambda_b; step k: d = c1 d + (c2s / lambda_b) dinv (f - Ax)
  const Real i0 = inv_lam[0], i1 = inv_lam[1];
  const Real a0 = Real(step == 0 ? c0s : c2s) * i0, a1 = Real(step == 0 ? c0s : c2s) * i1;
  const Real cc = Real(c1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const Real a = e < nu ? a0 : a1;
    if (step == 0) {
      const Real de = a * (dinv[e] * f[e]);
      d[e] = de;
      x[e] = de;
    } else {
      const Real de = cc * d[e] + a * (dinv[e] * (f[e] - Ax[e]));
      d[e] = de;
      x[e] += de;
    }
  }
}

template <typename Real>
cudaError_t launch_cheb(int step, long long n, long long nu, const Real* f, const Real* Ax, const Real* dinv, Real* d,
                        Real* x, const Real* inv_lam, double c0s, double c1, double c2s, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return launch_k(k_cheb<Real>, dim3((unsigned)g), dim3(BLK), 0, s, step, n, nu, f, Ax, dinv, d, x, inv_lam, c0s, c1,
                  c2s);
}
template cudaError_t launch_cheb<double>(int, long long, long long, const double*, const double*, const double*,
                                         double*, double*, const double*, double, double, double, cudaStream_t);
template cudaError_t launch_cheb<float>(int, long long, long long, const float*, const float*, const float*, float*,
                                        float*, const float*, double, double, double, cudaStream_t);

// ---- CG-Lanczos -------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// CG-Lanczos kernels. Each one also reduces a pair of block dot products: every CTA writes its
// partial sums, and the CTA that finishes last (counted on *cnt) adds the partials in a fixed order
// and performs the scalar step, so one iteration takes the apply and three kernels.
// scal: [rz0 rz1 pAp0 pAp1 alpha0 alpha1 beta0 beta1 rzn0 rzn1 dead0 dead1 | counter]

__device__ __forceinline__ bool cg_reduce_last(double s0, double s1, double* __restrict__ part, unsigned* cnt,
                                               double& r0, double& r1) {
  __shared__ double sh[32];
  __shared__ int last;
  r0 = block_sum(s0, sh);
  r1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r0;
    part[2 * blockIdx.x + 1] = r1;
    __threadfence();
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double t0 = 0.0, t1 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    t0 += __ldcg(part + 2 * b);
    t1 += __ldcg(part + 2 * b + 1);
  }
  r0 = block_sum(t0, sh);
  r1 = block_sum(t1, sh);
  if (threadIdx.x == 0) *cnt = 0u;
  return true;  // sums valid in thread 0
}

template <typename Real>
__global__ void __launch_bounds__(BLK) k_cg_init(long long n, long long nu, unsigned long long seed,
                                                 const unsigned char* __restrict__ flags, long long nn,
                                                 const Real* __restrict__ dinv, Real* __restrict__ r,
                                                 Real* __restrict__ z, Real* __restrict__ pv, double* __restrict__ part,
                                                 double* __restrict__ scal) {
  double s0 = 0.0, s1 = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int f = int(e / nn);
    const bool masked = (flags[e % nn] >> f) & 1u;
    const double v = masked ? 0.0 : (double)(splitmix64(seed, (uint64_t)e) >> 11) * 0x1.0p-53 - 0.5;
    r[e] = Real(v);
    const Real zz = dinv[e] * Real(v);
    z[e] = zz;
    pv[e] = zz;
    const double q = (double)Real(v) * (double)zz;
    if (e < nu) s0 += q;
    else s1 += q;
  }
  double r0, r1;
  if (cg_reduce_last(s0, s1, part, reinterpret_cast<unsigned*>(scal + 12), r0, r1) && threadIdx.x == 0) {
    scal[0] = r0;
    scal[1] = r1;
  }
}

// <p, Ap> of both blocks, then alpha = rz / pAp (a block whose recurrence broke down stays dead).
template <typename Real>
__global__ void __launch_bounds__(BLK) k_cg_pap(long long n, long long nu, const Real* __restrict__ pv,
                                                const Real* __restrict__ Ap, double* __restrict__ part,
                                                double* __restrict__ scal, double* __restrict__ ah, int it,
                                                int iters) {
  double s0 = 0.0, s1 = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = (double)pv[e] * (double)Ap[e];
    if (e < nu) s0 += v;
    else s1 += v;
  }
  double r0, r1;
  if (cg_reduce_last(s0, s1, part, reinterpret_cast<unsigned*>(scal + 12), r0, r1) && threadIdx.x == 0)
    cg_take_alpha(scal, ah, it, iters, r0, r1);
}

// r -= alpha Ap, z = D^{-1} r, Ap = 0 (the next apply accumulates into it), <r, z>, then
// beta = rz_new / rz and rz = rz_new.
template <typename Real>
__global__ void __launch_bounds__(BLK) k_cg_update(long long n, long long nu, Real* __restrict__ Ap,
                                                   const Real* __restrict__ dinv, double* __restrict__ scal,
                                                   Real* __restrict__ r, Real* __restrict__ z, double* __restrict__ part,
                                                   double* __restrict__ bh, int it, int iters) {
  const Real a0 = Real(scal[4]), a1 = Real(scal[5]);
  double s0 = 0.0, s1 = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // four elements per iteration, all loads first (the stores below would otherwise hold back the next
  // element's loads); the products are added in element order, as one element per iteration would
  for (; e + 3 * stride < n; e += 4 * stride) {
    Real rv[4], av[4], dv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      rv[u] = r[e + u * stride];
      av[u] = Ap[e + u * stride];
      dv[u] = dinv[e + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = e + u * stride;
      const Real rr = rv[u] - (i < nu ? a0 : a1) * av[u];
      r[i] = rr;
      const Real zz = dv[u] * rr;
      z[i] = zz;
      Ap[i] = Real(0);
      const double q = (double)rr * (double)zz;
      if (i < nu) s0 += q;
      else s1 += q;
    }
  }
  for (; e < n; e += stride) {
    const Real al = e < nu ? a0 : a1;
    const Real rr = r[e] - al * Ap[e];
    r[e] = rr;
    const Real zz = dinv[e] * rr;
    z[e] = zz;
    Ap[e] = Real(0);
    const double q = (double)rr * (double)zz;
    if (e < nu) s0 += q;
    else s1 += q;
  }
  double r0, r1;
  if (cg_reduce_last(s0, s1, part, reinterpret_cast<unsigned*>(scal + 12), r0, r1) && threadIdx.x == 0) {
    scal[8] = r0;
    scal[9] = r1;
    for (int b = 0; b < 2; ++b) {
      const double rzn = scal[8 + b], rz = scal[b];
      double be = 0.0;
      if (scal[10 + b] == 0.0) {
        be = rzn / rz;
        if (!(rzn > 0.0)) scal[10 + b] = 1.0;
      }
      scal[6 + b] = be;
      bh[b * iters + it] = be;
      scal[b] = rzn;
    }
  }
}

template <typename Real>
__global__ void k_cg_pupdate(long long n, long long nu, const Real* __restrict__ z, const double* __restrict__ scal,
                             Real* __restrict__ pv) {
  const Real b0 = Real(scal[6]), b1 = Real(scal[7]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    pv[e] = z[e] + (e < nu ? b0 : b1) * pv[e];
}

template <typename Real>
cudaError_t launch_cg_init(long long n, long long nu, unsigned long long seed, const unsigned char* flags,
                           long long nn, const Real* dinv, Real* r, Real* z, Real* pv, double* part, double* scal,
                           cudaStream_t s) {
  count_launch(); k_cg_init<Real><<<red_grid(n), BLK, 0, s>>>(n, nu, seed, flags, nn, dinv, r, z, pv, part, scal);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_cg_pap(long long n, long long nu, const Real* pv, const Real* Ap, double* part, double* scal,
                          double* alpha_hist, int it, int iters, cudaStream_t s) {
  count_launch(); k_cg_pap<Real><<<red_grid(n), BLK, 0, s>>>(n, nu, pv, Ap, part, scal, alpha_hist, it, iters);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_cg_update(long long n, long long nu, Real* Ap, const Real* dinv, double* scal, Real* r, Real* z,
                             double* part, double* beta_hist, int it, int iters, cudaStream_t s) {
  count_launch();
  k_cg_update<Real><<<red_grid(n), BLK, 0, s>>>(n, nu, Ap, dinv, scal, r, z, part, beta_hist, it, iters);
  return cudaGetLastError();
}
template <typename Real>
cudaError_t launch_cg_pupdate(long long n, long long nu, const Real* z, const double* scal, Real* pv, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  count_launch(); k_cg_pupdate<Real><<<(unsigned)g, BLK, 0, s>>>(n, nu, z, scal, pv);
  return cudaGetLastError();
}
#define PFF_INST_CG(R)                                                                                           \
  template cudaError_t launch_cg_init<R>(long long, long long, unsigned long long, const unsigned char*,         \
                                         long long, const R*, R*, R*, R*, double*, double*, cudaStream_t);      \
  template cudaError_t launch_cg_pap<R>(long long, long long, const R*, const R*, double*, double*, double*, int, \
                                        int, cudaStream_t);                                                     \
  template cudaError_t launch_cg_update<R>(long long, long long, R*, const R*, double*, R*, R*, double*, double*, \
                                           int, int, cudaStream_t);                                             \
  template cudaError_t launch_cg_pupdate<R>(long long, long long, const R*, const double*, R*, cudaStream_t);
PFF_INST_CG(double)
PFF_INST_CG(float)
#undef PFF_INST_CG

// lambda_max of the Lanczos tridiagonal by multisection with Sturm counts. The counts run in
// double-word arithmetic on the FP32 pipe (a full warp of FP64 divisions costs tens of times more
// on this GPU): the matrix is first scaled by a power of two so that its Gershgorin interval lies
// in [-1, 1], which keeps every quantity far inside the FP32 exponent range; the pivots d_j carry
// about 44 significant bits, so the bracket still closes to about 1e-13 relative.
__device__ __forceinline__ df64 df_div(df64 x, df64 y) {
  const float th = __fdiv_rn(x.hi, y.hi);
  float ph, pl;
  ph = __fmul_rn(y.hi, th);
  pl = __fmaf_rn(y.hi, th, -ph);
  pl = __fmaf_rn(y.lo, th, pl);
  const df64 r = x - df_make(ph, pl);
  const float tl = __fdiv_rn(r.hi, y.hi);
  float zh, zl;
  fast_two_sum(th, tl, zh, zl);
  return df_make(zh, zl);
}
// Number of eigenvalues below x of the tridiagonal (a, b2 = squared off-diagonals), all scaled.
__device__ int sturm_count_df(int k, const df64* a, const df64* b2, df64 x) {
  int cnt = 0;
  df64 d = a[0] - x;
  if (d.hi < 0.f) ++cnt;
  for (int j = 1; j < k; ++j) {
    if (fabsf(d.hi) < 1e-30f) d = df_make(d.hi < 0.f ? -1e-30f : 1e-30f, 0.f);  // keeps b2 / d finite
    d = (a[j] - x) - df_div(b2[j - 1], d);
    if (d.hi < 0.f) ++cnt;
  }
  return cnt;
}
// One warp per block b: the tridiagonal of the first k valid CG steps of block b, then
// multisection (each lane evaluates a Sturm count; the bracket shrinks 33-fold a round).
__global__ void k_tridiag_eig(int iters, const double* __restrict__ ah, const double* __restrict__ bh,
                              double* __restrict__ lam) {
  const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (b >= 2) return;
  __shared__ double sa[2][64], sb2[2][64];
  __shared__ df64 da[2][64], db2[2][64];
  __shared__ int sk[2];
  if (lane == 0) {
    int k = 0;
    while (k < iters && k < 64 && ah[b * iters + k] > 0.0) ++k;
    for (int j = 0; j < k; ++j) {
      const double al = ah[b * iters + j];
      sa[b][j] = 1.0 / al + (j > 0 ? bh[b * iters + j - 1] / ah[b * iters + j - 1] : 0.0);
      if (j + 1 < k) {
        const double off = sqrt(bh[b * iters + j]) / al;
        sb2[b][j] = off * off;
      }
    }
    sk[b] = k;
  }
  __syncwarp();
  const int k = sk[b];
  if (k == 0) {
    if (lane == 0) {
      lam[b] = 1.0;
      lam[2 + b] = 1.0;
      lam[4 + b] = 1.0;
      reinterpret_cast<float*>(lam + 6)[b] = 1.0f;
    }
    return;
  }
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < k; ++j) {
    double r = 0.0;
    if (j > 0) r += sqrt(sb2[b][j - 1]);
    if (j + 1 < k) r += sqrt(sb2[b][j]);
    lo = fmin(lo, sa[b][j] - r);
    hi = fmax(hi, sa[b][j] + r);
  }
  // power-of-two scale s with max(|lo|, |hi|) * s in (0.5, 1]
  int ex;
  frexp(fmax(fabs(lo), fabs(hi)), &ex);
  const double sc = ldexp(1.0, -ex);
  for (int j = lane; j < k; j += 32) {
    da[b][j] = df_from(sa[b][j] * sc);
    if (j + 1 < k) db2[b][j] = df_from(sb2[b][j] * sc * sc);
  }
  __syncwarp();
  // largest eigenvalue: the first point x with count(x) >= k
  double l = lo * sc, h = hi * sc;
  for (int round = 0; round < 12 && h - l > 1e-15 * fmax(fabs(l), fabs(h)); ++round) {
    const double x = l + (h - l) * (lane + 1) / 33.0;
    const unsigned ge = __ballot_sync(0xffffffffu, sturm_count_df(k, da[b], db2[b], df_from(x)) >= k);
    const int j = ge ? __ffs(ge) - 1 : 32;  // first lane whose point is at or above the eigenvalue
    const double nl = j == 0 ? l : l + (h - l) * j / 33.0;
    const double nh = j == 32 ? h : l + (h - l) * (j + 1) / 33.0;
    l = nl;
    h = nh;
  }
  if (lane == 0) {
    const double lm = h / sc;
    lam[b] = lm;
    lam[2 + b] = lo;  // Gershgorin lower bound
    // 1 / lambda_max for the smoother kernels (FP64 and FP32 copies); 0 disables the block's update
    const double il = (lm > 0.0 && lm < 1e300) ? 1.0 / lm : 0.0;
    lam[4 + b] = il;
    reinterpret_cast<float*>(lam + 6)[b] = (float)il;
  }
}
cudaError_t launch_tridiag_eig(int iters, const double* alpha_hist, const double* beta_hist, double* lam,
                               cudaStream_t s) {
  count_launch(); k_tridiag_eig<<<1, 64, 0, s>>>(iters, alpha_hist, beta_hist, lam);
  return cudaGetLastError();
}

__global__ void k_inv_diag(long long n, const double* __restrict__ d, double* __restrict__ di64,
                           float* __restrict__ di32) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[e];
    di64[e] = v;
    if (di32) di32[e] = (float)v;
  }
}
__global__ void k_inv_diag32(long long n, const float* __restrict__ d, float* __restrict__ di32) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    di32[e] = 1.0f / d[e];
}
cudaError_t launch_inv_diag32(long long n, const float* d, float* di32, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  count_launch(); k_inv_diag32<<<(unsigned)g, BLK, 0, s>>>(n, d, di32);
  return cudaGetLastError();
}
cudaError_t launch_inv_diag(long long n, const double* d, double* di64, float* di32, cudaStream_t s) {
  long long g = (n + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  count_launch(); k_inv_diag<<<(unsigned)g, BLK, 0, s>>>(n, d, di64, di32);
  return cudaGetLastError();
}

// ===========================================================================================
// Newton step helpers.
__global__ void k_active_set(int dim, long long nn, const double* __restrict__ R, const double* __restrict__ mass,
                             const double* __restrict__ phi_old, double c, double* __restrict__ U,
                             unsigned char* __restrict__ flags, int* __restrict__ cnt) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  bool act = false, chg = false;
  if (i < nn) {
    const double phi = U[dim * nn + i];
    const double crit = -R[dim * nn + i] / mass[i] + c * (phi - phi_old[i]);
    act = crit > 0.0;
    const unsigned char bit = (unsigned char)(1u << dim);
    const unsigned char fl = flags[i];
    chg = act != ((fl & bit) != 0);
    flags[i] = act ? (unsigned char)(fl | bit) : (unsigned char)(fl & ~bit);
    if (act) U[dim * nn + i] = phi_old[i];
  }
  const unsigned ba = __ballot_sync(0xffffffffu, act), bc = __ballot_sync(0xffffffffu, chg);
  if ((threadIdx.x & 31) == 0) {
    if (ba) atomicAdd(cnt, __popc(ba));
    if (bc) atomicAdd(cnt + 1, __popc(bc));
  }
}
cudaError_t launch_active_set(int dim, long long nn, const double* R, const double* mass, const double* phi_old,
                              double c, double* U, unsigned char* flags, int* cnt, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  count_launch(); k_active_set<<<grid_for(nn), BLK, 0, s>>>(dim, nn, R, mass, phi_old, c, U, flags, cnt);
  return cudaGetLastError();
}

__global__ void k_newton_rhs(int dim, long long nn, const double* __restrict__ R,
                             const unsigned char* __restrict__ flags, double* __restrict__ rhs) {
  const long long n = (dim + 1) * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int f = int(e / nn);
    rhs[e] = ((flags[e % nn] >> f) & 1u) ? 0.0 : -R[e];
  }
}
cudaError_t launch_newton_rhs(int dim, long long nn, const double* R, const unsigned char* flags, double* rhs,
                              cudaStream_t s) {
  long long g = ((dim + 1) * nn + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  count_launch(); k_newton_rhs<<<(unsigned)g, BLK, 0, s>>>(dim, nn, R, flags, rhs);
  return cudaGetLastError();
}

__global__ void k_masked_copy(int dim, long long nn, double scale, const double* __restrict__ x,
                              const unsigned char* __restrict__ flags, unsigned bits, double* __restrict__ out) {
  const long long n = (dim + 1) * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int f = int(e / nn);
    out[e] = (((flags[e % nn] & bits) >> f) & 1u) ? 0.0 : scale * x[e];
  }
}
cudaError_t launch_masked_copy(int dim, long long nn, double scale, const double* x, const unsigned char* flags,
                               unsigned bits, double* out, cudaStream_t s) {
  long long g = ((dim + 1) * nn + BLK - 1) / BLK;
  if (g > 152 * 16) g = 152 * 16;
  count_launch(); k_masked_copy<<<(unsigned)g, BLK, 0, s>>>(dim, nn, scale, x, flags, bits, out);
  return cudaGetLastError();
}

__global__ void k_set_active(int dim, long long nn, const unsigned char* __restrict__ a, unsigned char* __restrict__ fl) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const unsigned char bit = (unsigned char)(1u << dim);
  fl[i] = a[i] ? (unsigned char)(fl[i] | bit) : (unsigned char)(fl[i] & ~bit);
}
cudaError_t launch_set_active(int dim, long long nn, const unsigned char* active, unsigned char* flags,
                              cudaStream_t s) {
  count_launch(); k_set_active<<<grid_for(nn), BLK, 0, s>>>(dim, nn, active, flags);
  return cudaGetLastError();
}
__global__ void k_get_active(int dim, long long nn, const unsigned char* __restrict__ fl, unsigned char* __restrict__ a) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  a[i] = (fl[i] >> dim) & 1u;
}
cudaError_t launch_get_active(int dim, long long nn, const unsigned char* flags, unsigned char* active,
                              cudaStream_t s) {
  count_launch(); k_get_active<<<grid_for(nn), BLK, 0, s>>>(dim, nn, flags, active);
  return cudaGetLastError();
}

// Load stepping: u_comp := load on top-face nodes (comp = dim - 1: tension test; 0: shear test).
__global__ void k_lift_top(int comp, long long nn, const unsigned char* __restrict__ flags, double load,
                           double* __restrict__ U) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  if (flags[i] & 0x10u) U[comp * nn + i] = load;
}
// phi~ = clamp(2 h1 - h2, 0, 1) (or h1 when h2 is null); phi_old = h1.
__global__ void k_extrapolate(long long nn, const double* __restrict__ h1, const double* __restrict__ h2,
                              double* __restrict__ phit, double* __restrict__ phi_old) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double a = h1[i];
  double t = h2 ? 2.0 * a - h2[i] : a;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  phit[i] = t;
  phi_old[i] = a;
}
cudaError_t launch_load_step_prep(int comp, long long nn, const unsigned char* flags, double load, double* U,
                                  const double* h1, const double* h2, double* phit, double* phi_old, cudaStream_t s) {
  count_launch(); k_lift_top<<<grid_for(nn), BLK, 0, s>>>(comp, nn, flags, load, U);
  count_launch(); k_extrapolate<<<grid_for(nn), BLK, 0, s>>>(nn, h1, h2, phit, phi_old);
  return cudaGetLastError();
}

__global__ void k_lumped_mass(int dim, long long nn, int n1, const double* __restrict__ w1, double* __restrict__ m) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  long long rem = i;
  double v = 1.0;
  for (int t = 0; t < dim; ++t) {
    v *= w1[rem % n1];
    rem /= n1;
  }
  m[i] = v;
}
cudaError_t launch_lumped_mass(int dim, long long nn, int n1, const double* w1, double* mass, cudaStream_t s) {
  count_launch(); k_lumped_mass<<<grid_for(nn), BLK, 0, s>>>(dim, nn, n1, w1, mass);
  return cudaGetLastError();
}

}  // namespace pff
