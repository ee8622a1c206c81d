// pff_common.cuh -- shared device definitions of the phase-field fracture library.
//
// Tables of the 1D Q_p basis at the Gauss points, the tile geometry of the cell-batched
// operator kernels, the Mandel (orthonormal Voigt) representation of symmetric tensors, and
// the pointwise constitutive laws of Sec. 2.1 (degradation g, Miehe split) and of the
// eigen-derivative of Sec. 3.5 used by the tangent.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pff {

constexpr int MAXP = 4;
constexpr int MAXN = MAXP + 1;

// Masking of inputs/outputs of the cell operator kernels.
enum InMask { IN_RAW = 0, IN_ALL = 1, IN_DIRICHLET = 2 };
enum OutMask { OUT_RAW = 0, OUT_IDENTITY = 1, OUT_ZERO_DIRICHLET = 2 };
enum JacMode { JM_FULL = 0, JM_BLOCKDIAG = 1, JM_TRANSPOSE = 2 };

// 1D tables on the unit interval: S[q][k] = l_k(x_q), D[q][k] = l_k'(x_q) / h at the Gauss
// points x_q of the level, W[q] Gauss weights; JxW(q) = hd * prod_t W[q_t].
template <typename Real>
struct Tab {
  Real S[MAXN][MAXN];
  Real D[MAXN][MAXN];
  Real W[MAXN];
  Real hd;
};

// Tile shapes (cells per CTA) of the operator kernels, per dimension and degree.
template <int DIM, int P>
struct TileCfg;
template <> struct TileCfg<2, 1> { static constexpr int TX = 8, TY = 16, TZ = 1; };
template <> struct TileCfg<2, 2> { static constexpr int TX = 8, TY = 8, TZ = 1; };
template <> struct TileCfg<2, 3> { static constexpr int TX = 8, TY = 4, TZ = 1; };
template <> struct TileCfg<2, 4> { static constexpr int TX = 8, TY = 4, TZ = 1; };
template <> struct TileCfg<3, 1> { static constexpr int TX = 4, TY = 4, TZ = 2; };
template <> struct TileCfg<3, 2> { static constexpr int TX = 4, TY = 2, TZ = 2; };
template <> struct TileCfg<3, 3> { static constexpr int TX = 2, TY = 2, TZ = 2; };
template <> struct TileCfg<3, 4> { static constexpr int TX = 2, TY = 2, TZ = 1; };

// Programmatic dependent launch: a kernel launched with launch_k (below) may be scheduled while its
// predecessor in the stream is still running; it must call pdl_wait() before its first access to
// global memory, which returns once the predecessor grid has completed and its writes are visible.
// Without a programmatic predecessor the wait returns at once. No kernel triggers its dependents
// early (griddepcontrol.launch_dependents): at the start of every kernel that made the 2D Q2 256^2
// V-cycle slower (0.97 vs 0.80 ms), the waiting dependents taking SM slots from the running grid.
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// Host-side lookup of TileCfg.
template <int DIM, int P>
inline void tile_shape_of(int* t) {
  t[0] = TileCfg<DIM, P>::TX;
  t[1] = TileCfg<DIM, P>::TY;
  t[2] = TileCfg<DIM, P>::TZ;
}
inline void tile_shape(int dim, int p, int* t) {
  switch (dim * 10 + p) {
    case 21: tile_shape_of<2, 1>(t); break;
    case 22: tile_shape_of<2, 2>(t); break;
    case 23: tile_shape_of<2, 3>(t); break;
    case 24: tile_shape_of<2, 4>(t); break;
    case 31: tile_shape_of<3, 1>(t); break;
    case 32: tile_shape_of<3, 2>(t); break;
    case 33: tile_shape_of<3, 3>(t); break;
    default: tile_shape_of<3, 4>(t); break;
  }
}

// Geometry of one level as the kernels see it.
struct Geom {
  int dim, p, N, n1;
  long long nn;            // nodes (grid nodes and, with a cut slit, their copies)
  int tdim[3];             // cells per tile in x, y, z
  int ntile[3];            // tiles per direction
  int qpx, qpy, qpz;       // quadrature points of a tile per direction
  long long qpt;           // quadrature points per tile
  long long ntiles;
  // Slit cut into the mesh (Sec. 5.1): the nodes on the slit (last coordinate 1/2, x < 1/2; the tip
  // stays shared) get a second copy, numbered after the grid nodes, which the cells below the slit use.
  // The slit lies on a boundary between tile rows (tiles along the last axis).
  int cut;                 // 1: slit cut into the mesh, 0: one node per grid point
  int cut_row;             // grid index of the slit along the last axis (p N / 2)
  int cut_x;               // copied slit nodes have x index < cut_x (= p N / 2)
  int cut_tile;            // tile index along the last axis of the tiles just below the slit
  long long ngrid;         // grid nodes
};

// Material constants of the recomputed FP32 Jacobian (pw_jac_rc2).
struct MatConst32 {
  float lam, mu, gc_eps, gc_over_eps, omk, kappa;  // omk = 1 - kappa
};

// Copy of slit node (gx, gy) (gy: y index in 3D, 0 in 2D), numbered x fastest after the grid nodes.
__host__ __device__ __forceinline__ long long cut_copy(const Geom& g, int gx, int gy) {
  return g.ngrid + gx + (long long)g.cut_x * gy;
}
// Whether patch layer rl (along the last axis, npl layers) of tile layer tl at x index gx is the slit
// seen from below (those nodes are the copies) or from above (the grid nodes, not shared with the tiles
// below).
__host__ __device__ __forceinline__ bool cut_below(const Geom& g, int tl, int rl, int npl, int gx) {
  return g.cut && tl == g.cut_tile && rl == npl - 1 && gx < g.cut_x;
}
__host__ __device__ __forceinline__ bool cut_above(const Geom& g, int tl, int rl, int gx) {
  return g.cut && tl == g.cut_tile + 1 && rl == 0 && gx < g.cut_x;
}

// Chebyshev-Jacobi step fused into the block-diagonal apply (Sec. 3.3 smoother): for a node that
// only this tile touches, y = (G x)_i is final in registers, so the update
//   d_i <- c1 d_i + (2 rho_k / delta_b) dinv_i (f_i - y_i),   x_i <- x_i + d_i
// is done in place and y_i is never stored; seam nodes go through y and k_cheb_seam afterwards.
// With delta_b = (hi - lo) lambda_b / 2 the coefficient is c2s / lambda_b, c2s = 4 rho_k / (hi - lo)
// from the host and 1 / lambda_b from the device (inv_lam, 0 for an unusable estimate): no division
// (and, for FP32, no FP64 arithmetic) in the kernels.
// acc (last step of a post-smoothing): acc_i += x_i + d_i instead of x_i += d_i, so the correction is
// added to the cycle's iterate without a separate kernel.
template <typename Store>
struct ChebEpi {
  const Store* f;
  const Store* dinv;
  Store* d;
  Store* x;
  const Store* inv_lam;  // [2]: 1 / lambda_max of the u block and of the phi block
  double c1, c2s;
  Store* acc;
  int on;
  // Iterate and direction in two buffers each, seam sums in three (no seam launch between steps):
  // step k reads x_k from x and d_{k-1} from d and writes x_{k+1} to x_out and d_k to d_out on the nodes
  // of a single tile. With pp = 1 it first finishes step k-1 on the seam nodes of its patch, whose
  // y_{k-1} is complete in tp: d_{k-1} = c1p d_{k-2} + c2p dinv (f - y_{k-1}) with d_{k-2} in d_out, and
  // x_k = x_{k-1} + d_{k-1} with x_{k-1} in x_out; the tile that owns the node writes d_{k-1} to d and
  // x_k to x, and zeroes tz there (the seam sums of step k-2, which no one reads any more).
  // x_out = d_out = null: the single-buffer scheme, in place, seams by launch_cheb_seam.
  Store* x_out;
  Store* d_out;
  const Store* tp;
  Store* tz;
  double c1p, c2sp;
  int pp;
};

// One CG-Lanczos step (lambda_max estimate) folded into the block-diagonal 2D apply: the apply's input
// is p = z + beta p_old (beta per block from scal[6..7], 0 at the first step), built while the tile is
// staged (the apply's src is z); the tile that owns a node writes p there to p_out. Each tile adds p_i
// times its own contribution to (A p)_i over its nodes, per block: over all tiles that is <p, A p>, seam
// nodes included. The last CTA to finish adds the per-CTA partials in a fixed order and takes alpha
// (cg_take_alpha), which the update kernel then reads.
template <typename Store>
struct CgEpi {
  int on;
  const Store* p_old;
  Store* p_out;
  double* scal;  // CG-Lanczos scalars: rz, pAp, alpha, beta, rz_new, dead flags (2 each), counter at [12]
  double* part;  // per-CTA partial sums, 2 per CTA
  double* ah;    // alpha history
  int it, iters;
};

// alpha = rz / <p, A p> per block from the reduced <p, A p> (r0, r1); a block whose recurrence broke
// down stays dead (alpha 0).
__device__ __forceinline__ void cg_take_alpha(double* scal, double* ah, int it, int iters, double r0, double r1) {
  scal[2] = r0;
  scal[3] = r1;
  for (int b = 0; b < 2; ++b) {
    const double rz = scal[b], pAp = scal[2 + b];
    double al = 0.0;
    if (scal[10 + b] == 0.0 && pAp > 0.0 && rz > 0.0 && pAp < 1e300) al = rz / pAp;
    else scal[10 + b] = 1.0;
    scal[4 + b] = al;
    ah[b * iters + it] = al;
  }
}

// First Chebyshev step with zero initial guess, x = d = (c0s / lambda_b) dinv f, done by the kernel
// that produces f (the restriction, the V-cycle's residual update). nu: first phase-field DoF.
template <typename Real>
struct ChebStart {
  Real* d;
  Real* x;
  const Real* dinv;
  const Real* inv_lam;
  double c0s;
  long long nu;
  int on;
};

// ---------------------------------------------------------------------------------------------
// Mandel representation: a symmetric d x d tensor as an orthonormal vector of NM components,
// 2D (11, 22, 12), 3D (11, 22, 33, 23, 13, 12), shear components scaled by sqrt(2).
template <int DIM> struct Mandel;
template <> struct Mandel<2> {
  static constexpr int NM = 3;
  __host__ __device__ static constexpr int ia(int m) { return m == 0 ? 0 : (m == 1 ? 1 : 0); }
  __host__ __device__ static constexpr int ib(int m) { return m == 0 ? 0 : 1; }
};
template <> struct Mandel<3> {
  static constexpr int NM = 6;
  __host__ __device__ static constexpr int ia(int m) { return m < 3 ? m : (m == 3 ? 1 : 0); }
  __host__ __device__ static constexpr int ib(int m) { return m < 3 ? m : (m == 5 ? 1 : 2); }
};
__host__ __device__ constexpr int sym_index(int nm, int i, int j) { return i * nm - i * (i - 1) / 2 + (j - i); }

// Number of stored per-quadrature-point values of the Jacobian (all multiplied by JxW):
//   split none : g(phi~) lambda, g(phi~) mu, b (NM), c, k
//   split miehe: C (NM(NM+1)/2 upper triangle), b (NM), c, k
// with b = g'(phi) sigma^+ (Mandel), c = g''(phi) E_s^+ + G_c / eps, k = G_c eps.
__host__ __device__ constexpr int qp_nv(int dim, int split) {
  return split == 0 ? (2 + (dim == 2 ? 3 : 6) + 2)
                    : ((dim == 2 ? 6 : 21) + (dim == 2 ? 3 : 6) + 2);
}
constexpr int ST_NV = 4;  // per-point state for the residual: g(phi~), G_c, lambda, mu

// ---------------------------------------------------------------------------------------------
// Degradation (Sec. 2.1): g = (1 - kappa) phi^2 + kappa.
__host__ __device__ inline double deg_g(double phi, double kappa) { return (1.0 - kappa) * phi * phi + kappa; }
__host__ __device__ inline double deg_dg(double phi, double kappa) { return 2.0 * (1.0 - kappa) * phi; }
__host__ __device__ inline double deg_ddg(double kappa) { return 2.0 * (1.0 - kappa); }
__host__ __device__ inline double heav(double x) { return x >= 0.0 ? 1.0 : 0.0; }
__host__ __device__ inline double pos(double x) { return x > 0.0 ? x : 0.0; }

// Divided difference of x -> max(x, 0) at (a, b); H(a) when a == b.
__device__ inline double theta_dd(double a, double b) {
  return a == b ? heav(a) : (pos(a) - pos(b)) / (a - b);
}

// Eigen-decomposition of a symmetric 2x2 [[a, b], [b, c]]: l[0] >= l[1], columns of V. The half gap r and
// 1 / r come from one reciprocal square root, and the half-angle cosine and sine from another (no FP64
// division or hypot: both are long sequences on the FP64 pipe). Strains are far from the FP64 limits
// where hypot's scaling matters; a pair with |(a - c) / 2, b| below ~1e-154 counts as degenerate.
__device__ inline void eig_sym2(double a, double b, double c, double l[2], double V[2][2]) {
  const double m = 0.5 * (a + c), dd = 0.5 * (a - c);
  const double r2 = fma(dd, dd, b * b);
  double r = 0.0, cs = 1.0, sn = 0.0;
  if (r2 > 0.0) {
    // half-angle of (cos 2t, sin 2t) = (dd, b) / r
    const double ir = rsqrt(r2);
    r = r2 * ir;
    const double c2 = dd * ir, s2 = b * ir;
    if (c2 >= 0.0) {
      const double y = 0.5 * (1.0 + c2), ry = rsqrt(y);  // cos t = sqrt(y), sin t = s2 / (2 cos t)
      cs = y * ry;
      sn = 0.5 * s2 * ry;
    } else {
      const double y = 0.5 * (1.0 - c2), ry = rsqrt(y);  // sin t = sign(s2) sqrt(y), cos t = s2 / (2 sin t)
      sn = s2 < 0.0 ? -(y * ry) : y * ry;
      cs = 0.5 * fabs(s2) * ry;
    }
  }
  l[0] = m + r;
  l[1] = m - r;
  V[0][0] = cs;  V[1][0] = sn;   // v1
  V[0][1] = -sn; V[1][1] = cs;   // v2
}

// Eigen-decomposition of a symmetric 3x3 by cyclic Jacobi rotations (A is overwritten).
// Columns of V are the eigenvectors, l the eigenvalues (unsorted).
__device__ inline void eig_sym3(double A[3][3], double l[3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 24; ++sweep) {
    const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off == 0.0 || off <= 1e-36 * dia) break;
    for (int pi = 0; pi < 3; ++pi) {
      const int p = pi == 2 ? 1 : 0;
      const int q = pi == 0 ? 1 : 2;
      const double apq = A[p][q];
      if (apq == 0.0) continue;
      const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
      double t;
      if (fabs(th) > 1e150) t = 0.5 / th;
      else t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      A[p][p] -= t * apq;
      A[q][q] += t * apq;
      A[p][q] = A[q][p] = 0.0;
      const int r = 3 - p - q;
      const double arp = A[r][p], arq = A[r][q];
      A[r][p] = A[p][r] = c * arp - s * arq;
      A[r][q] = A[q][r] = s * arp + c * arq;
      for (int k = 0; k < 3; ++k) {
        const double vp = V[k][p], vq = V[k][q];
        V[k][p] = c * vp - s * vq;
        V[k][q] = s * vp + c * vq;
      }
    }
  }
  l[0] = A[0][0];
  l[1] = A[1][1];
  l[2] = A[2][2];
}

// Eigen system of a symmetric strain given as a full d x d array.
template <int DIM>
__device__ inline void eig_sym(const double e[DIM][DIM], double l[DIM], double V[DIM][DIM]) {
  if constexpr (DIM == 2) {
    eig_sym2(e[0][0], 0.5 * (e[0][1] + e[1][0]), e[1][1], l, V);
  } else {
    double A[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[i][j] = 0.5 * (e[i][j] + e[j][i]);
    eig_sym3(A, l, V);
  }
}

// Eigenvalues (and the trace) of magnitude at most 1e-12 times the largest eigenvalue magnitude
// are set to exactly 0: their sign is rounding noise and must not flip H or the tangent.
template <int DIM>
__device__ inline void snap_zero(double l[DIM], double& tr) {
  double sc = 0.0;
  for (int t = 0; t < DIM; ++t) sc = fmax(sc, fabs(l[t]));
  const double tol = 1e-12 * sc;
  for (int t = 0; t < DIM; ++t)
    if (fabs(l[t]) <= tol) l[t] = 0.0;
  if (fabs(tr) <= tol) tr = 0.0;
}

// Mandel vector of (a b^T + b a^T)/2 scaled: E_ii for a == b, E_ij = (a b^T + b a^T)/sqrt2.
template <int DIM>
__device__ inline void mandel_dyad(const double* a, const double* b, bool same, double* out) {
  constexpr int NM = Mandel<DIM>::NM;
  const double S2 = 1.4142135623730951;
  for (int m = 0; m < NM; ++m) {
    const int i = Mandel<DIM>::ia(m), j = Mandel<DIM>::ib(m);
    if (same) {
      out[m] = (i == j) ? a[i] * a[i] : S2 * a[i] * a[j];
    } else {
      out[m] = (i == j) ? S2 * a[i] * b[i] : (a[i] * b[j] + a[j] * b[i]);
    }
  }
}

}  // namespace pff
