// pff_kernels.h -- host launchers of the non-operator kernels of libpff (internal).
#pragma once
#include <cuda_runtime.h>
#include "pff_common.cuh"
#include "pff_df64.cuh"

namespace pff {

struct MatConst {
  double lambda, mu, gc, eps, kappa;
};

// Per-point data of the Jacobian (FP64, optional FP32 and double-word copies) and of the residual.
// part: QP_ALL; or, with the Miehe split, QP_STRAIN (everything that depends on u only, plus
// sigma+ and E_s+ into sp64 [tile][NM + 1][qpt]) followed by QP_PHASE (the coupling entries from
// sp64 and phi).
constexpr int QP_ALL = 0, QP_STRAIN = 1, QP_PHASE = 2;
cudaError_t launch_qp_setup(int dim, int p, int split, const double* U, const double* phit, const double* gcf,
                            const double* lamf, const double* muf, const Geom& g, const Tab<double>& tb,
                            const MatConst& mc, double* qp64, float* qp32, df64* qpdf, double* st64, cudaStream_t s,
                            double* sp64 = nullptr, int part = QP_ALL);
// diag(G_uu, G_phiphi) of a level into d (zeroed here), masked rows set to 1, from the per-point
// data of the same precision.
template <typename Real>
cudaError_t launch_diagonal(int dim, int p, int split, const Real* qp, const unsigned char* flags, const Geom& g,
                            const Tab<Real>& tb, Real* d, cudaStream_t s);
// (dR/dparam)^T v, three nodal outputs (zeroed here); tmp has 3 * n_cells * n^dim doubles.
cudaError_t launch_param_grad(int dim, int p, int split, const double* U, const double* v, const double* st64,
                              const Geom& g, const Tab<double>& tb, const MatConst& mc, double* tmp,
                              double* out_gc, double* out_lam, double* out_mu, cudaStream_t s);
// Dense coarse blocks: Au (nu x nu), Ap (nn x nn), B (nn x nu), masked rows/cols -> identity / 0.
cudaError_t launch_coarse_assemble(int dim, int p, int split, const double* qp64, const unsigned char* flags,
                                   const Geom& g, const Tab<double>& tb, double* Au, double* Ap, double* B,
                                   cudaStream_t s);
// In-place Gauss-Jordan inverse of an n x n matrix (no pivoting; SPD input), blocked;
// buf: gj_buffer_size(n) elements of the matrix type.
long long gj_buffer_size(int n);
template <typename Real>
cudaError_t launch_gj_inverse(Real* A, int n, Real* buf, cudaStream_t s);
// y = A x (dense, row major, n rows, m cols); y = beta * y + alpha * A x.
template <typename Real>
cudaError_t launch_gemv(const Real* A, int n, int m, const Real* x, Real* y, double alpha, double beta,
                        cudaStream_t s);

// Transfer tables of one degree (fine/coarse pair with ratio 2).
struct XferTab {
  double E[2 * MAXP + 1][MAXN];  // coarse basis k at the fine node o of a coarse cell
  double F[MAXN][MAXN];          // fine basis m at the coarse node k (inside fine cell FC[k])
  int FC[MAXN];
  int COL[MAXN];                 // fine offset co-located with coarse node k, or -1
};
template <typename Real>
cudaError_t launch_prolong(int dim, int p, const Real* xc, Real* yf, const unsigned char* flags_f,
                           const Geom& gc, const Geom& gf, const XferTab& xt, bool accumulate, cudaStream_t s);
// mask_fine = false skips Z_f (valid when x is already zero on masked fine rows, as the V-cycle's
// residuals are). With cs, also the first smoothing step on the coarse level (x = d = c0 dinv yc).
template <typename Real>
cudaError_t launch_restrict(int dim, int p, const Real* xf, Real* yc, const unsigned char* flags_f,
                            const unsigned char* flags_c, const Geom& gf, const Geom& gc, const XferTab& xt,
                            cudaStream_t s, bool mask_fine = true, const ChebStart<Real>* cs = nullptr);
// Evaluates `nfields` fine nodal fields (each nn_f long, consecutive) at the coarse nodes.
cudaError_t launch_state_interp(int dim, int p, const double* xf, double* yc, int nfields, const Geom& gf,
                                const Geom& gc, const XferTab& xt, cudaStream_t s);
// Coarse active bits from fine active bits at co-located nodes (the bit of field dim).
cudaError_t launch_coarse_active(int dim, int p, const unsigned char* flags_f, unsigned char* flags_c,
                                 const Geom& gf, const Geom& gc, const XferTab& xt, cudaStream_t s);

// ---- vectors ---------------------------------------------------------------------------
template <typename Real>
cudaError_t launch_axpby(long long n, double a, const Real* x, double b, Real* y, cudaStream_t s);
// res = r - t; t = 0; with cs.on also the first smoothing step of res (x = d = c0 dinv res).
template <typename Real>
cudaError_t launch_res_update(long long n, const Real* r, Real* t, Real* res, const ChebStart<Real>& cs,
                              cudaStream_t s);
template <typename Ti, typename To>
cudaError_t launch_cast(long long n, const Ti* x, To* y, cudaStream_t s);
// Two-block dot products of x and y over [0, nu) and [nu, n): result res[0], res[1] (device, FP64).
template <typename Real>
cudaError_t launch_dot2(long long n, long long nu, const Real* x, const Real* y, double* partial, double* res,
                        cudaStream_t s);
// h[i] = <V_i, w> for i < k, V row-major (k x n); partial >= k * 2 * 152 doubles.
cudaError_t launch_mdot(long long n, int k, const double* V, const double* w, double* partial, double* h,
                        cudaStream_t s);
// w -= sum_i V_i h[i]
cudaError_t launch_maxpy(long long n, int k, const double* V, const double* h, double* w, cudaStream_t s);
// x += sum_i Z_i y[i]
cudaError_t launch_zupdate(long long n, int k, const double* Z, const double* y, double* x, cudaStream_t s);
// y = x * inv[0]; with y32 != NULL also y32 = (float) y
cudaError_t launch_normalize(long long n, const double* x, const double* inv, double* y, float* y32,
                             cudaStream_t s);
// CGS2 of w against V_0 .. V_{k-1}: h1 = V^T w; w -= V h1; h2 = V^T w; w -= V h2; nrm = (<w, w>, 0, 1 / |w|).
// Three fused passes for k <= CGS_KMAX, else the separate passes; part >= max(CGS_KMAX, k) * CGS_GRID
// doubles; cnt: one zero-initialised counter (left zero).
constexpr int CGS_KMAX = 16;
constexpr int CGS_GRID_MAX = 152 * 4;  // four CTAs per SM (eight were slower for bases of 1 to 4 vectors)
cudaError_t launch_cgs2(long long n, int k, const double* V, double* w, double* part, double* h1, double* h2,
                        double* nrm, unsigned* cnt, cudaStream_t s);

// ---- Chebyshev-Jacobi and eigenvalue estimation -----------------------------------------
// step 0: x = d = dinv f / theta_b; step k: d = c1 d + (2 rho_k / delta_b) dinv (f - Ax), x += d,
// with 1 / theta_b = c0s inv_lam[b] and 2 rho_k / delta_b = c2s inv_lam[b] (inv_lam = 1 / lambda_max).
template <typename Real>
cudaError_t launch_cheb(int step, long long n, long long nu, const Real* f, const Real* Ax, const Real* dinv,
                        Real* d, Real* x, const Real* inv_lam, double c0s, double c1, double c2s, cudaStream_t s);
// CG-Lanczos on the two diagonal blocks (vectors in the multigrid precision, scalars in FP64).
// scal holds 16 doubles: [rz0 rz1 pAp0 pAp1 alpha0 alpha1 beta0 beta1 rzn0 rzn1 dead0 dead1], then a
// reduction counter that must be zero before the first call (every call leaves it zero); part holds
// 2 * 304 doubles. The histories are [2][iters].
// r = random start (0 on masked rows), z = pv = D^{-1} r, rz = <r, z>.
template <typename Real>
cudaError_t launch_cg_init(long long n, long long nu, unsigned long long seed, const unsigned char* flags,
                           long long nn, const Real* dinv, Real* r, Real* z, Real* pv, double* part, double* scal,
                           cudaStream_t s);
// pAp = <p, Ap>, alpha = rz / pAp -> alpha_hist[.][it].
template <typename Real>
cudaError_t launch_cg_pap(long long n, long long nu, const Real* pv, const Real* Ap, double* part, double* scal,
                          double* alpha_hist, int it, int iters, cudaStream_t s);
// r -= alpha Ap, z = D^{-1} r, Ap = 0, beta = <r, z> / rz -> beta_hist[.][it], rz = <r, z>.
template <typename Real>
cudaError_t launch_cg_update(long long n, long long nu, Real* Ap, const Real* dinv, double* scal, Real* r, Real* z,
                             double* part, double* beta_hist, int it, int iters, cudaStream_t s);
template <typename Real>
cudaError_t launch_cg_pupdate(long long n, long long nu, const Real* z, const double* scal, Real* pv,
                              cudaStream_t s);
// lam_max[b] from the Lanczos tridiagonal of the first k_valid CG steps of each block; lam holds 8
// doubles: lam_max[2], Gershgorin lower bounds[2], 1 / lam_max[2] (0 if unusable), and the two FP32
// inverses packed into lam[6].
cudaError_t launch_tridiag_eig(int iters, const double* alpha_hist, const double* beta_hist, double* lam,
                               cudaStream_t s);

// di = 1 / d (FP64 and, when di32 is not null, FP32 copies): the Jacobi scaling of the smoother.
cudaError_t launch_inv_diag(long long n, const double* d, double* di64, float* di32, cudaStream_t s);
// di32 = 1 / d (FP32 diagonal of the FP32 multigrid).
cudaError_t launch_inv_diag32(long long n, const float* d, float* di32, cudaStream_t s);

// ---- Newton step helpers ----------------------------------------------------------------
// Active set of Alg. 1 on the phase-field block: sets/clears the active bit (field dim), resets
// phi := phi_old on it, counts |A| and changes (cnt[0], cnt[1], device ints zeroed here).
cudaError_t launch_active_set(int dim, long long nn, const double* R, const double* mass, const double* phi_old,
                              double c, double* U, unsigned char* flags, int* cnt, cudaStream_t s);
// rhs = -R on unmasked rows, 0 on masked rows (all flag bits).
cudaError_t launch_newton_rhs(int dim, long long nn, const double* R, const unsigned char* flags, double* rhs,
                              cudaStream_t s);
// out = 0 where the node's flag bit of the field is set in `bits`, scale * x elsewhere.
cudaError_t launch_masked_copy(int dim, long long nn, double scale, const double* x, const unsigned char* flags,
                               unsigned bits, double* out, cudaStream_t s);
// Copies the active bit (field dim) from a byte array (nonzero = active) into the flags.
cudaError_t launch_set_active(int dim, long long nn, const unsigned char* active, unsigned char* flags,
                              cudaStream_t s);
cudaError_t launch_get_active(int dim, long long nn, const unsigned char* flags, unsigned char* active,
                              cudaStream_t s);
// Load step: u_comp := load on the top face; phi~ = clamp(2 h1 - h2, 0, 1) (h1 if h2 is null), phi_old = h1.
cudaError_t launch_load_step_prep(int comp, long long nn, const unsigned char* flags, double load, double* U,
                                  const double* h1, const double* h2, double* phit, double* phi_old, cudaStream_t s);
// Lumped phase-field mass: int psi_i over the mesh (tensor product of 1D GLL weight sums).
cudaError_t launch_lumped_mass(int dim, long long nn, int n1, const double* w1, double* mass, cudaStream_t s);

}  // namespace pff
