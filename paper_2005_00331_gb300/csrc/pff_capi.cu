// pff_capi.cu -- context, host orchestration and the C-ABI of libpff (see include/pff.h).
//
// The host side only builds meshes and tables, allocates, launches kernels on the caller's
// stream and keeps the scalar bookkeeping of the Krylov solver (Hessenberg matrix, Givens
// rotations). Every vector operation of the hot path runs in the kernels of this library.
#include <chrono>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pff.h"
#include "pff_kernels.h"
#include "pff_csr.h"
#include "pff_launch.h"

using namespace pff;

namespace {

// NVTX range over a scope: the entry points and the phases of a Newton step show up by name in
// profilers that trace NVTX (ncu --nvtx); without such a tool attached the calls do nothing.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
// Consecutive NVTX ranges for the phases of one call (each next() ends the previous phase).
struct Phases {
  bool open = false;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~Phases() {
    if (open) nvtxRangePop();
  }
};

// ---- 1D bases (closed forms for p <= 4) ----------------------------------------------------
void gll_nodes(int p, double* x) {
  const double s5 = 1.0 / std::sqrt(5.0), s37 = std::sqrt(3.0 / 7.0);
  switch (p) {
    case 1: x[0] = 0; x[1] = 1; break;
    case 2: x[0] = 0; x[1] = 0.5; x[2] = 1; break;
    case 3: x[0] = 0; x[1] = 0.5 * (1 - s5); x[2] = 0.5 * (1 + s5); x[3] = 1; break;
    default: x[0] = 0; x[1] = 0.5 * (1 - s37); x[2] = 0.5; x[3] = 0.5 * (1 + s37); x[4] = 1; break;
  }
}
void gll_weights(int p, double* w) {
  switch (p) {
    case 1: w[0] = w[1] = 0.5; break;
    case 2: w[0] = w[2] = 1.0 / 6; w[1] = 2.0 / 3; break;
    case 3: w[0] = w[3] = 1.0 / 12; w[1] = w[2] = 5.0 / 12; break;
    default: w[0] = w[4] = 1.0 / 20; w[1] = w[3] = 49.0 / 180; w[2] = 32.0 / 90; break;
  }
}
// n-point Gauss-Legendre on [0, 1] (closed forms of the roots of P_n).
void gauss(int n, double* x, double* w) {
  double t[5], v[5];
  switch (n) {
    case 1: t[0] = 0; v[0] = 2; break;
    case 2: t[0] = -1 / std::sqrt(3.0); t[1] = -t[0]; v[0] = v[1] = 1; break;
    case 3:
      t[0] = -std::sqrt(0.6); t[1] = 0; t[2] = -t[0];
      v[0] = v[2] = 5.0 / 9; v[1] = 8.0 / 9; break;
    case 4: {
      const double a = std::sqrt(3.0 / 7 - 2.0 / 7 * std::sqrt(6.0 / 5)), b = std::sqrt(3.0 / 7 + 2.0 / 7 * std::sqrt(6.0 / 5));
      t[0] = -b; t[1] = -a; t[2] = a; t[3] = b;
      v[1] = v[2] = (18 + std::sqrt(30.0)) / 36; v[0] = v[3] = (18 - std::sqrt(30.0)) / 36; break;
    }
    default: {
      const double a = std::sqrt(5 - 2 * std::sqrt(10.0 / 7)) / 3, b = std::sqrt(5 + 2 * std::sqrt(10.0 / 7)) / 3;
      t[0] = -b; t[1] = -a; t[2] = 0; t[3] = a; t[4] = b;
      v[2] = 128.0 / 225; v[1] = v[3] = (322 + 13 * std::sqrt(70.0)) / 900; v[0] = v[4] = (322 - 13 * std::sqrt(70.0)) / 900;
      break;
    }
  }
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (t[i] + 1);
    w[i] = 0.5 * v[i];
  }
}
double lag(const double* nd, int nn, int k, double x) {
  double v = 1;
  for (int m = 0; m < nn; ++m)
    if (m != k) v *= (x - nd[m]) / (nd[k] - nd[m]);
  return v;
}
double dlag(const double* nd, int nn, int k, double x) {
  double s = 0;
  for (int j = 0; j < nn; ++j) {
    if (j == k) continue;
    double t = 1 / (nd[k] - nd[j]);
    for (int m = 0; m < nn; ++m)
      if (m != k && m != j) t *= (x - nd[m]) / (nd[k] - nd[m]);
    s += t;
  }
  return s;
}

const char* g_last_cuda = "";

}  // namespace

// ---- context --------------------------------------------------------------------------------
// Work vectors per level and precision: r, e, t, res, dv, s, and the second iterate / direction buffers
// and two more seam-sum buffers of the 2D smoother (xb, db, t0, t2).
constexpr int NWORK = 10;

struct LevelData {
  int N = 0;
  long long nn = 0, nd = 0;
  double h = 0;
  Geom g{};
  Tab<double> t64{};
  Tab<float> t32{};
  unsigned char* flags = nullptr;
  double* U = nullptr;      // state DoF vector
  double* phit = nullptr;   // phi~ (follows U in memory so one interpolation covers both)
  double* fields = nullptr; // 3 nodal fields (G_c, lambda, mu) when given
  double* qp64 = nullptr;
  float* qp32 = nullptr;
  df64* qpdf = nullptr;     // per-point data as double-word pairs (float-float FP64 applies)
  Tab<df64> tdf{};
  double* st64 = nullptr;
  double* sp64 = nullptr;   // finest level, Miehe split: sigma+ (Mandel) and E_s+ per point of the current u
  double* d64 = nullptr;    // diagonal of diag(G_uu, G_phiphi), masked rows 1
  double* di64 = nullptr;   // its inverse (Jacobi scaling)
  float* s32 = nullptr;     // 2D: the state (u_x, u_y, phi, phi~) in FP32, read by the recomputed FP32 Jacobian
  float* d32 = nullptr;     // the diagonal computed in FP32 from the FP32 per-point data (FP32 multigrid)
  float* di32 = nullptr;
  double* lam = nullptr;    // device [lmax_u, lmax_phi, lower bounds]
  // per-level reduction scratch, so that the levels' setup branches can run concurrently
  double* lscal = nullptr;  // 16
  double* lhist = nullptr;  // 4 * eig_iters
  double* lpart = nullptr;  // reduction partials
  cudaStream_t aux = nullptr;
  cudaEvent_t join = nullptr;
  // multigrid work vectors, per precision: r, e, t, res, dv, s
  double* w64[NWORK] = {};
  float* w32[NWORK] = {};
};

struct pff_ctx {
  pff_params prm{};
  cudaStream_t s = nullptr;
  int dim = 2, p = 1, nlev = 0, nv = 0;
  std::vector<LevelData> lv;
  XferTab xt{};
  bool has_state = false, qp_valid = false, mg_ready = false, has_fields = false;
  bool st_valid = false;    // per-point residual state (depends on phi~ and the fields, not on U)
  bool strain_valid = false;  // finest-level strain pass (eigen-decompositions) of the current u
  bool diag64_ok = false;   // FP64 diagonals present (always with the FP64 multigrid; on demand with FP32)
  double* phi_old = nullptr;
  double* hist1 = nullptr;  // phase field of the previous load step
  double* hist2 = nullptr;  // ... and of the one before
  int nhist = 0;
  int load_comp = -1;       // displacement component of the top-face load (-1: dim - 1, tension)
  double* mass = nullptr;
  double* R = nullptr;
  double* rhs = nullptr;
  double* dU = nullptr;
  double* scratch = nullptr;   // 4 fine-sized FP64 vectors (CG-Lanczos, residual checks)
  double* partial = nullptr;   // reduction partials
  unsigned* kcnt = nullptr;    // CTA counter of the fused CGS2 passes (zero between launches)
  cudaEvent_t hcol = nullptr;  // recorded after the copy of an FGMRES Hessenberg column to the host
  const double* w32_of = nullptr;  // the FP64 vector whose FP32 copy the finest w32[0] holds, if any
  double* dres = nullptr;      // small device results
  double* hist = nullptr;      // CG alpha/beta histories
  int* cnt = nullptr;
  double* pinned = nullptr;    // host pinned scalars
  double* pgrad_tmp = nullptr;
  pff::CsrMat* csr = nullptr;  // assembled comparator matrix (pff_csr_assemble)
  // coarse dense blocks
  double *Au = nullptr, *Ap = nullptr, *Bc = nullptr, *gjbuf = nullptr, *cr = nullptr, *ce = nullptr, *ct = nullptr;
  // FP32 copies of the coarse blocks and their inverses (multigrid in FP32)
  float *Au32 = nullptr, *Ap32 = nullptr, *Bc32 = nullptr, *gjbuf32 = nullptr, *cr32 = nullptr, *ce32 = nullptr,
        *ct32 = nullptr;
  // FGMRES
  double *V = nullptr, *Z = nullptr, *w = nullptr, *hdev = nullptr, *ydev = nullptr;
  std::vector<void*> allocs;
  // bytes of device memory held, by owner (dalloc's tag): per level, Krylov basis, coarse blocks, other
  std::vector<long long> level_bytes;
  long long krylov_bytes = 0, coarse_bytes = 0, other_bytes = 0;
  // V-cycle replayed as a CUDA graph (captured once on a private stream; buffers never move)
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  // graphs: [0] FP64 / [1] FP32 V-cycle; setup without / with nodal fields; each in a plain variant
  // and one variant per timed kernel family (event-record nodes around the timed launches)
  cudaGraphExec_t vgraph[2][6] = {};
  bool vwarm[2] = {false, false};
  cudaGraphExec_t sgraph[2][6] = {};
  bool swarm[2] = {false, false};
  // event slots recorded by each profiled graph, and the replays whose events await collection
  std::vector<cudaEvent_t> gev;  // created by pff_profile; graphs take slots in capture order
  int gnext = 0;
  std::vector<std::pair<int, int>> vrange[2][6], srange[2][6];
  long long vkern[2][6] = {}, skern[2][6] = {};  // kernel launches per replay of each graph
  std::vector<std::pair<int, int>> pending;
  double prof_ms = 0.0;
  long long prof_n = 0;
  bool capturing = false;
  bool use_graph = true;
  bool fresh_active = false;  // the active set was just computed from the current U (set_state, active = NULL)
  int device = -1;  // the device of the context's stream, recorded at setup
  // kernel-family timing (pff_profile)
  int prof = 0;
  std::vector<cudaEvent_t> ev;
  int nev = 0;
};

// The coarse solve runs in FP32 only when the FP32 multigrid asks for it (coarse_precision 32).
inline bool coarse32(const pff_ctx* c) { return c->prm.mg_precision == 32 && c->prm.coarse_precision == 32; }
// With fp32_tangent = 1 the FP32 Jacobian of a 2D level is recomputed at the Gauss points from the nodal
// state (rather than read from the stored per-point data), unless nodal material fields are set (the
// recomputation takes constant lambda, mu, G_c).
inline bool use_rc32(const pff_ctx* c) { return c->dim == 2 && c->prm.fp32_tangent == 1 && !c->has_fields; }

namespace {

// Owners of device memory for the accounting of pff_memory: a level index (>= 0) or one of these.
constexpr int TAG_OTHER = -1, TAG_KRYLOV = -2, TAG_COARSE = -3;

template <typename T>
int dalloc(pff_ctx* c, T** p, long long n, int tag = TAG_OTHER) {
  *p = nullptr;
  if (n <= 0) n = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    return PFF_ERR_OOM;
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  const long long bytes = (long long)sizeof(T) * n;
  if (tag >= 0) {
    if ((size_t)tag >= c->level_bytes.size()) c->level_bytes.resize((size_t)tag + 1, 0);
    c->level_bytes[(size_t)tag] += bytes;
  } else if (tag == TAG_KRYLOV) {
    c->krylov_bytes += bytes;
  } else if (tag == TAG_COARSE) {
    c->coarse_bytes += bytes;
  } else {
    c->other_bytes += bytes;
  }
  return PFF_OK;
}

#define CK(...)                                 \
  do {                                          \
    cudaError_t e_ = (__VA_ARGS__);             \
    if (e_ != cudaSuccess) {                    \
      g_last_cuda = cudaGetErrorString(e_);     \
      cudaGetLastError();                       \
      return PFF_ERR_CUDA;                      \
    }                                           \
  } while (0)
#define CR(...)               \
  do {                        \
    int r_ = (__VA_ARGS__);   \
    if (r_ != PFF_OK) return r_; \
  } while (0)

void make_geom(LevelData& L, int dim, int p, bool cut) {
  Geom& g = L.g;
  g.dim = dim;
  g.p = p;
  g.N = L.N;
  g.n1 = p * L.N + 1;
  g.nn = L.nn;
  g.ngrid = dim == 2 ? (long long)g.n1 * g.n1 : (long long)g.n1 * g.n1 * g.n1;
  int t[3];
  tile_shape(dim, p, t);
  g.cut = cut ? 1 : 0;
  g.cut_row = p * L.N / 2;
  g.cut_x = p * L.N / 2;
  g.cut_tile = cut ? (L.N / 2) / t[dim - 1] - 1 : -1;
  for (int i = 0; i < 3; ++i) {
    g.tdim[i] = t[i];
    g.ntile[i] = (i < dim) ? (L.N + t[i] - 1) / t[i] : 1;
  }
  g.qpx = t[0] * (p + 1);
  g.qpy = t[1] * (p + 1);
  g.qpz = dim == 3 ? t[2] * (p + 1) : 1;
  g.qpt = (long long)g.qpx * g.qpy * g.qpz;
  g.ntiles = (long long)g.ntile[0] * g.ntile[1] * g.ntile[2];
}

void make_tabs(LevelData& L, int dim, int p) {
  const int n = p + 1;
  double xn[MAXN], xq[MAXN], wq[MAXN];
  gll_nodes(p, xn);
  gauss(n, xq, wq);
  std::memset(&L.t64, 0, sizeof(L.t64));
  std::memset(&L.t32, 0, sizeof(L.t32));
  for (int q = 0; q < n; ++q) {
    for (int k = 0; k < n; ++k) {
      L.t64.S[q][k] = lag(xn, n, k, xq[q]);
      L.t64.D[q][k] = dlag(xn, n, k, xq[q]) / L.h;
      L.t32.S[q][k] = (float)L.t64.S[q][k];
      L.t32.D[q][k] = (float)L.t64.D[q][k];
    }
    L.t64.W[q] = wq[q];
    L.t32.W[q] = (float)wq[q];
  }
  L.t64.hd = std::pow(L.h, dim);
  L.t32.hd = (float)L.t64.hd;
  auto split = [](double v) { return df64((float)v, (float)(v - (double)(float)v)); };
  for (int q = 0; q < MAXN; ++q) {
    for (int k = 0; k < MAXN; ++k) {
      L.tdf.S[q][k] = split(L.t64.S[q][k]);
      L.tdf.D[q][k] = split(L.t64.D[q][k]);
    }
    L.tdf.W[q] = split(L.t64.W[q]);
  }
  L.tdf.hd = split(L.t64.hd);
}

void make_xfer(XferTab& xt, int p) {
  double xn[MAXN];
  gll_nodes(p, xn);
  const int n = p + 1;
  std::memset(&xt, 0, sizeof(xt));
  for (int o = 0; o <= 2 * p; ++o) {
    const int fc = (o == 2 * p) ? 1 : o / p;
    const int j = o - fc * p;
    const double xi = 0.5 * (fc + xn[j]);
    for (int k = 0; k < n; ++k) {
      double v = lag(xn, n, k, xi);
      if (std::fabs(v) < 1e-15) v = 0.0;
      xt.E[o][k] = v;
    }
  }
  for (int k = 0; k < n; ++k) {
    const int fc = xn[k] < 0.5 ? 0 : 1;
    const double t = 2 * xn[k] - fc;
    xt.FC[k] = fc;
    xt.COL[k] = -1;
    for (int m = 0; m < n; ++m) {
      double v = lag(xn, n, m, t);
      if (std::fabs(v) < 1e-15) v = 0.0;
      xt.F[k][m] = v;
      if (std::fabs(t - xn[m]) < 1e-12) xt.COL[k] = fc * p + m;
    }
  }
}

// Node flags of a level (tension test: Dirichlet faces, slit), computed on the host.
// Number of copied slit nodes of a mesh with the slit cut into it: x index < p N / 2 on the slit, every y
// index in 3D.
long long cut_copies(int dim, int p, int N) {
  const long long n1 = (long long)p * N + 1;
  return (long long)(p * N / 2) * (dim == 2 ? 1 : n1);
}

std::vector<unsigned char> host_flags(int dim, int p, int N, bool cut) {
  const int n1 = p * N + 1;
  double xn[MAXN];
  gll_nodes(p, xn);
  std::vector<double> x1(n1);
  for (int i = 0; i < n1; ++i) {
    int c = i / p, k = i % p;
    if (c == N) {
      c = N - 1;
      k = p;
    }
    x1[i] = (c + xn[k]) / N;
  }
  long long nn = 1;
  for (int t = 0; t < dim; ++t) nn *= n1;
  std::vector<unsigned char> fl(nn, 0);
  for (long long i = 0; i < nn; ++i) {
    long long rem = i;
    int ijk[3] = {0, 0, 0};
    for (int t = 0; t < dim; ++t) {
      ijk[t] = int(rem % n1);
      rem /= n1;
    }
    const int vert = ijk[dim - 1];
    unsigned char f = 0;
    if (vert == 0) f |= PFF_FLAG_BOTTOM;
    if (vert == n1 - 1) f |= PFF_FLAG_TOP;
    if (vert == 0 || vert == n1 - 1)
      for (int c = 0; c < dim; ++c) f |= (unsigned char)(1u << c);
    if (std::fabs(x1[vert] - 0.5) <= 1e-12 && x1[ijk[0]] <= 0.5 + 1e-12) f |= PFF_FLAG_SLIT;
    fl[i] = f;
  }
  if (cut) {  // copies of the slit nodes (x index < p N / 2), x fastest, then y (3D)
    const int half = p * N / 2;
    const long long ny = dim == 2 ? 1 : n1;
    for (long long y = 0; y < ny; ++y)
      for (int x = 0; x < half; ++x) {
        const long long gnode = x + n1 * (dim == 2 ? (long long)half : y + n1 * half);
        fl.push_back((unsigned char)(fl[gnode] | PFF_FLAG_COPY));
      }
  }
  return fl;
}

template <typename Real> Real* qp_of(LevelData& L);
template <> double* qp_of<double>(LevelData& L) { return L.qp64; }
template <> float* qp_of<float>(LevelData& L) { return L.qp32; }
template <typename Real> const Tab<Real>& tab_of(LevelData& L);
template <> const Tab<double>& tab_of<double>(LevelData& L) { return L.t64; }
template <> const Tab<float>& tab_of<float>(LevelData& L) { return L.t32; }
template <typename Real> Real* dinv_of(LevelData& L);
template <> double* dinv_of<double>(LevelData& L) { return L.di64; }
// 1 / lambda_max of the two blocks in the given precision (written by the eigenvalue estimate)
template <typename Real> const Real* inv_lam_of(LevelData& L);
template <> const double* inv_lam_of<double>(LevelData& L) { return L.lam + 4; }
template <> const float* inv_lam_of<float>(LevelData& L) { return reinterpret_cast<const float*>(L.lam + 6); }
template <> float* dinv_of<float>(LevelData& L) { return L.di32; }
template <typename Real> Real** work_of(LevelData& L);
template <> double** work_of<double>(LevelData& L) { return L.w64; }
template <> float** work_of<float>(LevelData& L) { return L.w32; }

template <typename Real>
int ensure_work(pff_ctx* c, int l) {
  LevelData& L = c->lv[l];
  Real** w = work_of<Real>(L);
  if (w[0]) return PFF_OK;
  for (int i = 0; i < NWORK; ++i) {
    CR(dalloc(c, &w[i], L.nd, l));
    CK(cudaMemsetAsync(w[i], 0, sizeof(Real) * L.nd, c->s));
  }
  return PFF_OK;
}

constexpr int PROF_MAX_LAUNCHES = 16384;

bool prof_on(pff_ctx* c, int family) {
  return c->prof == family && (c->capturing || c->nev + 2 <= (int)c->ev.size());
}
// Records one timing event: from the per-call pool when running eagerly, from a fresh persistent
// event when the call is being captured into a graph (the event becomes an event-record node).
int prof_mark(pff_ctx* c) {
  if (c->capturing) {
    if (c->gnext >= (int)c->gev.size()) return PFF_OK;  // pool exhausted: this launch is not timed
    CK(cudaEventRecordWithFlags(c->gev[c->gnext++], c->s, cudaEventRecordExternal));
    return PFF_OK;
  }
  CK(cudaEventRecord(c->ev[c->nev++], c->s));
  return PFF_OK;
}
// After the stream has synchronised: adds the timings of graph replays launched since the last call.
int prof_collect(pff_ctx* c) {
  for (auto& r : c->pending) {
    for (int i = r.first; i + 1 < r.second; i += 2) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->gev[i], c->gev[i + 1]));
      c->prof_ms += ms;
      ++c->prof_n;
    }
  }
  c->pending.clear();
  return PFF_OK;
}

// Is a Jacobian launch of this precision on level l in the profiled family?
template <typename Real>
bool prof_jac(pff_ctx* c, int l) {
  const bool d = sizeof(Real) == 8;
  return prof_on(c, d ? PFF_PROF_JAC64 : PFF_PROF_JAC32) ||
         (l == 0 && prof_on(c, d ? PFF_PROF_JAC64_L0 : PFF_PROF_JAC32_L0));
}

// y = G x on level l (y zeroed first). With ce (2D), a fused Chebyshev step, with cg (2D) a CG-Lanczos
// step: see launch_jac; such
// launches are not timed by pff_profile (they move more than the apply's bytes).
template <typename Real>
int apply_level(pff_ctx* c, int l, const Real* x, Real* y, int mode, int inmask, int outmask,
                const ChebEpi<Real>* ce = nullptr, bool y_is_zero = false, const CgEpi<Real>* cg = nullptr) {
  LevelData& L = c->lv[l];
  if (!y_is_zero) CK(cudaMemsetAsync(y, 0, sizeof(Real) * L.nd, c->s));
  const bool timed = !ce && !cg && prof_jac<Real>(c, l);  // plain applies only
  if (timed) CR(prof_mark(c));
  if (sizeof(Real) == 8 && c->prm.fp64_mode == 1) {
    if (c->dim == 2)
      CK(launch_jac_df(c->dim, c->p, c->prm.split, reinterpret_cast<const double*>(x), reinterpret_cast<double*>(y),
                       L.flags, L.g, L.tdf, L.qpdf, mode, inmask, outmask, c->s,
                       reinterpret_cast<const ChebEpi<double>*>(ce), reinterpret_cast<const CgEpi<double>*>(cg)));
    else
      CK(launch_jac_df3(c->dim, c->p, c->prm.split, reinterpret_cast<const double*>(x), reinterpret_cast<double*>(y),
                        L.flags, L.g, L.tdf, L.qpdf, mode, inmask, outmask, c->s));
  } else if (sizeof(Real) == 4 && L.s32 && use_rc32(c)) {
    const float ke = (float)c->prm.kappa;
    const Rc32 rc{L.s32, MatConst32{(float)c->prm.lambda, (float)c->prm.mu, (float)(c->prm.gc * c->prm.eps),
                                    (float)(c->prm.gc / c->prm.eps), 1.0f - ke, ke}};
    CK(launch_jac(c->dim, c->p, c->prm.split, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(y),
                  L.flags, L.g, L.t32, L.qp32, mode, inmask, outmask, c->s,
                  reinterpret_cast<const ChebEpi<float>*>(ce), &rc, reinterpret_cast<const CgEpi<float>*>(cg)));
  } else if (sizeof(Real) == 4) {
    CK(launch_jac(c->dim, c->p, c->prm.split, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(y),
                  L.flags, L.g, L.t32, L.qp32, mode, inmask, outmask, c->s,
                  reinterpret_cast<const ChebEpi<float>*>(ce), nullptr, reinterpret_cast<const CgEpi<float>*>(cg)));
  } else {
    CK(launch_jac(c->dim, c->p, c->prm.split, reinterpret_cast<const double*>(x), reinterpret_cast<double*>(y),
                  L.flags, L.g, L.t64, L.qp64, mode, inmask, outmask, c->s,
                  reinterpret_cast<const ChebEpi<double>*>(ce), reinterpret_cast<const CgEpi<double>*>(cg)));
  }
  if (timed) CR(prof_mark(c));
  return PFF_OK;
}

// FP32 copy of a level's state for the recomputed FP32 Jacobian: U (u_x, u_y, phi) and phi~ are
// contiguous, so one cast covers the four fields.
int state32_level(pff_ctx* c, int l) {
  LevelData& L = c->lv[l];
  if (L.s32 && use_rc32(c)) CK(launch_cast<double, float>((c->dim + 2) * L.nn, L.U, L.s32, c->s));
  return PFF_OK;
}

int qp_setup_level(pff_ctx* c, int l) {
  LevelData& L = c->lv[l];
  MatConst mc{c->prm.lambda, c->prm.mu, c->prm.gc, c->prm.eps, c->prm.kappa};
  const double* F = L.fields;
  CK(launch_qp_setup(c->dim, c->p, c->prm.split, L.U, L.phit, c->has_fields ? F : nullptr,
                     c->has_fields ? F + L.nn : nullptr, c->has_fields ? F + 2 * L.nn : nullptr, L.g, L.t64, mc,
                     L.qp64, L.qp32, L.qpdf, L.st64, c->s));
  return state32_level(c, l);
}

int ensure_st(pff_ctx* c);

// Miehe split, finest level: the per-point work that depends on u only (eigen-decomposition,
// tangent, sigma+ and E_s+ for the residual), once per u; the active-set projection changes phi only.
int ensure_strain(pff_ctx* c) {
  CR(ensure_st(c));
  if (!c->strain_valid) {
    LevelData& L = c->lv[0];
    MatConst mc{c->prm.lambda, c->prm.mu, c->prm.gc, c->prm.eps, c->prm.kappa};
    const double* F = L.fields;
    CK(launch_qp_setup(c->dim, c->p, c->prm.split, L.U, L.phit, c->has_fields ? F : nullptr,
                       c->has_fields ? F + L.nn : nullptr, c->has_fields ? F + 2 * L.nn : nullptr, L.g, L.t64, mc,
                       L.qp64, L.qp32, L.qpdf, nullptr, c->s, L.sp64, QP_STRAIN));
    c->strain_valid = true;
  }
  return PFF_OK;
}

// Tangent per-point data of the finest level (and the residual state with it).
int ensure_qp(pff_ctx* c) {
  if (!c->has_state) return PFF_ERR_NO_STATE;
  if (c->qp_valid) return PFF_OK;
  LevelData& L = c->lv[0];
  if (L.sp64) {
    CR(ensure_strain(c));
    MatConst mc{c->prm.lambda, c->prm.mu, c->prm.gc, c->prm.eps, c->prm.kappa};
    const double* F = L.fields;
    CK(launch_qp_setup(c->dim, c->p, c->prm.split, L.U, L.phit, c->has_fields ? F : nullptr,
                       c->has_fields ? F + L.nn : nullptr, c->has_fields ? F + 2 * L.nn : nullptr, L.g, L.t64, mc,
                       L.qp64, L.qp32, L.qpdf, nullptr, c->s, L.sp64, QP_PHASE));
    CR(state32_level(c, 0));
  } else {
    CR(qp_setup_level(c, 0));
    c->st_valid = true;
  }
  c->qp_valid = true;
  return PFF_OK;
}

// Residual state per point only (g(phi~), G_c, lambda, mu): what the residual and the parameter
// gradient read; it does not change with U, so Newton iterations do not recompute it.
int ensure_st(pff_ctx* c) {
  if (!c->has_state) return PFF_ERR_NO_STATE;
  if (!c->st_valid) {
    LevelData& L = c->lv[0];
    MatConst mc{c->prm.lambda, c->prm.mu, c->prm.gc, c->prm.eps, c->prm.kappa};
    const double* F = L.fields;
    CK(launch_qp_setup(c->dim, c->p, c->prm.split, L.U, L.phit, c->has_fields ? F : nullptr,
                       c->has_fields ? F + L.nn : nullptr, c->has_fields ? F + 2 * L.nn : nullptr, L.g, L.t64, mc,
                       nullptr, nullptr, nullptr, L.st64, c->s));
    c->st_valid = true;
    c->strain_valid = false;  // the tangent depends on g(phi~) and the fields
    c->qp_valid = false;
  }
  return PFF_OK;
}

// FP64 diagonals of every level when the multigrid runs in FP32 (for FP64 queries and smoothing).
int ensure_diag64(pff_ctx* c) {
  if (c->diag64_ok) return PFF_OK;
  for (int l = 0; l < c->nlev; ++l) {
    LevelData& L = c->lv[l];
    CK(launch_diagonal<double>(c->dim, c->p, c->prm.split, L.qp64, L.flags, L.g, L.t64, L.d64, c->s));
    CK(launch_inv_diag(L.nd, L.d64, L.di64, nullptr, c->s));
  }
  c->diag64_ok = true;
  return PFF_OK;
}

int load_comp(const pff_ctx* c) { return c->load_comp < 0 ? c->dim - 1 : c->load_comp; }

int residual_into(pff_ctx* c, double* r, int outmask = OUT_ZERO_DIRICHLET) {
  CR(ensure_st(c));
  LevelData& L = c->lv[0];
  if (L.sp64) CR(ensure_strain(c));
  CK(cudaMemsetAsync(r, 0, sizeof(double) * L.nd, c->s));
  const bool timed = prof_on(c, PFF_PROF_RESIDUAL);
  if (timed) CR(prof_mark(c));
  CK(launch_res(c->dim, c->p, c->prm.split, L.U, r, L.flags, L.g, L.t64, L.st64, L.sp64, c->prm.eps, c->prm.kappa,
                c->s, outmask));
  if (timed) CR(prof_mark(c));
  return PFF_OK;
}

// lambda_max of D^{-1} G_uu and D^{-1} G_phiphi on level l by CG-Lanczos, in the precision of the
// multigrid that uses it (the estimate only places the smoothing interval); scalars in FP64.
template <typename Real>
int eig_estimate(pff_ctx* c, int l) {
  LevelData& L = c->lv[l];
  const long long n = L.nd, nu = c->dim * L.nn;
  CR(ensure_work<Real>(c, l));
  Real** w = work_of<Real>(L);
  Real *r = w[0], *z = w[1], *pv = w[2], *Ap = w[3];
  double* scal = L.lscal;  // 12 doubles and the reduction counter
  const int it_max = c->prm.eig_iters;
  double* ah = L.lhist;
  double* bh = L.lhist + 2 * it_max;
  CK(cudaMemsetAsync(scal, 0, 16 * sizeof(double), c->s));
  CK(cudaMemsetAsync(L.lhist, 0, 4 * it_max * sizeof(double), c->s));
  CK(cudaMemsetAsync(Ap, 0, sizeof(Real) * n, c->s));
  CK(launch_cg_init<Real>(n, nu, c->prm.eig_seed, L.flags, L.nn, dinv_of<Real>(L), r, z, pv, L.lpart, scal, c->s));
  if (c->dim == 2) {
    // the direction update p = z + beta p and <p, A p> (with alpha) are done by the apply (CgEpi): two
    // launches per step. p alternates between pv and w[6] (another tile may still read the old p).
    Real* P[2] = {pv, w[6]};
    for (int it = 0; it < it_max; ++it) {
      CgEpi<Real> cg{};
      cg.on = 1;
      cg.p_old = P[it % 2];  // beta is 0 at the first step (scal zeroed above)
      cg.p_out = P[(it + 1) % 2];
      cg.scal = scal;
      cg.part = L.lpart;
      cg.ah = ah;
      cg.it = it;
      cg.iters = it_max;
      // Ap is zero here: zeroed above, then by every update
      CR(apply_level<Real>(c, l, z, Ap, JM_BLOCKDIAG, IN_ALL, OUT_IDENTITY, nullptr, true, &cg));
      CK(launch_cg_update<Real>(n, nu, Ap, dinv_of<Real>(L), scal, r, z, L.lpart, bh, it, it_max, c->s));
    }
  } else {
    for (int it = 0; it < it_max; ++it) {
      // Ap is zero here: zeroed above, then by every update
      CR(apply_level<Real>(c, l, pv, Ap, JM_BLOCKDIAG, IN_ALL, OUT_IDENTITY, nullptr, true));
      CK(launch_cg_pap<Real>(n, nu, pv, Ap, L.lpart, scal, ah, it, it_max, c->s));
      CK(launch_cg_update<Real>(n, nu, Ap, dinv_of<Real>(L), scal, r, z, L.lpart, bh, it, it_max, c->s));
      CK(launch_cg_pupdate<Real>(n, nu, z, scal, pv, c->s));
    }
  }
  CK(launch_tridiag_eig(it_max, ah, bh, L.lam, c->s));
  CK(cudaMemsetAsync(pv, 0, sizeof(Real) * n, c->s));  // w[2] is the smoother's zeroed apply buffer
  return PFF_OK;
}

// Setup work of one level that does not depend on other levels once its state is known: per-point
// data (coarse levels), diagonal and its inverse, lambda_max (smoothed levels) or the dense coarse
// inverses (coarsest level).
int mg_level_branch(pff_ctx* c, int l) {
  LevelData& L = c->lv[l];
  if (l > 0) CR(qp_setup_level(c, l));
  if (c->prm.mg_precision == 32) {
    // the FP32 multigrid's Jacobi scaling, computed in FP32 from the FP32 per-point data
    CK(launch_diagonal<float>(c->dim, c->p, c->prm.split, L.qp32, L.flags, L.g, L.t32, L.d32, c->s));
    CK(launch_inv_diag32(L.nd, L.d32, L.di32, c->s));
  } else {
    CK(launch_diagonal<double>(c->dim, c->p, c->prm.split, L.qp64, L.flags, L.g, L.t64, L.d64, c->s));
    CK(launch_inv_diag(L.nd, L.d64, L.di64, L.di32, c->s));
  }
  if (l < c->nlev - 1) {
    if (c->prm.mg_precision == 32) CR(eig_estimate<float>(c, l));
    else CR(eig_estimate<double>(c, l));
  } else {
    // coarse level: dense blocks and their inverses (block forward substitution, Sec. 3.3)
    const int nn = (int)L.nn, nu = c->dim * nn;
    CK(launch_coarse_assemble(c->dim, c->p, c->prm.split, L.qp64, L.flags, L.g, L.t64, c->Au, c->Ap, c->Bc, c->s));
    if (coarse32(c)) {
      // FP32 coarse solve (non-default, coarse_precision 32): FP32 copies of the blocks inverted in FP32
      CK(launch_cast<double, float>((long long)nu * nu, c->Au, c->Au32, c->s));
      CK(launch_cast<double, float>((long long)nn * nn, c->Ap, c->Ap32, c->s));
      CK(launch_cast<double, float>((long long)nn * nu, c->Bc, c->Bc32, c->s));
      CK(launch_gj_inverse<float>(c->Au32, nu, c->gjbuf32, c->s));
      CK(launch_gj_inverse<float>(c->Ap32, nn, c->gjbuf32 + gj_buffer_size(nu), c->s));
    } else {
      CK(launch_gj_inverse<double>(c->Au, nu, c->gjbuf, c->s));
      CK(launch_gj_inverse<double>(c->Ap, nn, c->gjbuf + gj_buffer_size(nu), c->s));
    }
  }
  return PFF_OK;
}

// Every launch of the multigrid setup of one Newton state (no host synchronisation inside): the
// state is carried down the levels in sequence, then every level's branch runs on its own stream
// (forked from and joined back into the context's stream with events, which a graph capture turns
// into parallel branches).
int mg_build(pff_ctx* c) {
  const int nf_state = c->dim + 2;  // U (dim+1 fields) and phi~ are contiguous
  for (int l = 1; l < c->nlev; ++l) {
    LevelData &F = c->lv[l - 1], &L = c->lv[l];
    CK(launch_state_interp(c->dim, c->p, F.U, L.U, nf_state, F.g, L.g, c->xt, c->s));
    if (c->has_fields) CK(launch_state_interp(c->dim, c->p, F.fields, L.fields, 3, F.g, L.g, c->xt, c->s));
    CK(launch_coarse_active(c->dim, c->p, F.flags, L.flags, F.g, L.g, c->xt, c->s));
  }
  CK(cudaEventRecord(c->fork, c->s));
  const cudaStream_t main_s = c->s;
  int st = PFF_OK;
  for (int l = 0; l < c->nlev && st == PFF_OK; ++l) {
    LevelData& L = c->lv[l];
    if (cudaStreamWaitEvent(L.aux, c->fork, 0) != cudaSuccess) {
      st = PFF_ERR_CUDA;
      break;
    }
    c->s = L.aux;
    st = mg_level_branch(c, l);
    c->s = main_s;
    if (st == PFF_OK && cudaEventRecord(L.join, L.aux) != cudaSuccess) st = PFF_ERR_CUDA;
  }
  c->s = main_s;
  CR(st);
  for (int l = 0; l < c->nlev; ++l) CK(cudaStreamWaitEvent(c->s, c->lv[l].join, 0));
  return PFF_OK;
}

// Captures fn into a CUDA graph on the private stream and instantiates it into *exec.
template <class F>
int capture_graph(pff_ctx* c, cudaGraphExec_t* exec, std::pair<int, int>* range, long long* kernels, F fn) {
  cudaStream_t user = c->s;
  c->s = c->cap;
  const int ev0 = c->gnext;
  const long long k0 = launch_count();
  cudaError_t e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal);
  c->capturing = true;
  int st = e == cudaSuccess ? fn() : PFF_ERR_CUDA;
  c->capturing = false;
  *range = {ev0, c->gnext - ((c->gnext - ev0) & 1)};
  *kernels = launch_count() - k0;
  add_launches(-*kernels);  // captured, not launched
  cudaGraph_t gr = nullptr;
  if (e == cudaSuccess) {
    const cudaError_t e2 = cudaStreamEndCapture(c->s, &gr);
    if (e2 != cudaSuccess) e = e2;
  }
  c->s = user;
  if (st == PFF_OK && e == cudaSuccess) e = cudaGraphInstantiate(exec, gr, 0);
  if (gr) cudaGraphDestroy(gr);
  if (st != PFF_OK || e != cudaSuccess) {
    cudaGetLastError();
    *exec = nullptr;
    return PFF_ERR_CUDA;
  }
  return PFF_OK;
}

// Multigrid data of the current state. Same warm-up / capture / replay scheme as the V-cycle; one
// graph per "nodal fields present" setting.
int mg_setup(pff_ctx* c) {
  if (!c->has_state) return PFF_ERR_NO_STATE;
  if (c->mg_ready) return PFF_OK;
  CR(ensure_qp(c));
  const int key = c->has_fields ? 1 : 0, pv = c->prof;
  if (!c->use_graph || !c->swarm[key]) {
    CR(mg_build(c));
    c->swarm[key] = true;
  } else {
    std::pair<int, int> rg;
    if (!c->sgraph[key][pv] &&
        capture_graph(c, &c->sgraph[key][pv], &rg, &c->skern[key][pv], [&] { return mg_build(c); }) != PFF_OK) {
      c->use_graph = false;
      CR(mg_build(c));
      c->mg_ready = true;
      c->diag64_ok = c->prm.mg_precision != 32;
      return PFF_OK;
    }
    if (!c->sgraph[key][pv]) return PFF_ERR_CUDA;
    if (c->srange[key][pv].empty() && pv != PFF_PROF_OFF) c->srange[key][pv].push_back(rg);
    CK(cudaGraphLaunch(c->sgraph[key][pv], c->s));
    add_launches(c->skern[key][pv]);
    if (pv != PFF_PROF_OFF)
      for (auto& r : c->srange[key][pv]) c->pending.push_back(r);
  }
  c->mg_ready = true;
  c->diag64_ok = c->prm.mg_precision != 32;
  return PFF_OK;
}

// z = G_c^{-1} r on the coarsest level, in FP64 unless the FP32 multigrid asks for an FP32 coarse solve
// (an FP32 cycle casts its vector to FP64 and back around the FP64 solve):
// z_u = Au^{-1} r_u, z_phi = Ap^{-1} (r_phi - B z_u) (block forward substitution).
template <typename Real>
int coarse_solve_blocks(pff_ctx* c, const Real* Au, const Real* Ap, const Real* Bc, Real* ct, const Real* r, Real* z) {
  LevelData& C = c->lv[c->nlev - 1];
  const int nn = (int)C.nn, nu = c->dim * nn;
  CK(launch_gemv<Real>(Au, nu, nu, r, z, 1.0, 0.0, c->s));
  CK(cudaMemcpyAsync(ct, r + nu, sizeof(Real) * nn, cudaMemcpyDeviceToDevice, c->s));
  CK(launch_gemv<Real>(Bc, nn, nu, z, ct, -1.0, 1.0, c->s));
  CK(launch_gemv<Real>(Ap, nn, nn, ct, z + nu, 1.0, 0.0, c->s));
  return PFF_OK;
}

template <typename Real>
int coarse_solve(pff_ctx* c, const Real* r, Real* z);
template <>
int coarse_solve<double>(pff_ctx* c, const double* r, double* z) {
  if (!coarse32(c)) return coarse_solve_blocks<double>(c, c->Au, c->Ap, c->Bc, c->ct, r, z);
  const long long n = c->lv[c->nlev - 1].nd;
  CK(launch_cast<double, float>(n, r, c->cr32, c->s));
  CR(coarse_solve_blocks<float>(c, c->Au32, c->Ap32, c->Bc32, c->ct32, c->cr32, c->ce32));
  CK(launch_cast<float, double>(n, c->ce32, z, c->s));
  return PFF_OK;
}
template <>
int coarse_solve<float>(pff_ctx* c, const float* r, float* z) {
  if (coarse32(c)) return coarse_solve_blocks<float>(c, c->Au32, c->Ap32, c->Bc32, c->ct32, r, z);
  const long long n = c->lv[c->nlev - 1].nd;
  CK(launch_cast<float, double>(n, r, c->cr, c->s));
  CR(coarse_solve_blocks<double>(c, c->Au, c->Ap, c->Bc, c->ct, c->cr, c->ce));
  CK(launch_cast<double, float>(n, c->ce, z, c->s));
  return PFF_OK;
}

// x = S f: block-diagonal Chebyshev-Jacobi of degree cheb_degree with zero initial guess.
// started: the first step (x = d = dinv f / theta) was already done by the kernel that produced f.
// acc: add S f to acc instead (x is then scratch).
template <typename Real>
ChebStart<Real> cheb_start(pff_ctx* c, int l, Real* x, Real* dv) {
  LevelData& L = c->lv[l];
  ChebStart<Real> cs{};
  cs.d = dv;
  cs.x = x;
  cs.dinv = dinv_of<Real>(L);
  cs.inv_lam = inv_lam_of<Real>(L);
  cs.c0s = 2.0 / (c->prm.cheb_hi + c->prm.cheb_lo);
  cs.nu = c->dim * L.nn;
  cs.on = 1;
  return cs;
}

template <typename Real>
int smooth(pff_ctx* c, int l, const Real* f, Real* x, Real* t, Real* dv, bool started = false,
           Real* acc = nullptr) {
  LevelData& L = c->lv[l];
  const long long n = L.nd, nu = c->dim * L.nn;
  const double lo = c->prm.cheb_lo, hi = c->prm.cheb_hi;
  const double sigma = (hi + lo) / (hi - lo);
  double rho = 1.0 / sigma;
  const Real* il = inv_lam_of<Real>(L);
  const int deg = c->prm.cheb_degree;
  // theta_b = (hi + lo) lambda_b / 2, delta_b = (hi - lo) lambda_b / 2
  if (!started) CK(launch_cheb<Real>(0, n, nu, f, nullptr, dinv_of<Real>(L), dv, x, il, 2.0 / (hi + lo), 0.0, 0.0, c->s));
  bool added = false;
  if (c->dim == 2 && deg > 1) {
    // Steps 1 .. K fused into the block-diagonal apply. Step k reads x_k from X[k % 2] and d_{k-1} from
    // D[(k-1) % 2] and writes x_{k+1}, d_k to the other buffers on the nodes of a single tile; its seam
    // sums go to T[k % 3], and step k+1 finishes step k on the seam nodes while it stages its patch
    // (ChebEpi). Only the last step's seam nodes take a separate launch. Every T buffer is all zero on
    // entry and again on exit.
    CR(ensure_work<Real>(c, l));
    Real** w = work_of<Real>(L);
    Real* X[2] = {w[6], x};
    Real* D[2] = {dv, w[7]};
    Real* T[3] = {w[8], t, w[9]};
    const int K = deg - 1;
    double c1p = 0.0, c2sp = 0.0;
    for (int k = 1; k <= K; ++k) {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      ChebEpi<Real> ce{};
      ce.f = f;
      ce.dinv = dinv_of<Real>(L);
      ce.inv_lam = il;
      ce.x = X[k % 2];
      ce.x_out = X[(k + 1) % 2];
      ce.d = D[(k - 1) % 2];
      ce.d_out = D[k % 2];
      ce.c1 = rho_new * rho;
      ce.c2s = 4.0 * rho_new / (hi - lo);
      ce.acc = (acc && k == K) ? acc : nullptr;
      ce.on = 1;
      ce.pp = k >= 2;
      ce.tp = T[(k - 1) % 3];
      ce.tz = k >= 3 ? T[(k - 2) % 3] : nullptr;
      ce.c1p = c1p;
      ce.c2sp = c2sp;
      CR(apply_level<Real>(c, l, X[k % 2], T[k % 3], JM_BLOCKDIAG, IN_ALL, OUT_IDENTITY, &ce, true));
      if (k == K) {
        ce.tz = T[(K - 1) % 3];  // no later step reads the previous seam sums
        CK(launch_cheb_seam<Real>(L.g, T[K % 3], ce, c->s));
      }
      c1p = ce.c1;
      c2sp = ce.c2s;
      rho = rho_new;
    }
    added = acc != nullptr;
    // x_{K+1} is in X[(K + 1) % 2]; the caller's buffer is X[1]
    if (!acc && (K + 1) % 2 != 1) CK(cudaMemcpyAsync(x, X[0], sizeof(Real) * n, cudaMemcpyDeviceToDevice, c->s));
  }
  for (int k = 1; k < deg && c->dim != 2; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    {
      CR(apply_level<Real>(c, l, x, t, JM_BLOCKDIAG, IN_ALL, OUT_IDENTITY));
      CK(launch_cheb<Real>(k, n, nu, f, t, dinv_of<Real>(L), dv, x, il, 0.0, rho_new * rho, 4.0 * rho_new / (hi - lo),
                           c->s));
    }
    rho = rho_new;
  }
  if (acc && !added) CK(launch_axpby<Real>(n, 1.0, x, 1.0, acc, c->s));
  return PFF_OK;
}

// e = V-cycle(r) from level l down (Sec. 3.3): pre-smooth, residual, restrict, recurse,
// prolongate, post-smooth on the residual.
template <typename Real>
int vcycle_level(pff_ctx* c, int l, const Real* r, Real* e) {
  if (l == c->nlev - 1) return coarse_solve<Real>(c, r, e);
  CR(ensure_work<Real>(c, l));
  CR(ensure_work<Real>(c, l + 1));
  LevelData &L = c->lv[l], &Lc = c->lv[l + 1];
  Real** w = work_of<Real>(L);
  Real** wc = work_of<Real>(Lc);
  Real *t = w[2], *res = w[3], *dv = w[4], *sx = w[5];
  const bool zt = c->dim == 2;  // in 2D the apply buffer t is kept zeroed between uses
  ChebStart<Real> off{};
  off.on = 0;
  // pre-smoothing; below the finest level its first step was done by the restriction
  CR(smooth<Real>(c, l, r, e, t, dv, l > 0));
  CR(apply_level<Real>(c, l, e, t, JM_FULL, IN_ALL, OUT_IDENTITY, nullptr, zt));
  CK(launch_res_update<Real>(L.nd, r, t, res, off, c->s));
  // res is zero on masked fine rows (r is, and G has identity rows there with e = 0): no Z_f needed
  const bool coarsest = l + 1 == c->nlev - 1;
  const ChebStart<Real> csc = coarsest ? off : cheb_start<Real>(c, l + 1, wc[1], wc[4]);
  CK(launch_restrict<Real>(c->dim, c->p, res, wc[0], L.flags, Lc.flags, L.g, Lc.g, c->xt, c->s, false, &csc));
  CR(vcycle_level<Real>(c, l + 1, wc[0], wc[1]));
  CK(launch_prolong<Real>(c->dim, c->p, wc[1], e, L.flags, Lc.g, L.g, c->xt, true, c->s));
  CR(apply_level<Real>(c, l, e, t, JM_FULL, IN_ALL, OUT_IDENTITY, nullptr, zt));
  // post-smoothing on the new residual, started by the residual update and added into e
  CK(launch_res_update<Real>(L.nd, r, t, res, cheb_start<Real>(c, l, sx, dv), c->s));
  CR(smooth<Real>(c, l, res, sx, t, dv, true, e));
  return PFF_OK;
}

// V-cycle from the level-0 work vector r (w[0]) into e (w[1]). The first call per precision runs
// eagerly (it allocates work vectors and sets kernel attributes); the second captures the cycle
// into a CUDA graph on a private stream; later calls replay the graph on the caller's stream. While
// a kernel family is being timed the cycle runs eagerly so that every launch is timed.
template <typename Real>
int vcycle_exec(pff_ctx* c) {
  Real** w = work_of<Real>(c->lv[0]);
  const int gi = sizeof(Real) == 8 ? 0 : 1, pv = c->prof;
  if (!c->use_graph || !c->vwarm[gi]) {
    CR(vcycle_level<Real>(c, 0, w[0], w[1]));
    c->vwarm[gi] = true;
    return PFF_OK;
  }
  std::pair<int, int> rg;
  if (!c->vgraph[gi][pv] &&
      capture_graph(c, &c->vgraph[gi][pv], &rg, &c->vkern[gi][pv],
                    [&] { return vcycle_level<Real>(c, 0, w[0], w[1]); }) != PFF_OK) {
    c->use_graph = false;
    return vcycle_level<Real>(c, 0, w[0], w[1]);
  }
  if (c->vrange[gi][pv].empty() && pv != PFF_PROF_OFF) c->vrange[gi][pv].push_back(rg);
  CK(cudaGraphLaunch(c->vgraph[gi][pv], c->s));
  add_launches(c->vkern[gi][pv]);
  if (pv != PFF_PROF_OFF)
    for (auto& r : c->vrange[gi][pv]) c->pending.push_back(r);
  return PFF_OK;
}

// FP64 in/out; inside in mg_precision.
int precondition(pff_ctx* c, const double* r, double* z) {
  CR(mg_setup(c));
  LevelData& L = c->lv[0];
  if (c->prm.mg_precision == 32) {
    CR(ensure_work<float>(c, 0));
    // FGMRES writes the FP32 copy of its next basis vector when it normalises it
    if (c->w32_of != r) CK(launch_cast<double, float>(L.nd, r, L.w32[0], c->s));
    c->w32_of = nullptr;
    CR(vcycle_exec<float>(c));
    CK(launch_cast<float, double>(L.nd, L.w32[1], z, c->s));
  } else {
    CR(ensure_work<double>(c, 0));
    CK(cudaMemcpyAsync(L.w64[0], r, sizeof(double) * L.nd, cudaMemcpyDeviceToDevice, c->s));
    CR(vcycle_exec<double>(c));
    CK(cudaMemcpyAsync(z, L.w64[1], sizeof(double) * L.nd, cudaMemcpyDeviceToDevice, c->s));
  }
  return PFF_OK;
}

// ||x||^2 over both blocks, synchronising (host result).
int norm2_host(pff_ctx* c, const double* x, long long n, double* out) {
  CK(launch_dot2<double>(n, n, x, x, c->partial, c->dres, c->s));
  CK(cudaMemcpyAsync(c->pinned, c->dres, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  CR(prof_collect(c));
  *out = c->pinned[0] + c->pinned[1];
  return PFF_OK;
}

// Right-preconditioned flexible GMRES(m), x0 = 0, CGS2 orthogonalisation in FP64.
int fgmres(pff_ctx* c, const double* b, double* x, int* iters_out, double* rel_out) {
  CR(mg_setup(c));
  c->w32_of = nullptr;
  LevelData& L = c->lv[0];
  const long long n = L.nd;
  const int m = c->prm.gmres_restart;
  const double tol = c->prm.lin_rtol;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, c->s));
  double b2;
  CR(norm2_host(c, b, n, &b2));
  if (!std::isfinite(b2)) return PFF_ERR_NAN;
  const double beta0 = std::sqrt(b2);
  if (iters_out) *iters_out = 0;
  if (rel_out) *rel_out = 0.0;
  if (beta0 == 0.0) return PFF_OK;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  int its = 0;
  double rel = 1.0;
  int status = PFF_OK;
  double* r = c->w;  // residual of the current cycle
  bool first = true;
  while (true) {
    if (first) {
      CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->s));
    } else {
      CR(apply_level<double>(c, 0, x, r, JM_FULL, IN_ALL, OUT_IDENTITY));
      CK(launch_axpby<double>(n, 1.0, b, -1.0, r, c->s));
    }
    first = false;
    double r2;
    CR(norm2_host(c, r, n, &r2));
    const double beta = std::sqrt(r2);
    rel = beta / beta0;
    if (!std::isfinite(beta)) return PFF_ERR_NAN;
    if (rel <= tol || its >= c->prm.gmres_max_iters) break;
    CK(launch_axpby<double>(n, 1.0 / beta, r, 0.0, c->V, c->s));
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    bool stop = false;
    for (int j = 0; j < m; ++j) {
      double* Vj = c->V + (long long)j * n;
      double* Zj = c->Z + (long long)j * n;
      double* wv = c->V + (long long)(j + 1) * n;
      CR(precondition(c, Vj, Zj));
      CR(apply_level<double>(c, 0, Zj, wv, JM_FULL, IN_ALL, OUT_IDENTITY));
      // CGS2: hdev = (h1 [m + 1], h2 [m + 1], <w, w>, 0, 1 / |w|)
      CK(launch_cgs2(n, j + 1, c->V, wv, c->partial, c->hdev, c->hdev + (m + 1), c->hdev + 2 * (m + 1), c->kcnt,
                     c->s));
      CK(cudaMemcpyAsync(c->pinned, c->hdev, sizeof(double) * (2 * (m + 1) + 2), cudaMemcpyDeviceToHost, c->s));
      CK(cudaEventRecord(c->hcol, c->s));
      // V_{j+1} = w / |w| on the device (1/|w| from the CGS2 pass, 0 for w = 0), with the FP32 copy the
      // next V-cycle starts from, while the host waits for the column and applies the rotations (after
      // the last iteration this is one small kernel for nothing)
      float* w32 = nullptr;
      if (c->prm.mg_precision == 32) {
        CR(ensure_work<float>(c, 0));
        w32 = L.w32[0];
      }
      CK(launch_normalize(n, wv, c->hdev + 2 * (m + 1) + 2, wv, w32, c->s));
      c->w32_of = w32 ? wv : nullptr;
      CK(cudaEventSynchronize(c->hcol));
      CR(prof_collect(c));
      const double* hh = c->pinned;
      for (int i = 0; i <= j; ++i) H[i * m + j] = hh[i] + hh[(m + 1) + i];
      const double nw2 = hh[2 * (m + 1)] + hh[2 * (m + 1) + 1];
      if (!std::isfinite(nw2)) return PFF_ERR_NAN;
      const double nw = std::sqrt(nw2);
      H[(j + 1) * m + j] = nw;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      const double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      if (den == 0.0) {
        status = PFF_ERR_BREAKDOWN;
        stop = true;
        break;
      }
      cs[j] = H[j * m + j] / den;
      sn[j] = H[(j + 1) * m + j] / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      k = j + 1;
      ++its;
      rel = std::fabs(gv[j + 1]) / beta0;
      if (rel <= tol || its >= c->prm.gmres_max_iters || nw == 0.0) {
        stop = true;
        break;
      }
    }
    if (k > 0) {
      for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int jj = i + 1; jj < k; ++jj) s -= H[i * m + jj] * y[jj];
        y[i] = s / H[i * m + i];
      }
      std::memcpy(c->pinned, y.data(), sizeof(double) * k);
      CK(cudaMemcpyAsync(c->ydev, c->pinned, sizeof(double) * k, cudaMemcpyHostToDevice, c->s));
      CK(launch_zupdate(n, k, c->Z, c->ydev, x, c->s));
      CK(cudaStreamSynchronize(c->s));
    }
    if (stop && status != PFF_OK) break;
    if (stop && its >= c->prm.gmres_max_iters) {
      // final true residual below
    }
    if (stop && rel > tol && its < c->prm.gmres_max_iters) continue;
    if (stop) {
      // verify with the true residual
      CR(apply_level<double>(c, 0, x, r, JM_FULL, IN_ALL, OUT_IDENTITY));
      CK(launch_axpby<double>(n, 1.0, b, -1.0, r, c->s));
      double rr;
      CR(norm2_host(c, r, n, &rr));
      rel = std::sqrt(rr) / beta0;
      break;
    }
  }
  if (iters_out) *iters_out = its;
  if (rel_out) *rel_out = rel;
  if (status != PFF_OK) return status;
  if (rel > tol) return PFF_ERR_NOT_CONVERGED;
  return PFF_OK;
}

bool valid_prec(int p) { return p == 32 || p == 64; }

}  // namespace

// =============================================================================================
// C-ABI
extern "C" {

void pff_default_params(pff_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dim = 2;
  p->degree = 1;
  p->n_cells_1d = 32;
  p->coarse_min = 3;
  p->split = PFF_SPLIT_NONE;
  p->lambda = 121.15;
  p->mu = 80.77;
  p->gc = 2.7e-3;
  p->eps = 2.0 / 32;
  p->kappa = 1e-10;
  p->as_c = 1.0;
  p->mg_precision = 32;
  p->coarse_precision = 64;
  p->slit_cut = 0;
  p->fp32_tangent = 0;
  p->cheb_degree = 5;
  p->cheb_lo = 0.24;
  p->cheb_hi = 1.2;
  p->eig_iters = 15;
  p->eig_seed = 0;
  p->gmres_restart = 50;
  p->gmres_max_iters = 500;
  p->lin_rtol = 1e-6;
  p->fp64_mode = 0;
}

const char* pff_strerror(int st) {
  switch (st) {
    case PFF_OK: return "ok";
    case PFF_ERR_INVALID_ARG: return "invalid argument";
    case PFF_ERR_OOM: return "out of device memory";
    case PFF_ERR_CUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case PFF_ERR_NAN: return "non-finite value";
    case PFF_ERR_NOT_CONVERGED: return "linear solver did not converge";
    case PFF_ERR_BREAKDOWN: return "Krylov breakdown";
    case PFF_ERR_NO_STATE: return "no state set";
    case PFF_ERR_TOO_LARGE: return "problem too large for this entry point (allocation-free scratch or 32-bit CSR indices)";
    case PFF_ERR_UNAVAILABLE: return "an optional library (cuSPARSE) could not be loaded";
    default: return "unknown status";
  }
}

void pff_destroy(pff_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (auto& row : c->vgraph)
    for (cudaGraphExec_t g : row)
      if (g) cudaGraphExecDestroy(g);
  for (auto& row : c->sgraph)
    for (cudaGraphExec_t g : row)
      if (g) cudaGraphExecDestroy(g);
  for (cudaEvent_t e : c->gev) cudaEventDestroy(e);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->hcol) cudaEventDestroy(c->hcol);
  for (auto& L : c->lv) {
    if (L.aux) cudaStreamDestroy(L.aux);
    if (L.join) cudaEventDestroy(L.join);
  }
  csr_destroy(c->csr);
  for (void* q : c->allocs) cudaFree(q);
  if (c->pinned) cudaFreeHost(c->pinned);
  delete c;
}

static int setup_impl(pff_ctx* c) {
  const pff_params& P = c->prm;
  CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
  c->dim = P.dim;
  c->p = P.degree;
  std::vector<int> sizes{P.n_cells_1d};
  while (sizes.back() % 2 == 0 && sizes.back() / 2 >= P.coarse_min) sizes.push_back(sizes.back() / 2);
  c->nlev = (int)sizes.size();
  c->lv.resize(c->nlev);
  make_xfer(c->xt, c->p);
  for (int l = 0; l < c->nlev; ++l) {
    LevelData& L = c->lv[l];
    L.N = sizes[l];
    L.h = 1.0 / L.N;
    long long n1 = (long long)c->p * L.N + 1;
    const bool cut = l == 0 && c->prm.slit_cut;  // coarse levels keep one node per grid point
    L.nn = (c->dim == 2 ? n1 * n1 : n1 * n1 * n1) + (cut ? cut_copies(c->dim, c->p, L.N) : 0);
    L.nd = (c->dim + 1) * L.nn;
    make_geom(L, c->dim, c->p, cut);
    make_tabs(L, c->dim, c->p);
    const int nv = qp_nv(c->dim, P.split);
    CR(dalloc(c, &L.flags, L.nn, l));
    CR(dalloc(c, &L.U, L.nd + L.nn, l));  // U and phi~ contiguous
    L.phit = L.U + L.nd;
    CR(dalloc(c, &L.fields, 3 * L.nn, l));
    const long long nqp = L.g.ntiles * L.g.qpt;
    CR(dalloc(c, &L.qp64, nv * nqp, l));
    CR(dalloc(c, &L.qp32, nv * nqp, l));
    CR(dalloc(c, &L.qpdf, nv * nqp, l));
    CK(cudaMemsetAsync(L.qpdf, 0, sizeof(df64) * nv * nqp, c->s));
    CK(cudaMemsetAsync(L.qp64, 0, sizeof(double) * nv * nqp, c->s));
    CK(cudaMemsetAsync(L.qp32, 0, sizeof(float) * nv * nqp, c->s));
    if (l == 0) {
      CR(dalloc(c, &L.st64, ST_NV * nqp, l));
      CK(cudaMemsetAsync(L.st64, 0, sizeof(double) * ST_NV * nqp, c->s));
      if (c->prm.split == 1) {
        const int nm = c->dim == 2 ? 3 : 6;
        CR(dalloc(c, &L.sp64, (nm + 1) * nqp, l));
        CK(cudaMemsetAsync(L.sp64, 0, sizeof(double) * (nm + 1) * nqp, c->s));
      }
    }
    if (c->dim == 2) CR(dalloc(c, &L.s32, (c->dim + 2) * L.nn, l));
    CR(dalloc(c, &L.d64, L.nd, l));
    CR(dalloc(c, &L.di64, L.nd, l));
    CR(dalloc(c, &L.d32, L.nd, l));
    CR(dalloc(c, &L.di32, L.nd, l));
    CR(dalloc(c, &L.lam, 8, l));
    CR(dalloc(c, &L.lscal, 16, l));
    CR(dalloc(c, &L.lhist, 4 * P.eig_iters, l));
    CR(dalloc(c, &L.lpart, 2 * 152 * 32, l));  // 2 partial sums per CTA of the CG-Lanczos reductions
    CK(cudaStreamCreateWithFlags(&L.aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&L.join, cudaEventDisableTiming));
    std::vector<unsigned char> fl = host_flags(c->dim, c->p, L.N, cut);
    CK(cudaMemcpyAsync(L.flags, fl.data(), fl.size(), cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
  }
  LevelData& F = c->lv[0];
  CR(dalloc(c, &c->phi_old, F.nn));
  CR(dalloc(c, &c->hist1, F.nn));
  CR(dalloc(c, &c->hist2, F.nn));
  CR(dalloc(c, &c->mass, F.nn));
  CR(dalloc(c, &c->R, F.nd));
  CR(dalloc(c, &c->rhs, F.nd));
  CR(dalloc(c, &c->dU, F.nd));
  CR(dalloc(c, &c->scratch, 4 * F.nd));
  const int m = P.gmres_restart;
  CR(dalloc(c, &c->partial, std::max<long long>(std::max<long long>(2 * 152 * 2, (long long)(m + 2) * 152),
                                                (long long)CGS_KMAX * CGS_GRID_MAX)));
  CR(dalloc(c, &c->kcnt, 1, TAG_KRYLOV));
  CK(cudaMemsetAsync(c->kcnt, 0, sizeof(unsigned), c->s));
  CK(cudaEventCreateWithFlags(&c->hcol, cudaEventDisableTiming));
  CR(dalloc(c, &c->dres, 32));
  CR(dalloc(c, &c->hist, 4 * P.eig_iters));
  CR(dalloc(c, &c->cnt, 2));
  CR(dalloc(c, &c->V, (long long)(m + 1) * F.nd, TAG_KRYLOV));
  CR(dalloc(c, &c->Z, (long long)m * F.nd, TAG_KRYLOV));
  CR(dalloc(c, &c->w, F.nd, TAG_KRYLOV));
  CR(dalloc(c, &c->hdev, 3 * (m + 1) + 4, TAG_KRYLOV));
  CR(dalloc(c, &c->ydev, m + 1, TAG_KRYLOV));
  if (cudaMallocHost(&c->pinned, sizeof(double) * (4 * (m + 2) + 64)) != cudaSuccess) return PFF_ERR_OOM;
  LevelData& C = c->lv[c->nlev - 1];
  const long long nnc = C.nn, nuc = c->dim * C.nn;
  CR(dalloc(c, &c->Au, nuc * nuc, TAG_COARSE));
  CR(dalloc(c, &c->Ap, nnc * nnc, TAG_COARSE));
  CR(dalloc(c, &c->Bc, nnc * nuc, TAG_COARSE));
  if (coarse32(c)) {
    CR(dalloc(c, &c->Au32, nuc * nuc, TAG_COARSE));
    CR(dalloc(c, &c->Ap32, nnc * nnc, TAG_COARSE));
    CR(dalloc(c, &c->Bc32, nnc * nuc, TAG_COARSE));
    CR(dalloc(c, &c->gjbuf32, gj_buffer_size((int)nuc) + gj_buffer_size((int)nnc), TAG_COARSE));
    CR(dalloc(c, &c->cr32, C.nd, TAG_COARSE));
    CR(dalloc(c, &c->ce32, C.nd, TAG_COARSE));
    CR(dalloc(c, &c->ct32, C.nd, TAG_COARSE));
  } else {
    CR(dalloc(c, &c->gjbuf, gj_buffer_size((int)nuc) + gj_buffer_size((int)nnc), TAG_COARSE));
  }
  CR(dalloc(c, &c->cr, C.nd, TAG_COARSE));
  CR(dalloc(c, &c->ce, C.nd, TAG_COARSE));
  CR(dalloc(c, &c->ct, C.nd, TAG_COARSE));
  // lumped phase-field mass: 1D sums of GLL weights times h
  {
    const int n1 = c->p * F.N + 1;
    double wg[MAXN];
    gll_weights(c->p, wg);
    std::vector<double> w1(n1, 0.0);
    for (int cc = 0; cc < F.N; ++cc)
      for (int k = 0; k <= c->p; ++k) w1[cc * c->p + k] += wg[k] * F.h;
    if (!F.g.cut) {
      double* dw1;
      CR(dalloc(c, &dw1, n1));
      CK(cudaMemcpyAsync(dw1, w1.data(), sizeof(double) * n1, cudaMemcpyHostToDevice, c->s));
      CK(launch_lumped_mass(c->dim, F.nn, n1, dw1, c->mass, c->s));
    } else {
      // cut slit: the slit's grid nodes see only the cells above it, their copies only those below;
      // GLL weights are symmetric, so each side carries half the tensor-product weight
      std::vector<double> m(F.nn);
      const long long ng = F.g.ngrid;
      for (long long i = 0; i < ng; ++i) {
        long long rem = i;
        double v = 1.0;
        int ijk[3] = {0, 0, 0};
        for (int t = 0; t < c->dim; ++t) {
          ijk[t] = int(rem % n1);
          v *= w1[ijk[t]];
          rem /= n1;
        }
        if (ijk[c->dim - 1] == F.g.cut_row && ijk[0] < F.g.cut_x) v *= 0.5;
        m[i] = v;
      }
      const long long ny = c->dim == 2 ? 1 : n1;
      for (long long y = 0; y < ny; ++y)
        for (int x = 0; x < F.g.cut_x; ++x)
          m[cut_copy(F.g, x, (int)y)] = m[x + (long long)n1 * (c->dim == 2 ? F.g.cut_row : y + (long long)n1 * F.g.cut_row)];
      CK(cudaMemcpyAsync(c->mass, m.data(), sizeof(double) * F.nn, cudaMemcpyHostToDevice, c->s));
    }
    CK(cudaStreamSynchronize(c->s));
  }
  return PFF_OK;
}

int pff_setup_mesh(pff_ctx** out, const pff_params* p, void* stream) {
  if (!out || !p) return PFF_ERR_INVALID_ARG;
  *out = nullptr;
  if ((p->dim != 2 && p->dim != 3) || p->degree < 1 || p->degree > MAXP || p->n_cells_1d < 1 ||
      p->coarse_min < 1 || (p->split != PFF_SPLIT_NONE && p->split != PFF_SPLIT_MIEHE) ||
      !valid_prec(p->mg_precision) || p->cheb_degree < 1 || !(p->cheb_hi > p->cheb_lo) || !(p->cheb_lo > 0) ||
      p->eig_iters < 1 || p->eig_iters > 64 || p->gmres_restart < 1 || p->gmres_max_iters < 1 ||
      !(p->lin_rtol > 0) || !(p->eps > 0) || (p->fp64_mode != 0 && p->fp64_mode != 1) ||
      !valid_prec(p->coarse_precision) || (p->slit_cut != 0 && p->slit_cut != 1) ||
      (p->fp32_tangent != 0 && p->fp32_tangent != 1))
    return PFF_ERR_INVALID_ARG;
  if (p->slit_cut) {  // the slit must lie on a boundary between tile rows of the finest mesh
    int t[3];
    tile_shape(p->dim, p->degree, t);
    if (p->n_cells_1d % 2 || (p->n_cells_1d / 2) % t[p->dim - 1]) return PFF_ERR_INVALID_ARG;
  }
  {  // the operator kernels index DoFs (field-major node arrays) with 32-bit integers
    const double n1 = (double)p->degree * p->n_cells_1d + 1.0;  // in double: no integer overflow
    const double nodes = p->dim == 2 ? n1 * n1 + n1 : n1 * n1 * n1 + n1 * n1;
    if ((p->dim + 1) * nodes > 2147483647.0) return PFF_ERR_TOO_LARGE;
  }
  pff_ctx* c = new (std::nothrow) pff_ctx();
  if (!c) return PFF_ERR_OOM;
  c->prm = *p;
  c->s = static_cast<cudaStream_t>(stream);
  if (cudaStreamGetDevice(c->s, &c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return PFF_ERR_CUDA;
  }
  const int st = setup_impl(c);
  if (st != PFF_OK) {
    pff_destroy(c);
    return st;
  }
  *out = c;
  return PFF_OK;
}

int pff_sizes(const pff_ctx* c, long long* n_dofs, long long* n_nodes, int* n_levels) {
  if (!c) return PFF_ERR_INVALID_ARG;
  if (n_dofs) *n_dofs = c->lv[0].nd;
  if (n_nodes) *n_nodes = c->lv[0].nn;
  if (n_levels) *n_levels = c->nlev;
  return PFF_OK;
}

int pff_level_sizes(const pff_ctx* c, int level, long long* n_nodes, int* n_cells_1d) {
  if (!c || level < 0 || level >= c->nlev) return PFF_ERR_INVALID_ARG;
  if (n_nodes) *n_nodes = c->lv[level].nn;
  if (n_cells_1d) *n_cells_1d = c->lv[level].N;
  return PFF_OK;
}

int pff_node_flags(pff_ctx* c, int level, unsigned char* flags) {
  if (!c || !flags || level < 0 || level >= c->nlev) return PFF_ERR_INVALID_ARG;
  if (level > 0 && c->has_state) CR(mg_setup(c));
  CK(cudaMemcpyAsync(flags, c->lv[level].flags, c->lv[level].nn, cudaMemcpyDeviceToDevice, c->s));
  return PFF_OK;
}

int pff_set_state(pff_ctx* c, const double* U, const double* phi_old, const double* phi_tilde,
                  const unsigned char* active, const double* gc_field, const double* lambda_field,
                  const double* mu_field) {
  Range nvtx_range("pff_set_state");
  if (!c || !U || !phi_old) return PFF_ERR_INVALID_ARG;
  LevelData& L = c->lv[0];
  CK(cudaMemcpyAsync(L.U, U, sizeof(double) * L.nd, cudaMemcpyDeviceToDevice, c->s));
  CK(cudaMemcpyAsync(c->phi_old, phi_old, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, c->s));
  CK(cudaMemcpyAsync(L.phit, phi_tilde ? phi_tilde : phi_old, sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, c->s));
  c->has_fields = gc_field || lambda_field || mu_field;
  if (c->has_fields) {
    // missing fields of a partial set take the constants
    const double* src[3] = {gc_field, lambda_field, mu_field};
    const double cst[3] = {c->prm.gc, c->prm.lambda, c->prm.mu};
    for (int k = 0; k < 3; ++k) {
      if (src[k]) {
        CK(cudaMemcpyAsync(L.fields + k * L.nn, src[k], sizeof(double) * L.nn, cudaMemcpyDeviceToDevice, c->s));
      } else {
        std::vector<double> h(L.nn, cst[k]);
        CK(cudaMemcpyAsync(L.fields + k * L.nn, h.data(), sizeof(double) * L.nn, cudaMemcpyHostToDevice, c->s));
        CK(cudaStreamSynchronize(c->s));
      }
    }
  }
  c->has_state = true;
  c->qp_valid = false;
  c->st_valid = false;
  c->strain_valid = false;
  c->mg_ready = false;
  c->nhist = 0;
  c->fresh_active = false;
  if (active) {
    CK(launch_set_active(c->dim, L.nn, active, L.flags, c->s));
  } else {
    unsigned char* dz = reinterpret_cast<unsigned char*>(c->scratch);
    CK(cudaMemsetAsync(dz, 0, L.nn, c->s));
    CK(launch_set_active(c->dim, L.nn, dz, L.flags, c->s));
    CR(residual_into(c, c->R));
    CK(launch_active_set(c->dim, L.nn, c->R, c->mass, c->phi_old, c->prm.as_c, L.U, L.flags, c->cnt, c->s));
    c->qp_valid = false;
    // this is the first step of Alg. 1 at U: the next Newton step starts from it
    c->fresh_active = true;
  }
  return PFF_OK;
}

int pff_get_state(pff_ctx* c, double* U_out) {
  if (!c || !U_out) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  CK(cudaMemcpyAsync(U_out, c->lv[0].U, sizeof(double) * c->lv[0].nd, cudaMemcpyDeviceToDevice, c->s));
  return PFF_OK;
}

int pff_get_active(pff_ctx* c, unsigned char* a) {
  if (!c || !a) return PFF_ERR_INVALID_ARG;
  CK(launch_get_active(c->dim, c->lv[0].nn, c->lv[0].flags, a, c->s));
  return PFF_OK;
}

int pff_apply_jacobian(pff_ctx* c, int level, const void* x, void* y, int precision, int mode) {
  Range nvtx_range("pff_apply_jacobian");
  if (!c || !x || !y || level < 0 || level >= c->nlev || !valid_prec(precision) || x == y) return PFF_ERR_INVALID_ARG;
  const int jm = mode & 3;
  if (jm > 2 || (mode & ~15) || ((mode & PFF_MASK_RAW) && (mode & PFF_MASK_ADJOINT))) return PFF_ERR_INVALID_ARG;
  CR(ensure_qp(c));
  if (level > 0) CR(mg_setup(c));
  int inm = IN_ALL, outm = OUT_IDENTITY;
  if (mode & PFF_MASK_RAW) {
    inm = IN_RAW;
    outm = OUT_RAW;
  } else if (mode & PFF_MASK_ADJOINT) {
    inm = IN_DIRICHLET;
    outm = OUT_RAW;
  }
  if (precision == 64)
    return apply_level<double>(c, level, static_cast<const double*>(x), static_cast<double*>(y), jm, inm, outm);
  return apply_level<float>(c, level, static_cast<const float*>(x), static_cast<float*>(y), jm, inm, outm);
}

int pff_residual(pff_ctx* c, double* r) {
  Range nvtx_range("pff_residual");
  if (!c || !r) return PFF_ERR_INVALID_ARG;
  return residual_into(c, r);
}

int pff_reaction_force(pff_ctx* c, double* force) {
  Range nvtx_range("pff_reaction_force");
  if (!c || !force) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  LevelData& L = c->lv[0];
  double* r = c->scratch;  // the full residual, Dirichlet rows kept
  CR(residual_into(c, r, OUT_RAW));
  // the top face (last coordinate index n1 - 1) is the last n1^(dim-1) nodes of the lexicographic order
  const long long nface = c->dim == 2 ? (long long)L.g.n1 : (long long)L.g.n1 * L.g.n1;
  std::vector<double> h((size_t)nface);
  CK(cudaMemcpyAsync(h.data(), r + (long long)load_comp(c) * L.nn + (L.nn - nface), sizeof(double) * nface,
                     cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  double f = 0.0;
  for (double v : h) f += v;
  *force = f;
  return PFF_OK;
}

int pff_csr_pattern(int dim, int degree, int n_cells_1d, const unsigned char* flags, int* rowptr, int* col,
                    long long* nnz) {
  if ((dim != 2 && dim != 3) || degree < 1 || degree > 4 || n_cells_1d < 1 || !flags || !nnz)
    return PFF_ERR_INVALID_ARG;
  std::vector<int> rp, cl;
  if (!csr_pattern(dim, degree, n_cells_1d, flags, rp, cl)) return PFF_ERR_TOO_LARGE;
  *nnz = (long long)cl.size();
  if (rowptr) std::memcpy(rowptr, rp.data(), sizeof(int) * rp.size());
  if (col) std::memcpy(col, cl.data(), sizeof(int) * cl.size());
  return PFF_OK;
}

int pff_csr_probe_targets(int dim, int degree, int n_cells_1d, int f, int color, long long* targets) {
  const int m = 2 * degree + 1;
  if ((dim != 2 && dim != 3) || degree < 1 || degree > 4 || n_cells_1d < 1 || f < 0 || f > dim || !targets ||
      color < 0 || color >= (dim == 2 ? m * m : m * m * m))
    return PFF_ERR_INVALID_ARG;
  const int n1 = degree * n_cells_1d + 1;
  const long long nn = dim == 2 ? (long long)n1 * n1 : (long long)n1 * n1 * n1;
  for (long long r = 0; r < (dim + 1) * nn; ++r) targets[r] = probe_target(r, nn, n1, dim, degree, f, color);
  return PFF_OK;
}

int pff_csr_assemble(pff_ctx* c, long long* nnz) {
  Range nvtx_range("pff_csr_assemble");
  if (!c || c->prm.slit_cut) return PFF_ERR_INVALID_ARG;  // its pattern assumes one node per grid point
  if (!c->has_state) return PFF_ERR_NO_STATE;
  CR(ensure_qp(c));
  LevelData& L = c->lv[0];
  std::vector<unsigned char> fl((size_t)L.nn);
  CK(cudaMemcpyAsync(fl.data(), L.flags, (size_t)L.nn, cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  std::vector<int> rowptr, col;
  if (!csr_pattern(c->dim, c->p, L.N, fl.data(), rowptr, col)) return PFF_ERR_TOO_LARGE;
  csr_destroy(c->csr);
  c->csr = nullptr;
  CR(csr_create(&c->csr, L.nd, rowptr, col, c->s));
  // probe the native-FP64 operator of the linear solve with one coloured vector per (component, colour)
  double* x = c->scratch;
  double* y = c->scratch + L.nd;
  const int m = 2 * c->p + 1, ncolor = c->dim == 2 ? m * m : m * m * m;
  for (int f = 0; f <= c->dim; ++f) {
    for (int color = 0; color < ncolor; ++color) {
      CK(launch_probe_set(c->dim, c->p, L.nn, L.g.n1, f, color, x, c->s));
      CK(cudaMemsetAsync(y, 0, sizeof(double) * L.nd, c->s));
      CK(launch_jac(c->dim, c->p, c->prm.split, static_cast<const double*>(x), y, L.flags, L.g, L.t64, L.qp64,
                    JM_FULL, IN_ALL, OUT_IDENTITY, c->s));
      CK(launch_probe_gather(c->csr, c->dim, c->p, L.nn, L.g.n1, f, color, y, c->s));
    }
  }
  CK(cudaStreamSynchronize(c->s));
  if (nnz) *nnz = csr_nnz(c->csr);
  return PFF_OK;
}

int pff_csr_spmv_available(void) { return csr_spmv_available() ? 1 : 0; }

int pff_csr_spmv(pff_ctx* c, const double* x, double* y) {
  Range nvtx_range("pff_csr_spmv");
  if (!c || !x || !y || x == y) return PFF_ERR_INVALID_ARG;
  if (!c->csr) return PFF_ERR_NO_STATE;
  return csr_spmv(c->csr, x, y, c->s);
}

int pff_csr_export(pff_ctx* c, int* rowptr, int* col, double* val) {
  if (!c) return PFF_ERR_INVALID_ARG;
  if (!c->csr) return PFF_ERR_NO_STATE;
  const long long nr = c->lv[0].nd + 1, nz = csr_nnz(c->csr);
  if (rowptr)
    CK(cudaMemcpyAsync(rowptr, csr_rowptr(c->csr), sizeof(int) * nr, cudaMemcpyDeviceToDevice, c->s));
  if (col) CK(cudaMemcpyAsync(col, csr_col(c->csr), sizeof(int) * nz, cudaMemcpyDeviceToDevice, c->s));
  if (val) CK(cudaMemcpyAsync(val, csr_val(c->csr), sizeof(double) * nz, cudaMemcpyDeviceToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  return PFF_OK;
}

int pff_memory(pff_ctx* c, long long* level_bytes, long long* krylov, long long* coarse, long long* other,
               long long* total) {
  if (!c) return PFF_ERR_INVALID_ARG;
  long long sum = c->krylov_bytes + c->coarse_bytes + c->other_bytes;
  long long csr = 0;
  if (c->csr) csr = csr_nnz(c->csr) * (long long)(sizeof(int) + sizeof(double)) + (c->lv[0].nd + 1) * (long long)sizeof(int);
  for (int l = 0; l < c->nlev; ++l) {
    const long long b = (size_t)l < c->level_bytes.size() ? c->level_bytes[(size_t)l] : 0;
    if (level_bytes) level_bytes[l] = b;
    sum += b;
  }
  if (krylov) *krylov = c->krylov_bytes;
  if (coarse) *coarse = c->coarse_bytes;
  if (other) *other = c->other_bytes + csr;
  if (total) *total = sum + csr;
  return PFF_OK;
}

int pff_set_load_component(pff_ctx* c, int comp) {
  if (!c || comp < 0 || comp >= c->dim) return PFF_ERR_INVALID_ARG;
  c->load_comp = comp;
  return PFF_OK;
}

int pff_get_history(pff_ctx* c, double* phi1, double* phi2, int* n_hist) {
  if (!c || !n_hist) return PFF_ERR_INVALID_ARG;
  const long long nn = c->lv[0].nn;
  if (phi1 && c->nhist >= 1)
    CK(cudaMemcpyAsync(phi1, c->hist1, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->s));
  if (phi2 && c->nhist >= 2)
    CK(cudaMemcpyAsync(phi2, c->hist2, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  *n_hist = c->nhist;
  return PFF_OK;
}

int pff_set_history(pff_ctx* c, const double* phi1, const double* phi2, int n_hist) {
  if (!c || n_hist < 0 || n_hist > 2 || (n_hist >= 1 && !phi1) || (n_hist == 2 && !phi2))
    return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  const long long nn = c->lv[0].nn;
  if (n_hist >= 1) CK(cudaMemcpyAsync(c->hist1, phi1, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->s));
  if (n_hist == 2) CK(cudaMemcpyAsync(c->hist2, phi2, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  c->nhist = n_hist;
  return PFF_OK;
}

int pff_diagonal(pff_ctx* c, int level, void* diag, int precision) {
  if (!c || !diag || level < 0 || level >= c->nlev || !valid_prec(precision)) return PFF_ERR_INVALID_ARG;
  CR(mg_setup(c));
  LevelData& L = c->lv[level];
  if (precision == 64) {
    CR(ensure_diag64(c));
    CK(cudaMemcpyAsync(diag, L.d64, sizeof(double) * L.nd, cudaMemcpyDeviceToDevice, c->s));
  } else if (c->prm.mg_precision == 32) {
    CK(cudaMemcpyAsync(diag, L.d32, sizeof(float) * L.nd, cudaMemcpyDeviceToDevice, c->s));
  } else {
    CK(launch_cast<double, float>(L.nd, L.d64, static_cast<float*>(diag), c->s));
  }
  return PFF_OK;
}

int pff_lambda_max(pff_ctx* c, int level, double* lam2) {
  if (!c || !lam2 || level < 0 || level >= c->nlev) return PFF_ERR_INVALID_ARG;
  CR(mg_setup(c));
  CK(cudaMemcpyAsync(c->pinned, c->lv[level].lam, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  lam2[0] = c->pinned[0];
  lam2[1] = c->pinned[1];
  return PFF_OK;
}

int pff_level_state(pff_ctx* c, int level, double* U_level) {
  if (!c || !U_level || level < 0 || level >= c->nlev) return PFF_ERR_INVALID_ARG;
  CR(mg_setup(c));
  CK(cudaMemcpyAsync(U_level, c->lv[level].U, sizeof(double) * c->lv[level].nd, cudaMemcpyDeviceToDevice, c->s));
  return PFF_OK;
}

int pff_prolongate(pff_ctx* c, int level, const void* xc, void* yf, int precision) {
  if (!c || !xc || !yf || level < 0 || level + 1 >= c->nlev || !valid_prec(precision)) return PFF_ERR_INVALID_ARG;
  CR(mg_setup(c));
  LevelData &L = c->lv[level], &Lc = c->lv[level + 1];
  if (precision == 64)
    CK(launch_prolong<double>(c->dim, c->p, static_cast<const double*>(xc), static_cast<double*>(yf), L.flags, Lc.g,
                              L.g, c->xt, false, c->s));
  else
    CK(launch_prolong<float>(c->dim, c->p, static_cast<const float*>(xc), static_cast<float*>(yf), L.flags, Lc.g,
                             L.g, c->xt, false, c->s));
  return PFF_OK;
}

int pff_restrict(pff_ctx* c, int level, const void* xf, void* yc, int precision) {
  if (!c || !xf || !yc || level < 0 || level + 1 >= c->nlev || !valid_prec(precision)) return PFF_ERR_INVALID_ARG;
  CR(mg_setup(c));
  LevelData &L = c->lv[level], &Lc = c->lv[level + 1];
  if (precision == 64)
    CK(launch_restrict<double>(c->dim, c->p, static_cast<const double*>(xf), static_cast<double*>(yc), L.flags,
                               Lc.flags, L.g, Lc.g, c->xt, c->s));
  else
    CK(launch_restrict<float>(c->dim, c->p, static_cast<const float*>(xf), static_cast<float*>(yc), L.flags,
                              Lc.flags, L.g, Lc.g, c->xt, c->s));
  return PFF_OK;
}

int pff_smooth(pff_ctx* c, int level, const void* f, void* x, int precision) {
  if (!c || !f || !x || level < 0 || level >= c->nlev || !valid_prec(precision)) return PFF_ERR_INVALID_ARG;
  CR(mg_setup(c));
  if (precision == 64) {
    CR(ensure_diag64(c));
    CR(ensure_work<double>(c, level));
    LevelData& L = c->lv[level];
    return smooth<double>(c, level, static_cast<const double*>(f), static_cast<double*>(x), L.w64[2], L.w64[4]);
  }
  CR(ensure_work<float>(c, level));
  LevelData& L = c->lv[level];
  return smooth<float>(c, level, static_cast<const float*>(f), static_cast<float*>(x), L.w32[2], L.w32[4]);
}

int pff_coarse_solve(pff_ctx* c, const double* r, double* z) {
  if (!c || !r || !z) return PFF_ERR_INVALID_ARG;
  CR(mg_setup(c));
  return coarse_solve<double>(c, r, z);
}

int pff_vcycle(pff_ctx* c, const double* r, double* z) {
  Range nvtx_range("pff_vcycle");
  if (!c || !r || !z || r == z) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  CR(mg_setup(c));
  // the cycle assumes a residual that is zero on masked rows (Dirichlet DoFs, active set)
  double* rm = c->scratch;
  CK(launch_masked_copy(c->dim, c->lv[0].nn, 1.0, r, c->lv[0].flags, 0xffu, rm, c->s));
  return precondition(c, rm, z);
}

int pff_solve_linear(pff_ctx* c, const double* b, double* x, int* iters, double* rel) {
  Range nvtx_range("pff_solve_linear");
  if (!c || !b || !x || b == x) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  return fgmres(c, b, x, iters, rel);
}

int pff_solve_newton_step(pff_ctx* c, double* U_out, pff_report* rep) {
  Range nvtx_range("pff_solve_newton_step");
  if (!c) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  using clk = std::chrono::steady_clock;
  auto ms = [](clk::time_point a, clk::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  LevelData& L = c->lv[0];
  pff_report r{};
  CK(cudaStreamSynchronize(c->s));
  const auto t0 = clk::now();
  Phases phase;
  phase.next("residual and active set");
  // Alg. 1: residual, active set (phi reset to phi_old on it), residual of the projected state. After
  // pff_set_state with active = NULL the active set of this U is already there.
  if (!c->fresh_active) {
    CR(residual_into(c, c->R));
    CK(launch_active_set(c->dim, L.nn, c->R, c->mass, c->phi_old, c->prm.as_c, L.U, L.flags, c->cnt, c->s));
  }
  c->fresh_active = false;
  c->qp_valid = false;
  c->mg_ready = false;
  CR(residual_into(c, c->R));
  CK(launch_newton_rhs(c->dim, L.nn, c->R, L.flags, c->rhs, c->s));
  double r2;
  CR(norm2_host(c, c->rhs, L.nd, &r2));
  int cnt[2];
  CK(cudaMemcpy(cnt, c->cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  r.res_norm = std::sqrt(r2);
  r.n_active = cnt[0];
  r.n_changed = cnt[1];
  const auto t1 = clk::now();
  phase.next("multigrid setup");
  CR(mg_setup(c));
  CK(cudaStreamSynchronize(c->s));
  CR(prof_collect(c));
  const auto t2 = clk::now();
  phase.next("FGMRES");
  r.status = fgmres(c, c->rhs, c->dU, &r.gmres_iters, &r.gmres_rel);
  if (r.status == PFF_OK || r.status == PFF_ERR_NOT_CONVERGED) {
    CK(launch_axpby<double>(L.nd, 1.0, c->dU, 1.0, L.U, c->s));
    c->qp_valid = false;
    c->strain_valid = false;
    c->mg_ready = false;
    if (U_out) CK(cudaMemcpyAsync(U_out, L.U, sizeof(double) * L.nd, cudaMemcpyDeviceToDevice, c->s));
  }
  CK(cudaStreamSynchronize(c->s));
  const auto t3 = clk::now();
  r.t_residual_ms = ms(t0, t1);
  r.t_setup_ms = ms(t1, t2);
  r.t_solve_ms = ms(t2, t3);
  if (rep) *rep = r;
  return r.status;
}

int pff_solve_pdas(pff_ctx* c, int max_iters, double newton_rtol, double* U_out, pff_report* reps, int* n_steps) {
  Range nvtx_range("pff_solve_pdas");
  if (!c || max_iters < 1 || !(newton_rtol > 0)) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  double r0 = -1.0;
  int st = PFF_ERR_NOT_CONVERGED, k = 0;
  for (; k < max_iters;) {
    pff_report r{};
    const int s = pff_solve_newton_step(c, nullptr, &r);
    if (reps) reps[k] = r;
    ++k;
    if (s != PFF_OK && s != PFF_ERR_NOT_CONVERGED) {
      st = s;
      break;
    }
    if (r0 < 0) r0 = r.res_norm;
    // converged: active set unchanged against the previous step and the reduced residual small
    if (k > 1 && r.n_changed == 0 && r.res_norm <= newton_rtol * r0) {
      st = PFF_OK;
      break;
    }
  }
  if (n_steps) *n_steps = k;
  if (U_out) CK(cudaMemcpyAsync(U_out, c->lv[0].U, sizeof(double) * c->lv[0].nd, cudaMemcpyDeviceToDevice, c->s));
  CK(cudaStreamSynchronize(c->s));
  return st;
}

int pff_solve_load_step(pff_ctx* c, double load, int max_iters, double newton_rtol, pff_report* reps,
                        int* n_steps) {
  Range nvtx_range("pff_solve_load_step");
  if (!c || max_iters < 1 || !(newton_rtol > 0)) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  LevelData& L = c->lv[0];
  const long long nn = L.nn;
  // Before the first solved load step the previous phase field is the state's own (held in hist1 as a
  // work copy, not counted: it is not the solution of a load step, so phi~ is not extrapolated from it).
  if (c->nhist == 0)
    CK(cudaMemcpyAsync(c->hist1, L.U + c->dim * nn, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->s));
  CK(launch_load_step_prep(load_comp(c), nn, L.flags, load, L.U, c->hist1, c->nhist >= 2 ? c->hist2 : nullptr,
                           L.phit, c->phi_old, c->s));
  c->fresh_active = false;  // the load and phi_old changed
  c->qp_valid = false;
  c->st_valid = false;
  c->strain_valid = false;
  c->mg_ready = false;
  const int st = pff_solve_pdas(c, max_iters, newton_rtol, nullptr, reps, n_steps);
  if (st == PFF_OK) {
    if (c->nhist >= 1) std::swap(c->hist1, c->hist2);
    CK(cudaMemcpyAsync(c->hist1, L.U + c->dim * nn, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->s));
    c->nhist = c->nhist >= 1 ? 2 : 1;
    CK(cudaStreamSynchronize(c->s));
  }
  return st;
}

int pff_param_grad(pff_ctx* c, const double* v, double* g_gc, double* g_lambda, double* g_mu) {
  Range nvtx_range("pff_param_grad");
  if (!c || !v) return PFF_ERR_INVALID_ARG;
  CR(ensure_st(c));
  LevelData& L = c->lv[0];
  if (!c->pgrad_tmp) {
    const long long ncell = c->dim == 2 ? (long long)L.N * L.N : (long long)L.N * L.N * L.N;
    const int nq = c->dim == 2 ? (c->p + 1) * (c->p + 1) : (c->p + 1) * (c->p + 1) * (c->p + 1);
    CR(dalloc(c, &c->pgrad_tmp, 3 * ncell * nq));
  }
  MatConst mc{c->prm.lambda, c->prm.mu, c->prm.gc, c->prm.eps, c->prm.kappa};
  // Dirichlet rows of the residual are identically zero: their test values do not enter
  double* vm = c->scratch;
  CK(launch_masked_copy(c->dim, L.nn, 1.0, v, L.flags, (1u << c->dim) - 1u, vm, c->s));
  CK(launch_param_grad(c->dim, c->p, c->prm.split, L.U, vm, L.st64, L.g, L.t64, mc, c->pgrad_tmp, g_gc, g_lambda,
                       g_mu, c->s));
  return PFF_OK;
}

long long pff_launch_count(void) { return launch_count(); }

int pff_profile(pff_ctx* c, int family) {
  if (!c || family < PFF_PROF_OFF || family > PFF_PROF_RESIDUAL) return PFF_ERR_INVALID_ARG;
  if (family != PFF_PROF_OFF && c->ev.empty()) {
    c->ev.resize(2 * PROF_MAX_LAUNCHES);
    for (auto& e : c->ev) CK(cudaEventCreate(&e));
    c->gev.resize(2 * PROF_MAX_LAUNCHES);
    for (auto& e : c->gev) CK(cudaEventCreate(&e));
  }
  CK(cudaStreamSynchronize(c->s));
  c->pending.clear();
  c->prof = family;
  c->nev = 0;
  c->prof_ms = 0.0;
  c->prof_n = 0;
  return PFF_OK;
}

int pff_profile_result(pff_ctx* c, int* launches, double* total_ms) {
  if (!c) return PFF_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(c->s));
  CR(prof_collect(c));
  double tot = c->prof_ms;
  for (int i = 0; i + 1 < c->nev; i += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    tot += ms;
  }
  if (launches) *launches = (int)(c->nev / 2 + c->prof_n);
  if (total_ms) *total_ms = tot;
  return PFF_OK;
}

}  // extern "C"

// ---- allocation-free parameter gradient ---------------------------------------------------------
// Per-point scratch of pff_param_grad_noalloc: a file-scope array in device global memory. In host
// code g_noalloc_scratch only names the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[PFF_NOALLOC_SCRATCH_DOUBLES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mutex;

// Device address of the scratch array on the context's device (looked up once per device). The symbol
// address belongs to whichever device is current, so the context's device must be the current one.
int noalloc_scratch(const pff_ctx* c, double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev != c->device || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return PFF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return PFF_OK;
}
}  // namespace

extern "C" int pff_param_grad_noalloc(pff_ctx* c, const double* v, double* g_gc, double* g_lambda, double* g_mu) {
  Range nvtx_range("pff_param_grad_noalloc");
  if (!c || !v) return PFF_ERR_INVALID_ARG;
  if (!c->has_state) return PFF_ERR_NO_STATE;
  LevelData& L = c->lv[0];
  const long long ncell = c->dim == 2 ? (long long)L.N * L.N : (long long)L.N * L.N * L.N;
  const int nq = c->dim == 2 ? (c->p + 1) * (c->p + 1) : (c->p + 1) * (c->p + 1) * (c->p + 1);
  if (3 * ncell * nq > PFF_NOALLOC_SCRATCH_DOUBLES) return PFF_ERR_TOO_LARGE;
  double* tmp = nullptr;
  CR(noalloc_scratch(c, &tmp));
  CR(ensure_st(c));
  MatConst mc{c->prm.lambda, c->prm.mu, c->prm.gc, c->prm.eps, c->prm.kappa};
  double* vm = c->scratch;  // allocated with the context
  CK(launch_masked_copy(c->dim, L.nn, 1.0, v, L.flags, (1u << c->dim) - 1u, vm, c->s));
  CK(launch_param_grad(c->dim, c->p, c->prm.split, L.U, vm, L.st64, L.g, L.t64, mc, tmp, g_gc, g_lambda, g_mu, c->s));
  return PFF_OK;
}
