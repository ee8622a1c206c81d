// pff_csr.cu -- the assembled-matrix comparator: CSR pattern, probing kernels, cuSPARSE SpMV
// (the sparse-matrix product that the paper measures against the matrix-free one, Sec. 6.3,
// fig. compare:vmult).
#include <dlfcn.h>

#include <climits>
#include <cstdint>
#include <mutex>

#include <cusparse.h>  // types and enumerators only: the functions are resolved with dlsym

#include "../../include/pff.h"
#include "pff_csr.h"
#include "pff_launch.h"

namespace pff {

__host__ __device__ long long probe_target(long long r, long long nn, int n1, int dim, int p, int f, int color);

namespace {

constexpr int CSR_BLK = 256;

unsigned csr_grid(long long n) { return (unsigned)((n + CSR_BLK - 1) / CSR_BLK); }

// cuSPARSE entry points, looked up once per process.
struct SparseLib {
  bool ok = false;
  decltype(&cusparseCreate) create = nullptr;
  decltype(&cusparseDestroy) destroy = nullptr;
  decltype(&cusparseSetStream) set_stream = nullptr;
  decltype(&cusparseCreateCsr) create_csr = nullptr;
  decltype(&cusparseDestroySpMat) destroy_spmat = nullptr;
  decltype(&cusparseCreateDnVec) create_dnvec = nullptr;
  decltype(&cusparseDestroyDnVec) destroy_dnvec = nullptr;
  decltype(&cusparseSpMV_bufferSize) spmv_buffer_size = nullptr;
  decltype(&cusparseSpMV) spmv = nullptr;
};

template <typename F>
bool sym(void* h, const char* name, F& f) {
  f = reinterpret_cast<F>(dlsym(h, name));
  return f != nullptr;
}

SparseLib& sparse_lib() {
  static SparseLib L;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = nullptr;
    // by soname (the loader's paths, or a copy the process has loaded already), then in the
    // library directory of the toolkit that built libpff
    const char* names[] = {"libcusparse.so.12", "libcusparse.so",
#ifdef PFF_CUDA_LIBDIR
                           PFF_CUDA_LIBDIR "/libcusparse.so.12",
#endif
                           nullptr};
    for (int k = 0; names[k] && !h; ++k) h = dlopen(names[k], RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    L.ok = sym(h, "cusparseCreate", L.create) && sym(h, "cusparseDestroy", L.destroy) &&
           sym(h, "cusparseSetStream", L.set_stream) && sym(h, "cusparseCreateCsr", L.create_csr) &&
           sym(h, "cusparseDestroySpMat", L.destroy_spmat) && sym(h, "cusparseCreateDnVec", L.create_dnvec) &&
           sym(h, "cusparseDestroyDnVec", L.destroy_dnvec) &&
           sym(h, "cusparseSpMV_bufferSize", L.spmv_buffer_size) && sym(h, "cusparseSpMV", L.spmv);
  });
  return L;
}

__device__ __forceinline__ int node_color(long long j, int n1, int dim, int m) {
  const int x = (int)(j % n1);
  const int y = (int)((j / n1) % n1);
  const int z = dim == 3 ? (int)(j / ((long long)n1 * n1)) : 0;
  return x % m + m * (y % m + m * (z % m));
}

__global__ void k_probe_set(long long nd, long long nn, int n1, int dim, int m, int f, int color,
                            double* __restrict__ x) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const int comp = (int)(i / nn);
  x[i] = (comp == f && node_color(i - comp * nn, n1, dim, m) == color) ? 1.0 : 0.0;
}

__global__ void k_probe_gather(long long nrows, const int* __restrict__ rowptr, const int* __restrict__ col,
                               double* __restrict__ val, const double* __restrict__ y, long long nn, int n1, int dim,
                               int p, int f, int color) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const long long tl = probe_target(r, nn, n1, dim, p, f, color);
  if (tl < 0) return;
  const int target = (int)tl;
  int a = rowptr[r], b = rowptr[r + 1];  // bisection over the row's ascending columns, [a, b)
  while (a < b) {
    const int mid = a + ((b - a) >> 1);
    if (col[mid] < target) a = mid + 1;
    else b = mid;
  }
  if (a < rowptr[r + 1] && col[a] == target) val[a] = y[r];
}

}  // namespace

// The column of row r probed by (f, color): per direction, the one index of colour class color_t
// in the window of nodes sharing a cell with the row's node (the window spans at most 2p+1 = m
// indices); -1 when the window holds none. The pattern may still lack that column (a masked DoF, a
// phase-field column in a displacement row, or any column of a masked row but its diagonal).
__host__ __device__ long long probe_target(long long r, long long nn, int n1, int dim, int p, int f, int color) {
  const int m = 2 * p + 1, N = (n1 - 1) / p;
  long long i = r % nn;
  int cc = color;
  long long j = 0, stride = 1;
  for (int t = 0; t < dim; ++t) {
    const int it = (int)(i % n1);
    i /= n1;
    const int ct = cc % m;
    cc /= m;
    int clo = it / p, chi = it / p;
    if (it % p == 0) clo -= 1;
    if (clo < 0) clo = 0;
    if (chi > N - 1) chi = N - 1;
    const int lo = clo * p, hi = chi * p + p;
    const int jt = lo + ((ct - lo % m) % m + m) % m;
    if (jt > hi) return -1;
    j += jt * stride;
    stride *= n1;
  }
  return f * nn + j;
}

struct CsrMat {
  long long nrows = 0, nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  void* buf = nullptr;  // SpMV workspace
  size_t buf_bytes = 0;
  cusparseHandle_t handle = nullptr;
  cusparseSpMatDescr_t A = nullptr;
};

bool csr_pattern(int dim, int p, int N, const unsigned char* flags, std::vector<int>& rowptr, std::vector<int>& col) {
  const int n1 = p * N + 1;
  const long long nn = dim == 2 ? (long long)n1 * n1 : (long long)n1 * n1 * n1;
  const long long nd = (dim + 1) * nn;
  if (nd + 1 > INT_MAX) return false;
  // nodes sharing a cell with index i, per direction: [lo[i], hi[i]]
  std::vector<int> lo(n1), hi(n1);
  for (int i = 0; i < n1; ++i) {
    int clo = i / p, chi = i / p;
    if (i % p == 0) clo -= 1;
    if (clo < 0) clo = 0;
    if (chi > N - 1) chi = N - 1;
    lo[i] = clo * p;
    hi[i] = chi * p + p;
  }
  rowptr.assign((size_t)nd + 1, 0);
  col.clear();
  long long count = 0;
  for (int g = 0; g <= dim; ++g) {
    for (long long i = 0; i < nn; ++i) {
      const long long r = g * nn + i;
      rowptr[(size_t)r] = (int)count;
      if ((flags[i] >> g) & 1u) {
        col.push_back((int)r);
        ++count;
        continue;
      }
      const int ix = (int)(i % n1), iy = (int)((i / n1) % n1), iz = dim == 3 ? (int)(i / ((long long)n1 * n1)) : 0;
      const int fmax = g < dim ? dim - 1 : dim;
      const int zlo = dim == 3 ? lo[iz] : 0, zhi = dim == 3 ? hi[iz] : 0;
      for (int f = 0; f <= fmax; ++f)
        for (int z = zlo; z <= zhi; ++z)
          for (int y = lo[iy]; y <= hi[iy]; ++y)
            for (int x = lo[ix]; x <= hi[ix]; ++x) {
              const long long j = x + (long long)n1 * (y + (long long)n1 * z);
              if ((flags[j] >> f) & 1u) continue;
              col.push_back((int)(f * nn + j));
              ++count;
            }
      if (count > INT_MAX) return false;
    }
  }
  rowptr[(size_t)nd] = (int)count;
  return true;
}

int csr_create(CsrMat** out, long long nrows, const std::vector<int>& rowptr, const std::vector<int>& col,
               cudaStream_t s) {
  *out = nullptr;
  CsrMat* m = new CsrMat();
  m->nrows = nrows;
  m->nnz = (long long)col.size();
  const size_t nz = col.empty() ? 1 : col.size();
  if (cudaMalloc(&m->rowptr, sizeof(int) * rowptr.size()) != cudaSuccess ||
      cudaMalloc(&m->col, sizeof(int) * nz) != cudaSuccess || cudaMalloc(&m->val, sizeof(double) * nz) != cudaSuccess) {
    cudaGetLastError();
    csr_destroy(m);
    return PFF_ERR_OOM;
  }
  if (cudaMemcpyAsync(m->rowptr, rowptr.data(), sizeof(int) * rowptr.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(m->col, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(m->val, 0, sizeof(double) * nz, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    csr_destroy(m);
    return PFF_ERR_CUDA;
  }
  *out = m;
  return PFF_OK;
}

void csr_destroy(CsrMat* m) {
  if (!m) return;
  SparseLib& L = sparse_lib();
  if (m->A && L.ok) L.destroy_spmat(m->A);
  if (m->handle && L.ok) L.destroy(m->handle);
  if (m->buf) cudaFree(m->buf);
  if (m->val) cudaFree(m->val);
  if (m->col) cudaFree(m->col);
  if (m->rowptr) cudaFree(m->rowptr);
  delete m;
}

bool csr_spmv_available() { return sparse_lib().ok; }

long long csr_nnz(const CsrMat* m) { return m ? m->nnz : 0; }
const int* csr_rowptr(const CsrMat* m) { return m->rowptr; }
const int* csr_col(const CsrMat* m) { return m->col; }
const double* csr_val(const CsrMat* m) { return m->val; }

cudaError_t launch_probe_set(int dim, int p, long long nn, int n1, int f, int color, double* x, cudaStream_t s) {
  const long long nd = (dim + 1) * nn;
  count_launch();
  k_probe_set<<<csr_grid(nd), CSR_BLK, 0, s>>>(nd, nn, n1, dim, 2 * p + 1, f, color, x);
  return cudaGetLastError();
}

cudaError_t launch_probe_gather(CsrMat* m, int dim, int p, long long nn, int n1, int f, int color, const double* y,
                                cudaStream_t s) {
  count_launch();
  k_probe_gather<<<csr_grid(m->nrows), CSR_BLK, 0, s>>>(m->nrows, m->rowptr, m->col, m->val, y, nn, n1, dim, p, f,
                                                         color);
  return cudaGetLastError();
}

int csr_spmv(CsrMat* m, const double* x, double* y, cudaStream_t s) {
  SparseLib& L = sparse_lib();
  if (!L.ok) return PFF_ERR_UNAVAILABLE;
  const double one = 1.0, zero = 0.0;
  if (!m->handle) {
    if (L.create(&m->handle) != CUSPARSE_STATUS_SUCCESS) {
      m->handle = nullptr;
      return PFF_ERR_CUDA;
    }
    if (L.create_csr(&m->A, m->nrows, m->nrows, m->nnz, m->rowptr, m->col, m->val, CUSPARSE_INDEX_32I,
                     CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, CUDA_R_64F) != CUSPARSE_STATUS_SUCCESS) {
      m->A = nullptr;
      return PFF_ERR_CUDA;
    }
  }
  if (L.set_stream(m->handle, s) != CUSPARSE_STATUS_SUCCESS) return PFF_ERR_CUDA;
  cusparseDnVecDescr_t vx = nullptr, vy = nullptr;
  int st = PFF_OK;
  if (L.create_dnvec(&vx, m->nrows, const_cast<double*>(x), CUDA_R_64F) != CUSPARSE_STATUS_SUCCESS ||
      L.create_dnvec(&vy, m->nrows, y, CUDA_R_64F) != CUSPARSE_STATUS_SUCCESS) {
    st = PFF_ERR_CUDA;
  } else {
    size_t need = 0;
    if (L.spmv_buffer_size(m->handle, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, m->A, vx, &zero, vy, CUDA_R_64F,
                           CUSPARSE_SPMV_ALG_DEFAULT, &need) != CUSPARSE_STATUS_SUCCESS) {
      st = PFF_ERR_CUDA;
    } else if (need > m->buf_bytes) {
      if (m->buf) cudaFree(m->buf);
      m->buf = nullptr;
      m->buf_bytes = 0;
      if (cudaMalloc(&m->buf, need) != cudaSuccess) {
        cudaGetLastError();
        st = PFF_ERR_OOM;
      } else {
        m->buf_bytes = need;
      }
    }
    if (st == PFF_OK && L.spmv(m->handle, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, m->A, vx, &zero, vy, CUDA_R_64F,
                               CUSPARSE_SPMV_ALG_DEFAULT, m->buf) != CUSPARSE_STATUS_SUCCESS)
      st = PFF_ERR_CUDA;
  }
  if (vx) L.destroy_dnvec(vx);
  if (vy) L.destroy_dnvec(vy);
  return st;
}

}  // namespace pff
