// pff_csr.h -- the assembled-matrix comparator of libpff (internal): the CSR pattern of the masked
// Jacobian on a structured Q_p mesh, the probing kernels that fill it from the matrix-free operator,
// and y = A x by cuSPARSE (loaded at run time, so the library does not depend on it otherwise).
#pragma once
#include <cuda_runtime.h>
#include <vector>

namespace pff {

// Structural pattern of Z G Z + (I - Z) (Eq. (G), masked as in the linear solve) on the (pN+1)^dim
// node grid, rows and columns in the component-blocked DoF order [u_1 | ... | u_d | phi]:
// * a masked row (bit f of the node's flags for component f) holds its diagonal only;
// * an unmasked row of node i couples to the unmasked DoFs of every node that shares a cell with i
//   (per direction: [p c_lo, p c_hi + p] over the cells c_lo..c_hi that contain i), of the
//   displacement components for a displacement row (G_uphi = 0) and of all d+1 components for a
//   phase-field row. Columns of a row ascend.
// rowptr gets n_dofs + 1 entries. Returns false (outputs unspecified) when n_dofs or the number of
// entries does not fit a 32-bit index.
bool csr_pattern(int dim, int p, int N, const unsigned char* flags, std::vector<int>& rowptr, std::vector<int>& col);

struct CsrMat;  // device CSR (32-bit indices, FP64 values) and its cuSPARSE state

// Allocates the device arrays for the pattern and uploads it; values are zeroed. Returns a PFF_ERR_*
// status (PFF_OK on success).
int csr_create(CsrMat** out, long long nrows, const std::vector<int>& rowptr, const std::vector<int>& col,
               cudaStream_t s);
void csr_destroy(CsrMat* m);
long long csr_nnz(const CsrMat* m);
const int* csr_rowptr(const CsrMat* m);
const int* csr_col(const CsrMat* m);
const double* csr_val(const CsrMat* m);

// Probing with colours (2p+1)^dim per component: two nodes of one colour differ by a nonzero multiple
// of 2p+1 in some direction, so no row couples to both. x = indicator of the DoFs of component f
// whose node has colour `color`; after y = A x, every entry (r, c) of the pattern with c of component
// f and colour `color` takes y[r].
__host__ __device__ long long probe_target(long long r, long long nn, int n1, int dim, int p, int f, int color);
cudaError_t launch_probe_set(int dim, int p, long long nn, int n1, int f, int color, double* x, cudaStream_t s);
cudaError_t launch_probe_gather(CsrMat* m, int dim, int p, long long nn, int n1, int f, int color, const double* y,
                                cudaStream_t s);

// y = A x by cuSPARSE SpMV (FP64, default algorithm) on stream s. Returns PFF_OK, PFF_ERR_UNAVAILABLE
// when cuSPARSE cannot be loaded, or PFF_ERR_CUDA.
int csr_spmv(CsrMat* m, const double* x, double* y, cudaStream_t s);
// Whether cuSPARSE was found and all its entry points resolved (loads it on first call; no GPU work).
bool csr_spmv_available();

}  // namespace pff
