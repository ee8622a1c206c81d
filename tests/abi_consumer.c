/* A plain C99 consumer of include/pff.h: compiled with gcc and linked against libpff by
 * tests/test_library_abi.py, it calls the host-only entry points (no GPU needed) and checks their
 * results. Exit status 0 = every check passed; otherwise the number of the failed check. */
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "pff.h"

int main(void) {
  pff_params p;
  pff_default_params(&p);
  if (p.dim != 2 && p.dim != 3) return 1;
  /* defaults of the fields appended last: FP64 coarse solve, one node per grid point */
  if (p.coarse_precision != 64 || p.slit_cut != 0) return 13;
  if (!pff_strerror(PFF_ERR_UNAVAILABLE) || !strlen(pff_strerror(PFF_ERR_UNAVAILABLE))) return 2;

  /* 2D Q1, 2 x 2 cells, nothing masked: 3 x 3 nodes whose cell-coupling windows hold 2, 3, 2 indices
   * per direction, so sum_nodes |window| = (2 + 3 + 2)^2 = 49; displacement rows couple to the 2
   * displacement components, phase-field rows to all 3: nnz = (2 * 2 + 3) * 49 = 343. */
  unsigned char flags[9];
  memset(flags, 0, sizeof flags);
  long long nnz = -1;
  if (pff_csr_pattern(2, 1, 2, flags, NULL, NULL, &nnz) != PFF_OK || nnz != 343) return 3;
  int* rowptr = (int*)malloc(sizeof(int) * (27 + 1));
  int* col = (int*)malloc(sizeof(int) * (size_t)nnz);
  if (pff_csr_pattern(2, 1, 2, flags, rowptr, col, &nnz) != PFF_OK) return 4;
  if (rowptr[0] != 0 || rowptr[27] != 343) return 5;
  /* the centre node's u_x row: the 9 nodes of both displacement components, ascending */
  if (rowptr[5] - rowptr[4] != 18 || col[rowptr[4]] != 0 || col[rowptr[5] - 1] != 17) return 6;
  /* masking the centre node's phase field leaves its row the diagonal only */
  flags[4] = 1u << 2;
  if (pff_csr_pattern(2, 1, 2, flags, rowptr, col, &nnz) != PFF_OK) return 7;
  if (rowptr[2 * 9 + 4 + 1] - rowptr[2 * 9 + 4] != 1 || col[rowptr[2 * 9 + 4]] != 2 * 9 + 4) return 8;

  /* probing plan: colour 0 of component 0 (nodes with i = 0 mod 3 per direction, here the corner
   * node 0 only) is the column that row 0 (u_x at node 0) fills */
  long long targets[27];
  if (pff_csr_probe_targets(2, 1, 2, 0, 0, targets) != PFF_OK || targets[0] != 0) return 9;
  /* bad arguments come back as status codes */
  if (pff_csr_pattern(5, 1, 2, flags, NULL, NULL, &nnz) != PFF_ERR_INVALID_ARG) return 10;
  if (pff_csr_probe_targets(2, 1, 2, 3, 0, targets) != PFF_ERR_INVALID_ARG) return 11;
  if (pff_set_load_component(NULL, 0) != PFF_ERR_INVALID_ARG) return 12;
  free(rowptr);
  free(col);
  /* the struct layout, for the binding's ctypes mirror */
  printf("layout %zu %zu %zu %zu\n", sizeof(pff_params), offsetof(pff_params, fp64_mode),
         offsetof(pff_params, coarse_precision), offsetof(pff_params, slit_cut));
  printf("ok\n");
  return 0;
}
