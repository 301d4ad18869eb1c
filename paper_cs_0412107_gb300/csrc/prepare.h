// prepare.h -- host-side preparation of a matrix for the sweep.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mcinv.h"
#include "internal.h"

namespace mcinv {

struct Prepared {
    int64_t n = 0, nnz = 0;
    int cplx = 0, nlev = 0, blob_max = 0;
    std::vector<int32_t> perm, pos;       // position -> row, row -> position
    std::vector<ChunkDesc> chunks;        // one cycle's chunk sequence
    std::vector<uint8_t> stream;          // chunk blobs (constants left zero: filled on the GPU)
    std::vector<long long> cst_at;        // byte offset of each position's constants in the stream
    std::vector<double> diag_pos;         // c_ii by position (re,im for complex)
    // the flat form of the grid-wide sweep: GridRow by position (n + 1 records),
    // the entries of C and of C^dagger by position (EntR / EntC bytes), and the
    // first position of every dependency level (nlev + 1)
    std::vector<GridRow> grow;
    std::vector<uint8_t> gzent, gwent;
    std::vector<int32_t> lev_ptr;
};

// Validate C (MCINV_E_ARG / MCINV_E_SINGULAR_DIAG with a message), build C^dagger,
// the dependency levels (rows of a level sorted by decreasing work) and the
// chunk stream with shared-memory buffers of at least min_blob bytes.
mcinv_status prepare_matrix(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                            int min_blob, Prepared &P, std::string *err);

// The colour sweep order (Sec. 4: reordering the rows and columns of C):
// rows in ascending index order each take the smallest colour not used by an
// already-coloured neighbour in the graph of C + C^T (off-diagonal entries);
// order[k] lists colour 0's rows ascending, then colour 1's, ...  No two rows
// of one colour read each other, so the Gauss-Seidel sweep of P C P^T has one
// dependency level per colour.  Checks the CSR structure and the diagonal
// (errors name rows of C as given).
mcinv_status color_order(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                         std::vector<int32_t> &order, int *ncolors, std::string *err);

// C' = P C P^T: row k of C' is row order[k] of C, columns renumbered by the
// inverse order and sorted ascending.
void permute_csr(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                 const std::vector<int32_t> &order, std::vector<int64_t> &rp2, std::vector<int32_t> &col2,
                 std::vector<double> &val2);

}  // namespace mcinv
