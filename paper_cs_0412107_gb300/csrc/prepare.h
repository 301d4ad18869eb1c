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
};

// Validate C (MCINV_E_ARG / MCINV_E_SINGULAR_DIAG with a message), build C^dagger,
// the dependency levels (rows of a level sorted by decreasing work) and the
// chunk stream with shared-memory buffers of at least min_blob bytes.
mcinv_status prepare_matrix(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                            int min_blob, Prepared &P, std::string *err);

}  // namespace mcinv
