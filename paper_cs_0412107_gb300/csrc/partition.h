// partition.h -- the block partition of Sec. 4 (host side): C~ = S^-1 C S^-1.
#pragma once

#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/mcinv.h"

namespace mcinv {

struct Partition {
    std::vector<int64_t> block_ptr;               // contiguous blocks: rows block_ptr[b] .. block_ptr[b+1]-1
    std::vector<int64_t> sinv_off;                // offset of S_b^-1 (row-major, size^2) in sinv; empty for one row
    std::vector<std::complex<double>> sinv;      // S_b^-1
    std::vector<std::complex<double>> s;         // S_b (same offsets)
    int64_t multi = 0;                            // blocks of two or more rows
};

// Validate the partition, form S_b^-1 (principal square root of each diagonal
// block of two or more rows, Denman-Beavers) and C~ = S^-1 C S^-1 in CSR (sorted
// columns; the input's value type).  MCINV_E_ARG for a malformed input,
// MCINV_E_SINGULAR_DIAG for a block without a principal square root or a
// one-row block with a zero diagonal.
mcinv_status partition_transform(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int cplx,
                                 int64_t nblocks, const int64_t *block_ptr, std::vector<int64_t> &rp2,
                                 std::vector<int32_t> &col2, std::vector<double> &val2, Partition &part,
                                 std::string *err);

}  // namespace mcinv
