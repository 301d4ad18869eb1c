// tc_gemm.h -- tensor-core (tcgen05, TMA, TMEM) block contraction
//   D[M][N] = A[M][inner] . B[N][inner]^T,  A, B bf16 K-major, D fp32 row-major.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda.h>

#include <string>

namespace mcinv {

// Grouped contraction for a pool of matrices: tile t computes the 128 x 256
// block (m0, n0) of matrix `slot`; maps[2*slot] / maps[2*slot+1] are that
// matrix's A and B tensor maps (in device memory), outs[slot] its output.
struct GroupTile {
    int slot, m0, n0, pad;
};
struct GroupOut {
    float *D;   // M x N row-major FP32
    int M, N;
    int ktiles; // 64-wide slices of the contraction dimension this step
    int add;    // 0: D = A B^T; 1: D += A B^T (the product of an earlier step is kept)
};
bool tc_encode_operand(CUtensorMap *map, const uint16_t *base, long long rows, long long ld, long long inner,
                       bool is_b, const char **why);
cudaError_t tc_gemm_grouped_run(const GroupTile *tiles, const int *ntiles, const CUtensorMap *maps, const GroupOut *outs,
                                int grid, int *status, cudaStream_t s);

struct TcGemmPlan;

// A: a_rows x ld bf16 (rows padded to the tile height, pad rows zero),
// B: b_rows x ld bf16, D: M x N fp32.  Returns NULL (and why) when the
// device or the shapes are unsupported.
TcGemmPlan *tc_gemm_plan_create(const uint16_t *A, size_t a_rows, const uint16_t *B, size_t b_rows,
                                long long ld, float *D, long long M, long long N, std::string *why);
// Contract the first `inner` columns (a multiple of 64, <= ld).  A bounded
// device-side wait that expires sets bit 1 (value 2) of *status.
cudaError_t tc_gemm_run(TcGemmPlan *plan, long long inner, int *status, cudaStream_t s);
void tc_gemm_plan_destroy(TcGemmPlan *plan);

// One contraction without a plan object: tensor maps are built on the
// caller's stack with the true extents (M, N, inner), so operands need no
// padding; A's and B's bases must be 16-byte aligned and lda, ldb multiples of
// 8 elements.  No allocation of any kind.  On failure *why names the cause.
cudaError_t tc_gemm_run_direct(const uint16_t *A, long long lda, const uint16_t *B, long long ldb, long long M,
                               long long N, long long inner, float *D, int *status, cudaStream_t s,
                               const char **why);

}  // namespace mcinv
