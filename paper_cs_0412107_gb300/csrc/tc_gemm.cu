// tc_gemm.cu -- the block estimate's contraction on the 5th-generation tensor
// cores: D[M][N] = A[M][inner] . B[N][inner]^T with A = BF16 shadows of z rows
// (chains x cycles along `inner`), B = BF16 shadows of w rows, D in FP32.
// This is the sum over chains and cycles of z_r conj(w_s) of Eq. 1/C.
//
// tc_gemm_kernel (the allocation-free path) runs one CTA per 128 x 256 output
// tile, 128 threads:
//   warp 0 lane 0  TMA producer: 64-wide K slices of A and B into a 4-stage
//                  ring of 128B-swizzled shared-memory tiles (mbarrier tx counts)
//   warp 1 lane 0  MMA issuer: tcgen05.mma kind::f16 (BF16 x BF16 -> FP32),
//                  M=128, N=256, K=16, accumulator in TMEM (256 columns);
//                  tcgen05.commit frees ring slots and finally signals the epilogue
//   warps 0-3      epilogue: tcgen05.ld 32 lanes x 32 columns at a time -> D
// tc_gemm_persistent_kernel (the handle's path) runs one CTA per SM over all
// tiles with two TMEM accumulators (below).
// Every wait is bounded (globaltimer); on expiry the CTA records a timeout in
// `status`, abandons the tile, releases TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "tc_gemm.h"

namespace mcinv {

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* align */ + 256 /* barriers */;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity; false if the CTA gave up
// (another role aborted, or WAIT_NS elapsed).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (globaltimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with
// 128-byte swizzling: rows of 128 B, 8-row core groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)(16u >> 4) << 16;          // leading byte offset (unused with 128B swizzle)
    d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M x N.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                   float *__restrict__ D, int M, int N, int ktiles, int *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(accf + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(accf), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % STAGES;
            const uint32_t phase = (uint32_t)(kt / STAGES) & 1u;
            if (kt >= STAGES && !mbar_wait(smem_u32(&empty[s]), phase ^ 1u, abort_flag)) break;
            mbar_expect_tx(smem_u32(&full[s]), STAGE_BYTES);
            tma_load_2d(smem_u32(sA + s * A_BYTES), &ta, smem_u32(&full[s]), kt * BK, m0);
            tma_load_2d(smem_u32(sB + s * B_BYTES), &tb, smem_u32(&full[s]), kt * BK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        bool ok = true;
        for (int kt = 0; kt < ktiles; ++kt) {
            const int s = kt % STAGES;
            const uint32_t phase = (uint32_t)(kt / STAGES) & 1u;
            if (!mbar_wait(smem_u32(&full[s]), phase, abort_flag)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t a = sdesc(smem_u32(sA + s * A_BYTES));
            const uint64_t b = sdesc(smem_u32(sB + s * B_BYTES));
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)  // advance 16 elements = 32 bytes = 2 units of 16 B
                mma_bf16(tmem, a + 2 * kk, b + 2 * kk, (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(smem_u32(&empty[s]));
        }
        if (ok) mma_commit(smem_u32(accf));
    }
    __syncwarp();

    // epilogue: warp w owns TMEM lanes (tile rows) 32w .. 32w+31; tcgen05.ld is
    // warp-collective, so the decision to read is made warp-uniform
    const bool have = __all_sync(0xffffffffu, mbar_wait(smem_u32(accf), 0u, abort_flag));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < M) {
                float *dst = D + (size_t)row * N + n0 + c0;
                if (n0 + c0 + 32 <= N && (N & 3) == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *(float4 *)(dst + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                           __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (n0 + c0 + j < N) dst[j] = __uint_as_float(r[j]);
                }
            }
        }
    }
    if (*abort_flag && threadIdx.x == 0) {
        atomicOr(status, 2);
        // give TMA copies still in flight time to land before the CTA exits
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 10000000ull) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---------------------------------------------------------------------------
// Persistent single-matrix contraction: one CTA per SM walks the 128 x 256
// tiles (t = CTA, CTA + grid, ...; the column tiles of one row band are
// neighbours in t, so they run at the same time and the band's A rows are read
// from DRAM once).  Warps: 0 = TMA producer, 1 = MMA issuer, 2..5 = epilogue.
// Two 256-column TMEM accumulators alternate between a CTA's tiles, so the
// epilogue of one tile runs under the MMAs of the next.
//
// When the tiles leave a last, partly filled wave of at most half the grid
// (and are long enough, kSplitMinKtiles), those remaining tiles are split
// along the contraction dimension into s parts each (one part per CTA): a part
// writes its FP32 partial tile to a workspace, and for each 32-row quarter of
// the tile the warp that completes the count of that quarter's parts sums
// them in part order into D.  The sum order is fixed, so the result does not
// depend on which CTA finishes last.
// ---------------------------------------------------------------------------
struct PersistSched {
    int NT;       // column tiles
    int Tfull;    // tiles computed whole (t < Tfull)
    int s;        // parts of each remaining tile (1: none remain)
    int npieces;  // (tiles - Tfull) * s
    int ktiles;   // 64-wide slices of the contraction dimension
};

// Work item idx of CTA b: a whole tile, or (last) its part of a split tile.
__device__ __forceinline__ bool persist_item(const PersistSched &S, int b, int G, int idx, int &m0, int &n0, int &k0,
                                             int &k1, int &piece)
{
    const int nfull = b < S.Tfull ? (S.Tfull - 1 - b) / G + 1 : 0;
    int t;
    if (idx < nfull) {
        t = b + idx * G;
        k0 = 0;
        k1 = S.ktiles;
        piece = -1;
    } else if (idx == nfull && b < S.npieces) {
        t = S.Tfull + b / S.s;
        const int q = b % S.s;
        k0 = (int)((long long)q * S.ktiles / S.s);
        k1 = (int)((long long)(q + 1) * S.ktiles / S.s);
        piece = b;
    } else {
        return false;
    }
    m0 = (t / S.NT) * BM;
    n0 = (t % S.NT) * BN;
    return true;
}

__global__ void __launch_bounds__(192, 1)
    tc_gemm_persistent_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                              float *__restrict__ D, int M, int N, const PersistSched S, float *__restrict__ work,
                              int *__restrict__ cnt, int *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;  // [2]
    uint64_t *tempty = tfull + 2;       // [2]
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x, G = gridDim.x;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(smem_u32(&full[st]), 1);
            mbar_init(smem_u32(&empty[st]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&tfull[a]), 1);
            mbar_init(smem_u32(&tempty[a]), 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    int m0, n0, k0, k1, piece;

    if (warp == 0) {
        if (lane == 0) {
            int kg = 0;  // k-slices issued so far (ring position)
            for (int idx = 0; !*abort_flag && persist_item(S, b, G, idx, m0, n0, k0, k1, piece); ++idx) {
                bool ok = true;
                for (int kt = k0; kt < k1; ++kt, ++kg) {
                    const int st = kg % STAGES;
                    const uint32_t phase = (uint32_t)(kg / STAGES) & 1u;
                    if (kg >= STAGES && !mbar_wait(smem_u32(&empty[st]), phase ^ 1u, abort_flag)) { ok = false; break; }
                    mbar_expect_tx(smem_u32(&full[st]), STAGE_BYTES);
                    tma_load_2d(smem_u32(sA + st * A_BYTES), &ta, smem_u32(&full[st]), kt * BK, m0);
                    tma_load_2d(smem_u32(sB + st * B_BYTES), &tb, smem_u32(&full[st]), kt * BK, n0);
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int kg = 0, tl = 0;
            for (int idx = 0; !*abort_flag && persist_item(S, b, G, idx, m0, n0, k0, k1, piece); ++idx, ++tl) {
                const int ab = tl & 1;  // this item's accumulator
                const uint32_t acc = tmem + (uint32_t)(ab * TMEM_COLS);
                // the epilogue must have drained this accumulator (two items ago)
                if (tl >= 2 && !mbar_wait(smem_u32(&tempty[ab]), (uint32_t)((tl >> 1) - 1) & 1u, abort_flag)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool ok = true;
                for (int kt = k0; kt < k1; ++kt, ++kg) {
                    const int st = kg % STAGES;
                    const uint32_t phase = (uint32_t)(kg / STAGES) & 1u;
                    if (!mbar_wait(smem_u32(&full[st]), phase, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t a = sdesc(smem_u32(sA + st * A_BYTES));
                    const uint64_t bd = sdesc(smem_u32(sB + st * B_BYTES));
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(acc, a + 2 * kk, bd + 2 * kk, (kt > k0 || kk > 0) ? 1u : 0u);
                    mma_commit(smem_u32(&empty[st]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&tfull[ab]));
            }
        }
    } else {
        // epilogue warps 2..5: warp w reads TMEM lanes 32*(w%4) .. +31 (tile rows)
        const int q = warp & 3;
        const int rt = q * 32 + lane;  // row within the tile
        int tl = 0;
        for (int idx = 0; persist_item(S, b, G, idx, m0, n0, k0, k1, piece); ++idx, ++tl) {
            const int ab = tl & 1;
            const bool have =
                __all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[ab]), (uint32_t)(tl >> 1) & 1u, abort_flag));
            if (!have) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = m0 + rt;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t)(ab * TMEM_COLS) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
                if (piece >= 0) {
                    float *wp = work + (size_t)piece * BM * BN + (size_t)rt * BN + c0;
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *(float4 *)(wp + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                          __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                } else if (row < M) {
                    float *dst = D + (size_t)row * N + n0 + c0;
                    if (n0 + c0 + 32 <= N && (N & 3) == 0) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *(float4 *)(dst + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                               __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (n0 + c0 + j < N) dst[j] = __uint_as_float(r[j]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[ab])) : "memory");
            if (piece >= 0) {
                // count this warp's 32 rows of the part in; the warp completing the s
                // arrivals of its quarter of the tile sums those rows' parts in part
                // order (the four quarters in parallel, no barrier between warps)
                const int tq = (piece / S.s) * 4 + q;
                __threadfence();
                __syncwarp();
                int last = 0;
                if (lane == 0) {
                    const int old = atomicAdd(&cnt[tq], 1);
                    last = (old == S.s - 1);
                    if (last) cnt[tq] = 0;  // ready for the next launch
                }
                last = __shfl_sync(0xffffffffu, last, 0);
                if (last) {
                    __threadfence();
                    const float *w0 = work + (size_t)(piece / S.s) * S.s * BM * BN + (size_t)q * 32 * BN;
                    // 32 rows x 64 float4: lanes along a row, 8 float4 a lane in flight per part
#pragma unroll 1
                    for (int f0 = 0; f0 < 32 * BN / 4; f0 += 8 * 32) {
                        float4 v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) v[u] = __ldcg((const float4 *)w0 + f0 + u * 32 + lane);
                        for (int j = 1; j < S.s; ++j) {
                            float4 x[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                x[u] = __ldcg((const float4 *)(w0 + (size_t)j * BM * BN) + f0 + u * 32 + lane);
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                v[u].x += x[u].x; v[u].y += x[u].y; v[u].z += x[u].z; v[u].w += x[u].w;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int f = f0 + u * 32 + lane;
                            const int grow = m0 + q * 32 + f / (BN / 4), gcol = n0 + (f % (BN / 4)) * 4;
                            if (grow < M) {
                                float *dst = D + (size_t)grow * N + gcol;
                                if (gcol + 4 <= N && (N & 3) == 0) {
                                    *(float4 *)dst = v[u];
                                } else {
                                    const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                                    for (int j = 0; j < 4; ++j)
                                        if (gcol + j < N) dst[j] = vv[j];
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    __syncwarp();
    if (*abort_flag && threadIdx.x == 0) {
        atomicOr(status, 2);
        // give TMA copies still in flight time to land before the CTA exits
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 10000000ull) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

bool encode(CUtensorMap *map, const uint16_t *base, size_t rows, long long ld, int box_rows, std::string *why)
{
    auto fn = encode_fn();
    if (!fn) {
        if (why) *why = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (why) *why = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}


// ---------------------------------------------------------------------------
// Grouped, persistent variant for a pool of matrices: CTAs walk a device tile
// table (matrix, m0, n0); each matrix has its own pair of tensor maps in
// global memory and its own output.  Warps: 0 = TMA producer, 1 = MMA issuer,
// 2..5 = epilogue (warp w reads TMEM lanes 32*(w%4) .. +31).  The smem ring's
// stage/phase counters run on across tiles.  Two 256-column accumulators in
// TMEM alternate between tiles (tmem_full / tmem_empty per accumulator), so
// the MMAs of one tile run while the epilogue drains the previous one.  A
// matrix whose output is marked `add` has the tile added to D (the products of
// several steps summed before one fold).  Each 32 x 32 chunk of the epilogue
// goes through a staging square in shared memory, so that D is written (and,
// to add, read) row by row, 32 consecutive columns a warp instruction.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(192, 1)
    tc_gemm_grouped_kernel(const GroupTile *__restrict__ tiles, const int *__restrict__ ntiles_p,
                           const CUtensorMap *__restrict__ maps, const GroupOut *__restrict__ outs, int *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;  // [2]
    uint64_t *tempty = tfull + 2;       // [2]
    uint32_t *tmem_slot = (uint32_t *)(tempty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = *ntiles_p;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int kg = 0;  // k-slices issued so far (ring position)
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const GroupTile tile = tiles[t];
                const CUtensorMap *ma = &maps[2 * tile.slot], *mb = &maps[2 * tile.slot + 1];
                const int kt_n = outs[tile.slot].ktiles;
                for (int kt = 0; kt < kt_n; ++kt, ++kg) {
                    const int s = kg % STAGES;
                    const uint32_t phase = (uint32_t)(kg / STAGES) & 1u;
                    if (kg >= STAGES && !mbar_wait(smem_u32(&empty[s]), phase ^ 1u, abort_flag)) break;
                    mbar_expect_tx(smem_u32(&full[s]), STAGE_BYTES);
                    tma_load_2d(smem_u32(sA + s * A_BYTES), ma, smem_u32(&full[s]), kt * BK, tile.m0);
                    tma_load_2d(smem_u32(sB + s * B_BYTES), mb, smem_u32(&full[s]), kt * BK, tile.n0);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int kg = 0, tl = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tl) {
                const int kt_n = outs[tiles[t].slot].ktiles;
                const int ab = tl & 1;  // this tile's accumulator
                const uint32_t acc = tmem + (uint32_t)(ab * TMEM_COLS);
                // the epilogue must have drained this accumulator (two tiles ago)
                if (tl >= 2 && !mbar_wait(smem_u32(&tempty[ab]), (uint32_t)((tl >> 1) - 1) & 1u, abort_flag)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool ok = true;
                for (int kt = 0; kt < kt_n; ++kt, ++kg) {
                    const int s = kg % STAGES;
                    const uint32_t phase = (uint32_t)(kg / STAGES) & 1u;
                    if (!mbar_wait(smem_u32(&full[s]), phase, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t a = sdesc(smem_u32(sA + s * A_BYTES));
                    const uint64_t b = sdesc(smem_u32(sB + s * B_BYTES));
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(acc, a + 2 * kk, b + 2 * kk, (kt > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(smem_u32(&empty[s]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&tfull[ab]));
            }
        }
    } else {
        // epilogue warps 2..5
        const int q = warp & 3;
        float *stage = (float *)(smem + STAGES * STAGE_BYTES + 256) + q * 32 * 33;
        int tl = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
            const GroupTile tile = tiles[t];
            const GroupOut o = outs[tile.slot];
            const int ab = tl & 1;
            const bool have = __all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[ab]), (uint32_t)(tl >> 1) & 1u, abort_flag));
            if (!have) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t)(ab * TMEM_COLS) + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
                // D = (or +=) the chunk, through this warp's 32 x 33 staging square, so
                // that a warp instruction reads and writes 32 consecutive columns of one row
#pragma unroll
                for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
                __syncwarp();
                const int col = tile.n0 + c0 + lane;
#pragma unroll 1
                for (int r0 = 0; r0 < 32; r0 += 16) {
                    // the 16 rows' loads first (independent), then the adds and stores
                    float dv[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int grow = tile.m0 + q * 32 + r0 + u;
                        dv[u] = (o.add && grow < o.M && col < o.N) ? __ldcg(o.D + (size_t)grow * o.N + col) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int grow = tile.m0 + q * 32 + r0 + u;
                        if (grow < o.M && col < o.N)
                            o.D[(size_t)grow * o.N + col] = dv[u] + stage[(r0 + u) * 33 + lane];
                    }
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[ab])) : "memory");
        }
    }
    __syncwarp();
    if (*abort_flag && threadIdx.x == 0) {
        atomicOr(status, 2);
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 10000000ull) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS));
}

}  // namespace

bool tc_encode_operand(CUtensorMap *map, const uint16_t *base, long long rows, long long ld, long long inner,
                       bool is_b, const char **why)
{
    auto fn = encode_fn();
    if (!fn) {
        if (why) *why = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)(is_b ? BN : BM)};
    cuuint32_t estr[2] = {1, 1};
    if (fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        if (why) *why = "cuTensorMapEncodeTiled rejected an operand";
        return false;
    }
    return true;
}

cudaError_t tc_gemm_grouped_run(const GroupTile *tiles, const int *ntiles, const CUtensorMap *maps, const GroupOut *outs,
                                int grid, int *status, cudaStream_t s)
{
    // the ring, its barriers, and four 32 x 33 FP32 staging squares for D += A B^T
    const int smem = STAGES * STAGE_BYTES + 1024 + 256 + 4 * 32 * 33 * 4;
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc_gemm_grouped_kernel<<<grid, 192, smem, s>>>(tiles, ntiles, maps, outs, status);
    return cudaGetLastError();
}

namespace {
}  // namespace

// Split a last, partly filled wave only when a tile is long enough for the
// parts' fix-up (a read of every part's 128 KB) to cost less than the wait for
// whole tiles: 512 k-slices of 64 are about 0.17 ms of tensor-core time a tile.
constexpr int kSplitMinKtiles = 512;
// at most this many parts a tile, so that the fix-up's reads stay short
constexpr long long kSplitMaxParts = 16;

struct TcGemmPlan {
    CUtensorMap ta, tb;
    float *D;
    long long M, N, ld;
    int sms;        // CTAs of the persistent grid (one per SM)
    float *work;    // sms partial 128 x 256 tiles of a split last wave
    int *cnt;       // arrivals per (split tile, 32-row quarter)
};

TcGemmPlan *tc_gemm_plan_create(const uint16_t *A, size_t a_rows, const uint16_t *B, size_t b_rows,
                                long long ld, float *D, long long M, long long N, std::string *why)
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        if (why) *why = "no CUDA device";
        return nullptr;
    }
    if (major != 10 || minor != 3) {
        if (why) *why = "the tcgen05 contraction is built for sm_103a only";
        return nullptr;
    }
    if (ld % BK || a_rows % BM || b_rows % BN || (long long)a_rows < M || (long long)b_rows < N ||
        ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || M > (1LL << 31) || N > (1LL << 31)) {
        if (why) *why = "unsupported shape or alignment";
        return nullptr;
    }
    TcGemmPlan *p = new TcGemmPlan;
    std::memset(p, 0, sizeof *p);
    if (!encode(&p->ta, A, a_rows, ld, BM, why) || !encode(&p->tb, B, b_rows, ld, BN, why)) {
        delete p;
        return nullptr;
    }
    if (cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(tc_gemm_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
            cudaSuccess) {
        if (why) *why = "cannot reserve shared memory";
        delete p;
        return nullptr;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    p->sms = sms;
    if (cudaMalloc((void **)&p->work, (size_t)sms * BM * BN * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&p->cnt, (size_t)sms * 4 * sizeof(int)) != cudaSuccess ||
        cudaMemset(p->cnt, 0, (size_t)sms * 4 * sizeof(int)) != cudaSuccess) {
        if (why) *why = "cannot allocate the split-tile workspace";
        cudaFree(p->work);
        cudaFree(p->cnt);
        delete p;
        return nullptr;
    }
    p->D = D;
    p->M = M;
    p->N = N;
    p->ld = ld;
    return p;
}

cudaError_t tc_gemm_run(TcGemmPlan *p, long long inner, int *status, cudaStream_t s)
{
    if (!p || inner <= 0 || inner % BK || inner > p->ld) return cudaErrorInvalidValue;
    const long long MT = (p->M + BM - 1) / BM, NT = (p->N + BN - 1) / BN, T = MT * NT;
    if (T > (1LL << 30)) return cudaErrorInvalidValue;
    const int ktiles = (int)(inner / BK);
    const int G = (int)std::min<long long>(T, p->sms);
    const long long R = T / G, r = T % G;
    PersistSched S;
    S.NT = (int)NT;
    S.ktiles = ktiles;
    S.s = 1;
    S.Tfull = (int)T;
    S.npieces = 0;
    if (R >= 1 && r > 0 && 2 * r <= G && ktiles >= kSplitMinKtiles) {
        // a last wave of r tiles on G CTAs: split each into G / r parts
        S.s = (int)std::min<long long>(std::min<long long>(G / r, kSplitMaxParts), ktiles);
        S.Tfull = (int)(R * G);
        S.npieces = (int)(r * S.s);
        // a contraction abandoned after an expired wait leaves its counts behind
        cudaError_t e = cudaMemsetAsync(p->cnt, 0, (size_t)r * 4 * sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    tc_gemm_persistent_kernel<<<G, 192, SMEM_BYTES, s>>>(p->ta, p->tb, p->D, (int)p->M, (int)p->N, S, p->work,
                                                         p->cnt, status);
    return cudaGetLastError();
}

void tc_gemm_plan_destroy(TcGemmPlan *p)
{
    if (!p) return;
    cudaFree(p->work);
    cudaFree(p->cnt);
    delete p;
}

cudaError_t tc_gemm_run_direct(const uint16_t *A, long long lda, const uint16_t *B, long long ldb, long long M,
                               long long N, long long inner, float *D, int *status, cudaStream_t s,
                               const char **why)
{
    // the tensor maps live on this stack frame and are passed by value to the
    // kernel; their extents are the true M, N and inner, so TMA fills the
    // ragged edges of the last tiles with zeros
    auto fn = encode_fn();
    if (!fn) {
        if (why) *why = "cuTensorMapEncodeTiled unavailable";
        return cudaErrorNotSupported;
    }
    CUtensorMap ta, tb;
    const uint16_t *bases[2] = {A, B};
    const long long lds[2] = {lda, ldb}, rows[2] = {M, N};
    const int boxr[2] = {BM, BN};
    CUtensorMap *maps[2] = {&ta, &tb};
    for (int k = 0; k < 2; ++k) {
        cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows[k]};
        cuuint64_t strides[1] = {(cuuint64_t)lds[k] * 2};
        cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)boxr[k]};
        cuuint32_t estr[2] = {1, 1};
        if (fn(maps[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)bases[k], dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            if (why) *why = "cuTensorMapEncodeTiled rejected an operand (base must be 16-byte aligned, ld a multiple of 8)";
            return cudaErrorInvalidValue;
        }
    }
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
    tc_gemm_kernel<<<grid, 128, SMEM_BYTES, s>>>(ta, tb, D, (int)M, (int)N, (int)((inner + BK - 1) / BK), status);
    return cudaGetLastError();
}

}  // namespace mcinv
