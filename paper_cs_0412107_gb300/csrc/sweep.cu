// sweep.cu -- the hot path of the correlated-chains sampler on sm_103a:
//   * the Z2 noise plane (Philox4x32-10, Eqs. 5a/5b),
//   * the per-row constants of Eqs. 4/5 formed in FP64,
//   * the coupled noisy Gauss-Seidel sweep of Eqs. 4 and 5 for a slice of
//     chains per CTA, with the z_i conj(w_i) diagonal partials (Eq. 1/C)
//     and the BF16 shadows for the tensor-core block contraction fused in.
#include <cuda_bf16.h>

#include "internal.h"
#include "sweep_core.cuh"

namespace mcinv {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by two fixed odd constants, swaps the high halves
// across (xored with the other words and the round key), and the key is
// advanced by a Weyl sequence between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k)
{
    const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kMul0, x.x), lo0 = kMul0 * x.x;
        const uint32_t hi1 = __umulhi(kMul1, x.z), lo1 = kMul1 * x.z;
        x = make_uint4(hi1 ^ x.y ^ k.x, lo1, hi0 ^ x.w ^ k.y, lo0);
        k.x += kWeyl0;
        k.y += kWeyl1;
    }
    return x;
}

// Noise plane for cycles cycle0 .. cycle0+ncyc-1: out[cyc][cw][pos[row]] holds
// the sign bits of chains 32cw .. 32cw+31 at `row`.  One Philox call yields
// the 128 bits of rows 128rb .. 128rb+127 of one chain (row r -> bit r%32 of
// word (r/32)%4); a warp of 32 chains transposes each of its four 32 x 32 bit
// blocks (lane = chain, bit = row) so every word is written once.  The plane
// is stored by position so the sweep reads it coalesced.
__global__ void __launch_bounds__(128) noise_kernel(uint64_t seed, uint32_t matrix,
                                                    uint64_t chain_base, int K, int n, int nw,
                                                    uint32_t cycle0, const int *__restrict__ pos,
                                                    uint32_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int cw = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (cw >= nw) return;  // whole warp
    const int rb = blockIdx.x, cyc = blockIdx.z;
    const int chain = cw * 32 + lane;
    const uint4 r = philox4x32_10(
        make_uint4((uint32_t)rb, (uint32_t)(chain_base + (uint64_t)chain), cycle0 + (uint32_t)cyc, matrix),
        make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)));
    const bool valid = chain < K;
    const uint32_t xs[4] = {r.x, r.y, r.z, r.w};
    uint32_t *dst = out + ((size_t)cyc * nw + cw) * (size_t)n;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // the 32 x 32 bit block (lane i, bit j) transposed by halving block swaps: at
        // width s each lane trades the half of its word whose bit index has bit s unlike
        // its own lane index with the lane s away; lane j ends with bit i = block (i, j)
        uint32_t x = valid ? xs[q] : 0u;
#pragma unroll
        for (int sw = 16; sw > 0; sw >>= 1) {
            const uint32_t m = sw == 16 ? 0x0000ffffu : sw == 8 ? 0x00ff00ffu : sw == 4 ? 0x0f0f0f0fu
                               : sw == 2 ? 0x33333333u : 0x55555555u;  // bits j with (j & sw) == 0
            const uint32_t t = __shfl_xor_sync(0xffffffffu, x, sw);
            x = (lane & sw) ? ((x & ~m) | ((t >> sw) & m)) : ((x & m) | ((t & m) << sw));
        }
        const int row = rb * 128 + q * 32 + lane;
        if (row < n) dst[pos[row]] = x;
    }
}

cudaError_t launch_noise(uint64_t seed, uint32_t matrix, uint64_t chain_base, int K, int n,
                         uint32_t cycle0, int ncyc, const int *pos, uint32_t *out, cudaStream_t s)
{
    const int nw = (K + 31) / 32;
    dim3 grid((n + 127) / 128, (nw + 3) / 4, ncyc);
    noise_kernel<<<grid, 128, 0, s>>>(seed, matrix, chain_base, K, n, nw, cycle0, pos, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-row constants in FP64: inv_d = 1/c_ii, alpha = 1/sqrt(c_ii),
// beta = 1/conj(sqrt(c_ii)) (Eq. 5's 1/sqrt(c*_ii) read so that
// alpha conj(beta) = 1/c_ii).  Real storage with c_ii < 0 keeps real
// arithmetic: alpha = 1/sqrt|c|, beta = -1/sqrt|c|.
// ---------------------------------------------------------------------------
__device__ inline double2 crecip64(double a, double b)
{
    // 1/(a+ib) with the operands scaled by max(|a|,|b|) to avoid overflow
    const double m = fmax(fabs(a), fabs(b));
    const double x = a / m, y = b / m;
    const double den = m * (x * x + y * y);
    return make_double2(x / den, -y / den);
}

__device__ inline double2 csqrt64(double a, double b)
{
    // principal square root: the result has a non-negative real part, and the
    // sign of its imaginary part follows the sign of b (including -0)
    const double r = hypot(a, b);
    if (r == 0.0) return make_double2(0.0, b);
    if (a >= 0.0) {
        const double t = sqrt(0.5 * (r + a));
        return make_double2(t, b / (2.0 * t));
    }
    const double t = sqrt(0.5 * (r - a));
    return make_double2(fabs(b) / (2.0 * t), copysign(t, b));
}

__global__ void constants_kernel(int n, const double *__restrict__ diag, int cplx, uint8_t *stream,
                                 const long long *__restrict__ cst_at, int *bad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (!cplx) {
        const double c = diag[p];
        if (!(c != 0.0) || !isfinite(c)) { atomicMin(bad, p); return; }
        const double r = sqrt(fabs(c));
        CstR k;
        k.alpha = (float)(1.0 / r);
        k.beta = (float)((c > 0.0 ? 1.0 : -1.0) / r);
        k.inv_d = (float)(1.0 / c);
        k.pad = 0.f;
        *(CstR *)(stream + cst_at[p]) = k;
    } else {
        const double a = diag[2 * p], b = diag[2 * p + 1];
        if (!isfinite(a) || !isfinite(b) || (a == 0.0 && b == 0.0)) { atomicMin(bad, p); return; }
        const double2 s = csqrt64(a, b);
        const double2 al = crecip64(s.x, s.y);
        const double2 be = crecip64(s.x, -s.y);
        const double2 d = crecip64(a, b);
        CstC k;
        k.alpha = make_float2((float)al.x, (float)al.y);
        k.beta = make_float2((float)be.x, (float)be.y);
        k.inv_d = make_float2((float)d.x, (float)d.y);
        k.pad = make_float2(0.f, 0.f);
        *(CstC *)(stream + cst_at[p]) = k;
    }
}

cudaError_t launch_constants(int n, const double *diag, int cplx, uint8_t *stream,
                             const long long *cst_at, int *bad, cudaStream_t s)
{
    constants_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, diag, cplx, stream, cst_at, bad);
    return cudaGetLastError();
}

template <bool CPLX, int LPR, int V, int U, bool CLUSTER>
__global__ void __launch_bounds__(512, 1) cc_sweep_kernel(const SweepArgs a)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    constexpr int RPW = 32 / LPR;  // rows per warp instruction
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bars = (uint64_t *)(smem + 2 * (size_t)a.blob_max);
    volatile int *abort_flag = (volatile int *)(bars + 2);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int sub = lane / LPR;
    const int cl = lane % LPR;
    const int Q = CLUSTER ? a.ctas_per_slice : 1;
    const int rank = CLUSTER ? (int)cluster_rank() : 0;
    const int slice = blockIdx.x / Q;
    const int c0 = (slice * LPR + cl) * V;  // first chain of this lane (K % V == 0)
    const bool chain_ok = c0 < a.K;
    const size_t K = (size_t)a.K;
    const int stride = Q * nwarps * RPW;
    const int first = (rank * nwarps + warp) * RPW;
    const uint32_t cshift = (uint32_t)(c0 & 31);
    const int seg = a.seg;
    S *dpart = (S *)a.diag_part + (size_t)(c0 / (seg * V)) * a.n;
    const bool dlead = (cl % seg) == 0;
    const int total = a.ncyc * a.nchunks;

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[1])));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (total > 0) {
            const ChunkDesc d = a.chunks[0];
            stage_chunk(smem_addr(smem), a.stream + d.off, (uint32_t)d.bytes, smem_addr(&bars[0]));
        }
    }
    __syncthreads();

    bool diverged = false;
    bool level_end = false;  // did the previous chunk end a dependency level?
    float tsum = 0.f;        // this lane's share of the cycle's trace series value
    for (int t = 0; t < total; ++t) {
        const int cyc = t / a.nchunks;
        const int b = t & 1;
        const ChunkDesc d = a.chunks[t - cyc * a.nchunks];
        const int cur = a.cur ^ (cyc & 1);
        const T *zo = (const T *)a.z[cur];
        T *zn = (T *)a.z[cur ^ 1];
        const T *wo = (const T *)a.w[cur];
        T *wn = (T *)a.w[cur ^ 1];
        const uint8_t *buf = smem + (size_t)b * a.blob_max;
        // One thread observes chunk t's arrival; one barrier then publishes it
        // to the CTA, ends chunk t-1 (its buffer is free again) and, after a
        // level, is the cluster barrier that makes the level's rows visible to
        // every CTA of the slice.
        if (threadIdx.x == 0 && !*abort_flag && !wait_chunk(smem_addr(&bars[b]), (uint32_t)(t >> 1) & 1u))
            *abort_flag = 1;
        if constexpr (CLUSTER) {
            if (level_end) cluster_barrier();
            else __syncthreads();
        } else {
            __syncthreads();
        }
        level_end = (d.flags & CHUNK_LEVEL_END) != 0;
        if (threadIdx.x == 0 && t + 1 < total && !*abort_flag) {
            // order the CTA's generic-proxy reads of that buffer before the
            // async-proxy write of the next blob
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const ChunkDesc dn = a.chunks[(t + 1) % a.nchunks];
            stage_chunk(smem_addr(smem + (size_t)(b ^ 1) * a.blob_max), a.stream + dn.off, (uint32_t)dn.bytes,
                        smem_addr(&bars[b ^ 1]));
        }
        if (!*abort_flag) {
            ChunkWork w;
            w.buf = buf; w.d = d;
            w.zo = zo; w.zn = zn; w.wo = wo; w.wn = wn;
            w.noise = a.noise ? a.noise + ((size_t)cyc * a.nw + (size_t)(c0 >> 5)) * (size_t)a.n : nullptr;
            w.dpart = dpart; w.diag = a.diag_part != nullptr; w.dlead = dlead; w.seg = seg;
            w.rpos = a.rpos; w.spos = a.spos; w.zsh = a.zsh; w.wsh = a.wsh; w.ldsh = a.ldsh; w.kp = a.kp;
            w.shcol = a.cyc0_in_batch + cyc;
            w.K = K; w.c0 = c0; w.first = first; w.stride = stride; w.sub = sub;
            w.chain_ok = chain_ok; w.cshift = cshift;
            w.tq = a.tq;
            diverged |= sweep_chunk_rows<CPLX, LPR, V, U, CLUSTER>(w, &tsum);
            if (a.tpart && (t + 1) % a.nchunks == 0) {
                // end of a cycle: this warp's partial of the trace series, reduced in a
                // fixed order, one slot per (cycle, CTA, warp)
                float v = tsum;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0) a.tpart[((size_t)cyc * gridDim.x + blockIdx.x) * nwarps + warp] = v;
                tsum = 0.f;
            }
        }
    }
    // the last chunk's rows are done before anyone leaves (the cluster's CTAs
    // may still read them through the cluster-wide view until then)
    if constexpr (CLUSTER) cluster_barrier();
    if (diverged) atomicOr(a.status, 1);
    if (threadIdx.x == 0 && *abort_flag) {
        atomicOr(a.status, 4);
        const uint64_t t0 = gtimer();  // let copies still in flight land before exit
        while (gtimer() - t0 < 10000000ull) {
        }
    }
}

static size_t sweep_smem(int blob_max) { return 2 * (size_t)blob_max + 64; }

template <bool CPLX, int LPR, int V, int U, bool CL>
static cudaError_t prepare(int blob_max, int q)
{
    auto kern = cc_sweep_kernel<CPLX, LPR, V, U, CL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem(blob_max));
    if (e == cudaSuccess && CL && q > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <bool CPLX, int LPR, int V, int U>
static cudaError_t launch_one(const SweepArgs &a, int slices, int threads, cudaStream_t s)
{
    const size_t smem = sweep_smem(a.blob_max);
    if (a.ctas_per_slice <= 1) {
        cudaError_t e = prepare<CPLX, LPR, V, U, false>(a.blob_max, 1);
        if (e != cudaSuccess) return e;
        cc_sweep_kernel<CPLX, LPR, V, U, false><<<slices, threads, smem, s>>>(a);
        return cudaGetLastError();
    }
    cudaError_t e = prepare<CPLX, LPR, V, U, true>(a.blob_max, a.ctas_per_slice);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(slices * a.ctas_per_slice));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.ctas_per_slice;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cc_sweep_kernel<CPLX, LPR, V, U, true>, a);
}

template <bool CPLX, int V, int U>
static cudaError_t launch_sweep_v(const SweepArgs &a, int LPR, int slices, int threads, cudaStream_t s)
{
    switch (LPR) {
    case 1: return launch_one<CPLX, 1, V, U>(a, slices, threads, s);
    case 2: return launch_one<CPLX, 2, V, U>(a, slices, threads, s);
    case 4: return launch_one<CPLX, 4, V, U>(a, slices, threads, s);
    case 8: return launch_one<CPLX, 8, V, U>(a, slices, threads, s);
    case 16: return launch_one<CPLX, 16, V, U>(a, slices, threads, s);
    case 32: return launch_one<CPLX, 32, V, U>(a, slices, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep(const SweepArgs &a, int cplx, int lanes_per_row, int chains_per_lane,
                         int slices, int threads, cudaStream_t s)
{
    if (cplx) {
        if (chains_per_lane == 2) return launch_sweep_v<true, 2, 8>(a, lanes_per_row, slices, threads, s);
        if (chains_per_lane == 1) return launch_sweep_v<true, 1, 8>(a, lanes_per_row, slices, threads, s);
    } else {
        if (chains_per_lane == 4) return launch_sweep_v<false, 4, 8>(a, lanes_per_row, slices, threads, s);
        if (chains_per_lane == 1) return launch_sweep_v<false, 1, 8>(a, lanes_per_row, slices, threads, s);
    }
    return cudaErrorInvalidValue;
}

int max_active_clusters(int cplx, int lanes_per_row, int chains_per_lane, int threads, int q, int blob_max)
{
    // how many clusters of q CTAs can be resident at once (0 if none)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)q);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = sweep_smem(blob_max);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const void *k = nullptr;
    cudaError_t e = cudaErrorInvalidValue;
#define MCINV_PICK(C, L, V, U)                                                     \
    if (cplx == C && lanes_per_row == L && chains_per_lane == V) {                   \
        k = (const void *)cc_sweep_kernel<C, L, V, U, true>;                         \
        e = prepare<C, L, V, U, true>(blob_max, q);                                  \
    }
#define MCINV_PICK_L(C, V, U) MCINV_PICK(C, 1, V, U) MCINV_PICK(C, 2, V, U) MCINV_PICK(C, 4, V, U) \
    MCINV_PICK(C, 8, V, U) MCINV_PICK(C, 16, V, U) MCINV_PICK(C, 32, V, U)
    MCINV_PICK_L(true, 2, 8)
    MCINV_PICK_L(true, 1, 8)
    MCINV_PICK_L(false, 4, 8)
    MCINV_PICK_L(false, 1, 8)
#undef MCINV_PICK_L
#undef MCINV_PICK
    if (!k || e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace mcinv
