// pool.cu -- many matrices advanced together (the batched form) and the
// continuous-batching engine the server runs on.
//
// A pool owns one device-memory arena (a single cudaMalloc at creation) and a
// set of slots.  A matrix admitted into a slot gets its chunk stream, chain
// state, noise plane, accumulators and (for the full inverse) BF16 shadows
// and products carved out of the arena by a host-side first-fit allocator;
// admission fails with MCINV_E_NOMEM when they do not fit, and the caller
// queues the request.  Every step advances every admitted matrix by B cycles
// (burn-in or sampling by its own schedule) with a fixed sequence of
// persistent kernels that read their work from device tables:
//   noise  : (slot, 128-row block) entries -> Philox noise planes
//   sweep  : (slot, chain slice) work items pulled from a device queue: the
//            chain-sliced row arithmetic over the chunk stream, or (the ring
//            form) a CTA per (slot, 128-chain block) whose warps take the rows
//            of each level with bulk-staged gathers (sweep_ring.cuh), a CTA
//            barrier between levels
//   block  : grouped tcgen05 contraction over (slot, 128x256 tile) entries
//   fold   : block and diagonal FP64 folds over (slot, range) segments
// so the step is captured once as a CUDA graph and replayed whatever the
// membership; the host only rewrites the tables between steps.  Matrices are
// independent and every reduction has a fixed order, so a matrix's results do
// not depend on what else is in the pool.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/mcinv.h"
#include "internal.h"
#include "prepare.h"
#include "sweep_core.cuh"
#include "sweep_ring.cuh"
#include "tc_gemm.h"

namespace mcinv {

// ---------------------------------------------------------------------------
// device tables
// ---------------------------------------------------------------------------
struct PoolSlotDev {
    const uint8_t *stream;
    const ChunkDesc *chunks;
    const int *perm, *pos;
    float *z[2], *w[2];          // z[1] = z[0] + n K (one allocation), same for w
    // the flat form for the ring form (see internal.h GridRow): records with
    // .row = i K / 4, entries per cycle parity (.col: vector index from z[0]),
    // constants by position, the first position of every level
    const GridRow *grows;
    const EntR *gzent[2], *gwent[2];
    const CstR *gcst;
    const int *levptr;
    int nlev;
    uint32_t *noise;    // [B][nw][n] by position
    float *dpart;       // [units][n] by position
    double *dacc;       // [G][n] by position
    uint16_t *zsh, *wsh;
    float *D;
    double *bsum, *bsq;
    long long ldsh, kp;
    int n, nchunks;
    uint32_t matrix_id, cycle0;  // Philox matrix word; global cycle of this step's first cycle
    int cur;                     // state buffer before this step
    int nb, ns;                  // burn-in and sampling cycles this step
    int inverse;                 // accumulate the full inverse
    double scale_sq;             // 1 / (K^2 ns)
};
struct PoolItem {
    int slot, slice;
};
struct PoolRB {
    int slot, rb;
};
struct PoolSeg {
    int slot, kind;  // kind 0: block elements, 1: diagonal positions
    long long begin, count;
};
struct PoolCounts {
    int items, rbs, tiles, segs;
    int queue;  // work-queue head of the sweep (reset every step)
    int pad[3];
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 pool_philox(uint4 x, uint2 k)
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

// Noise planes of every slot for this step's cycles (same bit layout as the
// single-matrix noise kernel): a CTA of 4 warps takes one (slot, row block).
__global__ void __launch_bounds__(128) pool_noise_kernel(const PoolSlotDev *__restrict__ slots,
                                                         const PoolRB *__restrict__ rbs, const PoolCounts *cnt,
                                                         uint64_t seed, uint64_t chain_base, int K, int nw)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    for (int e = blockIdx.x; e < cnt->rbs; e += gridDim.x) {
        const PoolRB rb = rbs[e];
        const PoolSlotDev &S = slots[rb.slot];
        const int ncyc = S.nb + S.ns;
        for (int cyc = 0; cyc < ncyc; ++cyc) {
            for (int cw = warp; cw < nw; cw += 4) {
                const int chain = cw * 32 + lane;
                const uint4 r = pool_philox(
                    make_uint4((uint32_t)rb.rb, (uint32_t)(chain_base + (uint64_t)chain), S.cycle0 + (uint32_t)cyc, S.matrix_id),
                    key);
                const bool valid = chain < K;
                const uint32_t xs[4] = {r.x, r.y, r.z, r.w};
                uint32_t *dst = S.noise + ((size_t)cyc * nw + cw) * (size_t)S.n;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // the 32 x 32 bit block (lane = chain, bit = row) transposed by halving block
                    // swaps, as in the single-matrix noise plane
                    uint32_t x = valid ? xs[q] : 0u;
#pragma unroll
                    for (int sw = 16; sw > 0; sw >>= 1) {
                        const uint32_t m = sw == 16 ? 0x0000ffffu : sw == 8 ? 0x00ff00ffu : sw == 4 ? 0x0f0f0f0fu
                                           : sw == 2 ? 0x33333333u : 0x55555555u;  // bits j with (j & sw) == 0
                        const uint32_t t = __shfl_xor_sync(0xffffffffu, x, sw);
                        x = (lane & sw) ? ((x & ~m) | ((t >> sw) & m)) : ((x & m) | ((t & m) << sw));
                    }
                    const int row = rb.rb * 128 + q * 32 + lane;
                    if (row < S.n) dst[S.pos[row]] = x;
                }
            }
        }
    }
}

// Persistent sweep: CTAs pull (slot, chain slice) items from the device queue
// and run the slot's burn-in then sampling cycles of this step over its chunk
// stream, with the same row arithmetic as the single-matrix sweep.
template <int LPR, int V, int U>
__global__ void __launch_bounds__(512, 1) pool_sweep_kernel(const PoolSlotDev *__restrict__ slots,
                                                            const PoolItem *__restrict__ items, PoolCounts *cnt,
                                                            int K, int nw, int blob_max, int seg, int *status)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bars = (uint64_t *)(smem + 2 * (size_t)blob_max);
    volatile int *abort_flag = (volatile int *)(bars + 2);
    volatile int *item_slot = abort_flag + 1;
    constexpr int RPW = 32 / LPR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int sub = lane / LPR, cl = lane % LPR;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[1])));
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int g = 0;  // chunks staged so far by this CTA: buffer g & 1, parity (g >> 1) & 1
    bool diverged = false;
    for (;;) {
        if (threadIdx.x == 0) *item_slot = atomicAdd(&cnt->queue, 1);
        __syncthreads();
        const int it = *item_slot;
        if (it >= cnt->items || *abort_flag) break;
        const PoolItem item = items[it];
        const PoolSlotDev &S = slots[item.slot];
        const int c0 = (item.slice * LPR + cl) * V;
        const bool chain_ok = c0 < K;
        const int ncyc = S.nb + S.ns;
        const int total = ncyc * S.nchunks;
        if (threadIdx.x == 0 && total > 0) {
            const ChunkDesc d = S.chunks[0];
            stage_chunk(smem_addr(smem + (size_t)(g & 1) * blob_max), S.stream + d.off, (uint32_t)d.bytes,
                        smem_addr(&bars[g & 1]));
        }
        for (int t = 0; t < total; ++t, ++g) {
            const int cyc = t / S.nchunks;
            const int b = g & 1;
            const ChunkDesc d = S.chunks[t - cyc * S.nchunks];
            const int cur = S.cur ^ (cyc & 1);
            if (threadIdx.x == 0 && !*abort_flag && !wait_chunk(smem_addr(&bars[b]), (uint32_t)(g >> 1) & 1u))
                *abort_flag = 1;
            __syncthreads();
            if (threadIdx.x == 0 && t + 1 < total && !*abort_flag) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const ChunkDesc dn = S.chunks[(t + 1) % S.nchunks];
                stage_chunk(smem_addr(smem + (size_t)(b ^ 1) * blob_max), S.stream + dn.off, (uint32_t)dn.bytes,
                            smem_addr(&bars[b ^ 1]));
            }
            if (*abort_flag) continue;
            const bool acc = cyc >= S.nb;
            ChunkWork w;
            w.buf = smem + (size_t)b * blob_max;
            w.d = d;
            w.zo = S.z[cur]; w.zn = S.z[cur ^ 1]; w.wo = S.w[cur]; w.wn = S.w[cur ^ 1];
            w.noise = S.noise + ((size_t)cyc * nw + (size_t)(c0 >> 5)) * (size_t)S.n;
            w.diag = acc;
            w.dpart = S.dpart + (size_t)(c0 / (seg * V)) * S.n;
            w.dlead = (cl % seg) == 0;
            w.seg = seg;
            const bool sh = acc && S.inverse;
            w.rpos = sh ? S.perm : nullptr;  // full inverse: R = S = every row in order
            w.spos = sh ? S.perm : nullptr;
            w.zsh = S.zsh; w.wsh = S.wsh; w.ldsh = S.ldsh; w.kp = S.kp;
            w.shcol = cyc - S.nb;
            w.K = (size_t)K;
            w.c0 = c0;
            w.first = warp * RPW;
            w.stride = nwarps * RPW;
            w.sub = sub;
            w.chain_ok = chain_ok;
            w.cshift = (uint32_t)(c0 & 31);
            w.tq = nullptr;
            float tdummy = 0.f;
            diverged |= sweep_chunk_rows<false, LPR, V, U, false>(w, &tdummy);
        }
        __syncthreads();  // the item's last chunk is done before its buffers are reused
    }
    if (diverged) atomicOr(status, 1);
    if (threadIdx.x == 0 && *abort_flag) {
        atomicOr(status, 4);
        const uint64_t t0 = gtimer();
        while (gtimer() - t0 < 10000000ull) {
        }
    }
}

// The ring form of the sweep: a CTA of NT / 32 warps takes a (slot, chain
// block) item from the device queue and runs the slot's cycles of this step;
// warp w takes the rows lb + w, lb + w + NT / 32, ... of each level with
// bulk-staged gathers (ring::level_bulk, the same arithmetic), and a CTA
// barrier ends every level: the whole chain block of the matrix is this CTA's.
// Shapes: 12 warps of 32 slots or 16 warps of 24 slots of 512 bytes for a
// 128-chain block (G = 1), or 12 warps of 18 slots of 1 KB for a 256-chain
// block (G = 2: two vectors a lane, the row's fixed work paid once for both).
// The warps' rings, barriers and their phases persist across items.
template <int NT, int G>
constexpr int pool_ring_slots() { return G == 2 ? 18 : NT == 512 ? ring::RING16 : ring::RING; }
template <int NT, int G>
constexpr size_t pool_ring_smem()
{
    return (size_t)(NT / 32) * (pool_ring_slots<NT, G>() * ring::SEGB * G + ring::NBAR * sizeof(uint64_t));
}

template <int NT, int G>
__global__ void __launch_bounds__(NT, 1) pool_ring_kernel(const PoolSlotDev *__restrict__ slots,
                                                          const PoolItem *__restrict__ items, PoolCounts *cnt, int K,
                                                          int nw, int seg, int *status)
{
    using namespace ring;
    static_assert(pool_ring_smem<NT, G>() <= 227u * 1024u, "rings fit the shared memory of a CTA");
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int item_s, abort_s;
    volatile int *abort_flag = &abort_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NWARP = NT / 32;
    constexpr int RB = pool_ring_slots<NT, G>() * SEGB * G;  // ring bytes of a warp
    const uint32_t ring0 = smem_addr(smem) + (uint32_t)(warp * RB);
    const uint32_t bar0 = smem_addr(smem) + (uint32_t)(NWARP * RB + warp * NBAR * sizeof(uint64_t));
    if (lane == 0) {
        for (int b = 0; b < NBAR; ++b) mbar_init1(bar0 + 8u * b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x == 0) abort_s = 0;
    __syncthreads();
    Lanes<false, 4, G> w;
    w.init(lane, 0, 1, K, 1, seg, nullptr, nullptr, ring0, bar0);  // the ring; the block is set per item
    const int kv = K / 4;
    bool diverged = false;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(&cnt->queue, 1);
        __syncthreads();
        const int it = item_s;
        if (it >= cnt->items || *abort_flag) break;
        const PoolItem item = items[it];
        const PoolSlotDev &S = slots[item.slot];
        const int ncyc = S.nb + S.ns;
        Mat<false> m;
        m.rows = S.grows;
        m.cst = S.gcst;
        m.z0 = S.z[0];
        m.w0 = S.w[0];
        m.has_noise = true;
        m.zsh = S.zsh;
        m.wsh = S.wsh;
        m.ldsh = S.ldsh;
        m.kp = S.kp;
        m.tq = nullptr;
        float tdummy = 0.f;
        for (int cyc = 0; cyc < ncyc && !*abort_flag; ++cyc) {
            const bool acc = cyc >= S.nb;
            // the item's chain block; diagonal partials while sampling
            w.set_block(item.slice, kv, K, S.n, acc ? (void *)S.dpart : nullptr, S.noise);
            const int cur = S.cur ^ (cyc & 1);
            m.zn_off = cur ? 0u : (uint32_t)S.n * (uint32_t)kv;
            m.zent = cur ? S.gzent[1] : S.gzent[0];
            m.went = cur ? S.gwent[1] : S.gwent[0];
            m.noise_cyc = (size_t)cyc * nw * (size_t)S.n;
            const bool sh = acc && S.inverse;
            m.rpos = sh ? S.perm : nullptr;  // full inverse: R = S = every row in order
            m.spos = sh ? S.perm : nullptr;
            m.shcol = cyc - S.nb;
            m.check_div = cyc == ncyc - 1;
            for (int l = 0; l < S.nlev; ++l) {
                // the last level's state stores (this CTA's) before this level's bulk reads
                asm volatile("fence.proxy.async.global;" ::: "memory");
                if (!*abort_flag)
                    level_bulk<false, 4, G, false, pool_ring_slots<NT, G>()>(w, m, __ldg(&S.levptr[l]) + warp,
                                                                             __ldg(&S.levptr[l + 1]), NWARP, tdummy,
                                                                             diverged, abort_flag);
                __syncthreads();
            }
        }
    }
    if (diverged) atomicOr(status, 1);
    if (threadIdx.x == 0 && *abort_flag) {
        atomicOr(status, 4);
        const uint64_t t0 = gtimer();  // let copies still in flight land before exit
        while (gtimer() - t0 < 10000000ull) {
        }
    }
}

// Folds after the contraction: block segments add the FP32 batch product to
// the FP64 sums and batch-mean moments; diagonal segments add the units'
// partials of each group to the FP64 group sums (by position, so that the
// read-modify-writes are coalesced; the estimate maps positions to rows) and
// clear them.
__global__ void __launch_bounds__(256) pool_fold_kernel(const PoolSlotDev *__restrict__ slots,
                                                        const PoolSeg *__restrict__ segs, const PoolCounts *cnt,
                                                        int units, int G)
{
    for (int e = blockIdx.x; e < cnt->segs; e += gridDim.x) {
        const PoolSeg sg = segs[e];
        const PoolSlotDev &S = slots[sg.slot];
        if (sg.kind == 0) {
            // eight elements a thread per step, every load issued before the stores
            // (segments start at multiples of 2^16), explicit round-to-nearest double
            // operations as in the single-matrix fold
            const float4 *__restrict__ D4 = (const float4 *)(S.D + sg.begin);
            double2 *__restrict__ s2 = (double2 *)(S.bsum + sg.begin);
            double2 *__restrict__ q2 = (double2 *)(S.bsq + sg.begin);
            const double sc = S.scale_sq;
            const long long q8 = sg.count / 8;
            for (long long k = threadIdx.x; k < q8; k += blockDim.x) {
                const float4 v0 = D4[2 * k], v1 = D4[2 * k + 1];
                double2 a[4], c[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) { a[h] = s2[4 * k + h]; c[h] = q2[4 * k + h]; }
                const double x[8] = {(double)v0.x, (double)v0.y, (double)v0.z, (double)v0.w,
                                     (double)v1.x, (double)v1.y, (double)v1.z, (double)v1.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    a[h].x = __dadd_rn(a[h].x, x[2 * h]);
                    a[h].y = __dadd_rn(a[h].y, x[2 * h + 1]);
                    c[h].x = __fma_rn(__dmul_rn(x[2 * h], x[2 * h]), sc, c[h].x);
                    c[h].y = __fma_rn(__dmul_rn(x[2 * h + 1], x[2 * h + 1]), sc, c[h].y);
                }
#pragma unroll
                for (int h = 0; h < 4; ++h) { s2[4 * k + h] = a[h]; q2[4 * k + h] = c[h]; }
            }
            for (long long k = 8 * q8 + threadIdx.x; k < sg.count; k += blockDim.x) {
                const long long x = sg.begin + k;
                const double v = S.D[x];
                S.bsum[x] = __dadd_rn(S.bsum[x], v);
                S.bsq[x] = __fma_rn(__dmul_rn(v, v), S.scale_sq, S.bsq[x]);
            }
        } else {
            const int upg = units / G;
            const size_t n = (size_t)S.n;
            for (long long k = threadIdx.x; k < sg.count; k += blockDim.x) {
                float *__restrict__ dp = S.dpart + sg.begin + k;
                double *__restrict__ da = S.dacc + sg.begin + k;
                // eight groups at a time: their partials loaded together, then summed in unit
                // order from zero, cleared, and added to the group sums
                for (int g0 = 0; g0 < G; g0 += 8) {
                    double sum[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        double s = 0.0;
                        if (g0 + j < G)
                            for (int u = 0; u < upg; ++u) s += (double)dp[(size_t)((g0 + j) * upg + u) * n];
                        sum[j] = s;
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (g0 + j < G) {
                            for (int u = 0; u < upg; ++u) dp[(size_t)((g0 + j) * upg + u) * n] = 0.f;
                            da[(size_t)(g0 + j) * n] += sum[j];
                        }
                    }
                }
            }
        }
    }
}

// The full inverse of P C P^T back to the rows and columns of C: entry (r, c)
// of C^-1 is entry (pos[r], pos[c]) of the sampled matrix's inverse (pos: the
// position of each row of C in the colour order).  Reads gathered within a row,
// writes coalesced.
__global__ void block_unpermute_kernel(long long n, const int *__restrict__ pos, const double *__restrict__ mean_p,
                                       const double *__restrict__ se_p, double *__restrict__ mean_c,
                                       double *__restrict__ se_c)
{
    const long long total = n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / n, c = e - r * n;
        const long long src = (long long)pos[r] * n + pos[c];
        mean_c[e] = mean_p[src];
        se_c[e] = se_p[src];
    }
}

template <int LPR>
static cudaError_t launch_pool_sweep_l(int V, const PoolSlotDev *slots, const PoolItem *items, PoolCounts *cnt, int K,
                                       int nw, int blob_max, int seg, int *status, int grid, int threads, cudaStream_t s)
{
    const size_t smem = 2 * (size_t)blob_max + 64;
    cudaError_t e;
    if (V == 4) {
        e = cudaFuncSetAttribute(pool_sweep_kernel<LPR, 4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        pool_sweep_kernel<LPR, 4, 8><<<grid, threads, smem, s>>>(slots, items, cnt, K, nw, blob_max, seg, status);
    } else {
        e = cudaFuncSetAttribute(pool_sweep_kernel<LPR, 1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        pool_sweep_kernel<LPR, 1, 8><<<grid, threads, smem, s>>>(slots, items, cnt, K, nw, blob_max, seg, status);
    }
    return cudaGetLastError();
}

static cudaError_t launch_pool_sweep(int LPR, int V, const PoolSlotDev *slots, const PoolItem *items, PoolCounts *cnt,
                                     int K, int nw, int blob_max, int seg, int *status, int grid, int threads,
                                     cudaStream_t s)
{
    if ((LPR == 32 && (threads == 384 || threads == 512)) || (LPR == 64 && threads == 384)) {
        // the ring form: 128-chain blocks (12 or 16 warps) or 256-chain blocks (12 warps)
        auto kern = LPR == 64 ? pool_ring_kernel<384, 2> : threads == 384 ? pool_ring_kernel<384, 1> : pool_ring_kernel<512, 1>;
        const size_t smem = LPR == 64 ? pool_ring_smem<384, 2>() : threads == 384 ? pool_ring_smem<384, 1>() : pool_ring_smem<512, 1>();
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, threads, smem, s>>>(slots, items, cnt, K, nw, seg, status);
        return cudaGetLastError();
    }
    switch (LPR) {
    case 1: return launch_pool_sweep_l<1>(V, slots, items, cnt, K, nw, blob_max, seg, status, grid, threads, s);
    case 2: return launch_pool_sweep_l<2>(V, slots, items, cnt, K, nw, blob_max, seg, status, grid, threads, s);
    case 4: return launch_pool_sweep_l<4>(V, slots, items, cnt, K, nw, blob_max, seg, status, grid, threads, s);
    case 8: return launch_pool_sweep_l<8>(V, slots, items, cnt, K, nw, blob_max, seg, status, grid, threads, s);
    case 16: return launch_pool_sweep_l<16>(V, slots, items, cnt, K, nw, blob_max, seg, status, grid, threads, s);
    case 32: return launch_pool_sweep_l<32>(V, slots, items, cnt, K, nw, blob_max, seg, status, grid, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mcinv

using namespace mcinv;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// First-fit allocator over the arena: offsets only, no device calls.
class Arena {
public:
    void reset(size_t bytes)
    {
        free_.clear();
        free_[0] = bytes;
        size_ = bytes;
        used_ = 0;
    }
    // returns false if no free range fits
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

struct Alloc {
    size_t off = 0, bytes = 0;
};

struct HostSlot {
    bool used = false;
    int64_t ticket = -1;
    int64_t n = 0, nnz = 0;
    int nchunks = 0, nlev = 0;
    uint32_t matrix_id = 0;
    int64_t burnin = 0, samples = 0;  // schedule
    int64_t cycle = 0;                // cycles run
    int64_t sampled = 0, batches = 0; // samples accumulated, block batches folded
    int64_t pend = 0, folded = 0;     // sampling cycles in the FP32 product not yet folded; folded
    int pend_steps = 0;               // sampling steps summed in the FP32 product since the last fold
    int inverse = 0;
    int cur = 0;
    std::vector<int32_t> ord;  // MCINV_F_COLOR_ORDER: row k of the sampled P C P^T is row ord[k] of C
    std::vector<int32_t> perm; // position p (level order) is row perm[p] of the sampled matrix
    std::vector<Alloc> allocs;
    PoolSlotDev dev{};
    CUtensorMap maps[2];
};

}  // namespace

struct mcinv_pool_ctx {
    // options
    int64_t K = 256;
    uint64_t seed = 0;
    int64_t chain_base = 0;
    int B = 8, G = 32, units = 0, seg = 1, nw = 0;
    int F = 8;                         // steps whose block products are summed before a fold
    int LPR = 8, V = 4, threads = 512, grid_sweep = 152;
    int blob_max = 48 * 1024;
    int max_slots = 0;
    bool tuned = false, fixed_shape = false, color = false;
    int tune_next = 0;                 // next candidate shape to time
    std::vector<double> tune_score;    // ms per unit of work, per candidate
    cudaStream_t stream = nullptr;
    // memory
    uint8_t *arena = nullptr;
    size_t arena_bytes = 0;
    Arena heap;
    // slots
    std::vector<HostSlot> slots;
    std::map<int64_t, int> ticket_slot;
    int64_t next_ticket = 1;
    // device tables
    PoolSlotDev *d_slots = nullptr;
    PoolItem *d_items = nullptr;
    PoolRB *d_rbs = nullptr;
    GroupTile *d_tiles = nullptr;
    GroupOut *d_outs = nullptr;
    PoolSeg *d_segs = nullptr;
    PoolCounts *d_cnt = nullptr;
    CUtensorMap *d_maps = nullptr;
    double *d_counts = nullptr;
    int *d_status = nullptr;
    size_t cap_items = 0, cap_rbs = 0, cap_tiles = 0, cap_segs = 0;
    // pinned staging of the tables
    uint8_t *h_stage = nullptr;
    size_t stage_bytes = 0;
    cudaEvent_t staged = nullptr;
    // graph of one step
    cudaGraphExec_t graph = nullptr;
    int graph_LPR = 0, graph_threads = 0;
    // accounting
    int64_t steps = 0, launches = 0;
    double step_ms_last = 0.0;
    std::vector<double> counts;
    std::string err;
};

static thread_local std::string g_pool_error;

static mcinv_status pfail(mcinv_pool_ctx *p, mcinv_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (p) p->err = buf;
    else g_pool_error = buf;
    return st;
}

#define PCUDA(p, call)                                                                                     \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return pfail((p), MCINV_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

extern "C" void mcinv_pool_default_options(mcinv_pool_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->K = 256;
    o->batch_cycles = 8;
    o->max_slots = 512;
    o->groups = 32;
}

extern "C" mcinv_status mcinv_pool_create(mcinv_pool_t *out, const mcinv_pool_options *o_in)
{
    if (!out) return pfail(nullptr, MCINV_E_ARG, "out is NULL");
    *out = nullptr;
    mcinv_pool_options o;
    if (o_in) o = *o_in;
    else mcinv_pool_default_options(&o);
    if (o.K < 4 || o.K % 4 || o.K > (1 << 16)) return pfail(nullptr, MCINV_E_ARG, "pool K must be a multiple of 4 in [4, 65536]");
    if (o.max_slots < 1 || o.max_slots > (1 << 20)) return pfail(nullptr, MCINV_E_ARG, "max_slots out of range");
    if (o.mem_budget <= 0) return pfail(nullptr, MCINV_E_ARG, "mem_budget must be > 0");
    mcinv_pool_ctx *p = new (std::nothrow) mcinv_pool_ctx;
    if (!p) return pfail(nullptr, MCINV_E_NOMEM, "host allocation failed");
    p->K = o.K;
    p->seed = o.seed;
    p->chain_base = o.chain_base;
    p->B = o.batch_cycles > 0 ? o.batch_cycles : 8;
    if (o.fold_steps < 0 || o.fold_steps > 1024) {
        delete p;
        return pfail(nullptr, MCINV_E_ARG, "fold_steps must be in [0, 1024]");
    }
    p->F = o.fold_steps > 0 ? o.fold_steps : 8;
    p->max_slots = (int)o.max_slots;
    p->stream = (cudaStream_t)o.stream;
    p->color = (o.flags & MCINV_F_COLOR_ORDER) != 0;
    p->nw = (int)((o.K + 31) / 32);
    p->V = 4;
    if (o.chains_per_cta > 0) {
        p->LPR = o.chains_per_cta / 4;
        const bool ring2 = p->LPR == 64 && o.chains_per_cta == 256 && (o.threads_per_cta == 0 || o.threads_per_cta == 384);
        if (!ring2 && (p->LPR < 1 || p->LPR > 32 || (p->LPR & (p->LPR - 1)) || o.chains_per_cta != 4 * p->LPR)) {
            delete p;
            return pfail(nullptr, MCINV_E_ARG,
                         "chains_per_cta must be 4 x a power of two <= 128, or 256 (the ring form, 384 threads)");
        }
        p->fixed_shape = true;
    } else {
        p->LPR = 8;  // 32-chain slices; the first steps time the alternatives
    }
    p->threads = o.threads_per_cta > 0 ? o.threads_per_cta : p->LPR == 64 ? 384 : 512;
    if (p->threads % 32 || p->threads > 512) {
        delete p;
        return pfail(nullptr, MCINV_E_ARG, "threads_per_cta must be a multiple of 32, <= 512");
    }
    if (o.threads_per_cta > 0) p->fixed_shape = p->fixed_shape || o.chains_per_cta > 0;
    // SE units: seg lanes (seg x 4 chains) with seg <= every candidate slice's lanes (>= 2)
    const int Greq = o.groups > 0 ? o.groups : 32;
    int seg = 1;
    const int minL = p->fixed_shape ? std::min(p->LPR, 32) : 2;
    while (seg * 2 <= minL && (int64_t)seg * 2 * 4 * Greq <= o.K) seg *= 2;
    p->seg = seg;
    p->units = (int)((o.K + seg * 4 - 1) / (seg * 4));
    p->G = 1;
    for (int g = std::min(Greq, p->units); g >= 1; --g)
        if (p->units % g == 0) { p->G = g; break; }
    p->counts.assign(p->G, 0.0);
    for (int k = 0; k < p->units; ++k)
        p->counts[k / (p->units / p->G)] += (double)std::min<int64_t>(seg * 4, o.K - (int64_t)k * seg * 4);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->grid_sweep = sms;
    auto bail = [&](mcinv_status st) {
        std::string m = p->err;
        mcinv_pool_destroy(p);
        g_pool_error = m;
        return st;
    };
    cudaError_t e = cudaMalloc((void **)&p->arena, (size_t)o.mem_budget);
    if (e != cudaSuccess) {
        cudaGetLastError();
        pfail(p, MCINV_E_NOMEM, "cannot reserve the %lld-byte arena: %s", (long long)o.mem_budget, cudaGetErrorString(e));
        return bail(MCINV_E_NOMEM);
    }
    p->arena_bytes = (size_t)o.mem_budget;
    p->heap.reset(p->arena_bytes);
    p->slots.resize(p->max_slots);
    if ((e = cudaMalloc((void **)&p->d_slots, sizeof(PoolSlotDev) * p->max_slots)) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_maps, sizeof(CUtensorMap) * 2 * p->max_slots)) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_outs, sizeof(GroupOut) * p->max_slots)) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_cnt, sizeof(PoolCounts))) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&p->d_counts, sizeof(double) * p->G)) != cudaSuccess ||
        (e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(p->d_cnt, 0, sizeof(PoolCounts))) != cudaSuccess ||
        (e = cudaMemcpy(p->d_counts, p->counts.data(), sizeof(double) * p->G, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->staged, cudaEventDisableTiming)) != cudaSuccess) {
        pfail(p, MCINV_E_CUDA, "pool tables: %s", cudaGetErrorString(e));
        return bail(MCINV_E_CUDA);
    }
    *out = p;
    return MCINV_OK;
}

// Device footprint of a matrix in the pool, part by part (arena bytes).
static void slot_parts(const mcinv_pool_ctx *p, const Prepared &P, int inverse, std::vector<size_t> &parts)
{
    const size_t n = (size_t)P.n, K = (size_t)p->K;
    const size_t kp = (K + 63) / 64 * 64;
    parts.clear();
    parts.push_back(P.stream.size());                              // 0 stream
    parts.push_back(P.chunks.size() * sizeof(ChunkDesc));          // 1 chunks
    parts.push_back(n * 4);                                        // 2 perm
    parts.push_back(n * 4);                                        // 3 pos
    parts.push_back(2 * n * K * 4);                                // 4 z (both buffers)
    parts.push_back(2 * n * K * 4);                                // 5 w (both buffers)
    parts.push_back((size_t)p->B * p->nw * n * 4);                 // 6 noise
    parts.push_back((size_t)p->units * n * 4);                     // 7 dpart
    parts.push_back((size_t)p->G * n * 8);                         // 8 dacc
    if (inverse) {
        const size_t ld = (size_t)p->B * kp;
        parts.push_back((n + 127) / 128 * 128 * ld * 2);          // 9 zsh
        parts.push_back((n + 255) / 256 * 256 * ld * 2);          // 10 wsh
        parts.push_back(n * n * 4);                                // 11 D
        parts.push_back(n * n * 8);                                // 12 bsum
        parts.push_back(n * n * 8);                                // 13 bsq
    }
    // the flat form of the ring form (kGridParts parts, last)
    parts.push_back(P.grow.size() * sizeof(GridRow));              // records
    parts.push_back(P.gzent.size());                               // C entries, cycles from buffer 0
    parts.push_back(P.gzent.size());                               // C entries, cycles from buffer 1
    parts.push_back(P.gwent.size());                               // C^dagger entries, buffer 0
    parts.push_back(P.gwent.size());                               // C^dagger entries, buffer 1
    parts.push_back(n * sizeof(CstR));                             // constants by position
    parts.push_back(P.lev_ptr.size() * 4);                         // level starts
}
static constexpr int kGridParts = 7;

extern "C" mcinv_status mcinv_pool_footprint(mcinv_pool_t p, int64_t n, int64_t nnz, int32_t want_inverse, int64_t *bytes)
{
    if (!p || !bytes || n <= 0) return pfail(p, MCINV_E_ARG, "bad arguments");
    // an estimate from the shapes alone (the stream is bounded by ~48 B per row + 16 B per entry x 2)
    const size_t K = (size_t)p->K, un = (size_t)n;
    size_t b = un * 48 + (size_t)nnz * 32 + 4096 + 8 * un + 4 * un * K * 4 + (size_t)p->B * p->nw * un * 4 +
               (size_t)p->units * un * 4 + (size_t)p->G * un * 8 + un * 36 + (size_t)nnz * 32 + 8 * 256;
    if (want_inverse) {
        const size_t ld = (size_t)p->B * ((K + 63) / 64 * 64);
        b += (un + 127) / 128 * 128 * ld * 2 + (un + 255) / 256 * 256 * ld * 2 + un * un * 20;
    }
    *bytes = (int64_t)b;
    return MCINV_OK;
}

static void slot_release(mcinv_pool_ctx *p, HostSlot &s)
{
    for (const Alloc &a : s.allocs) p->heap.release(a.off, a.bytes);
    s.allocs.clear();
    s.used = false;
    s.ticket = -1;
}

extern "C" mcinv_status mcinv_pool_submit(mcinv_pool_t p, int64_t n, const int64_t *row_ptr, const int32_t *col,
                                          const double *val, uint32_t matrix_id, int64_t burnin, int64_t samples,
                                          int32_t want_inverse, int64_t *ticket)
{
    if (!p || !ticket) return pfail(p, MCINV_E_ARG, "NULL argument");
    if (burnin < 0 || samples < 1) return pfail(p, MCINV_E_ARG, "need burnin >= 0 and samples >= 1");
    int si = -1;
    for (int k = 0; k < p->max_slots; ++k)
        if (!p->slots[k].used) { si = k; break; }
    if (si < 0) return pfail(p, MCINV_E_NOMEM, "no free slot");
    Prepared P;
    std::string why;
    // the colour order (Sec. 4 reordering): sample P C P^T, map rows back in the results
    std::vector<int32_t> ord;
    std::vector<int64_t> rp2;
    std::vector<int32_t> col2;
    std::vector<double> val2;
    if (p->color) {
        int nc = 0;
        mcinv_status st = color_order(n, row_ptr, col, val, 0, ord, &nc, &why);
        if (st != MCINV_OK) return pfail(p, st, "%s", why.c_str());
        permute_csr(n, row_ptr, col, val, 0, ord, rp2, col2, val2);
        row_ptr = rp2.data();
        col = col2.data();
        val = val2.data();
    }
    if (2.0 * (double)n * (double)(p->K / 4) >= 4294967296.0)
        return pfail(p, MCINV_E_UNSUPPORTED, "n K too large for the pool's 32-bit state indices");
    mcinv_status st = prepare_matrix(n, row_ptr, col, val, 0, p->blob_max, P, &why);
    if (st != MCINV_OK) return pfail(p, st, "%s", why.c_str());
    if (P.blob_max > p->blob_max) return pfail(p, MCINV_E_UNSUPPORTED, "a row has too many entries for the pool's chunks");
    std::vector<size_t> parts;
    slot_parts(p, P, want_inverse, parts);
    HostSlot &s = p->slots[si];
    s = HostSlot{};
    s.ord = std::move(ord);
    s.perm = P.perm;
    for (size_t b : parts) {
        Alloc a;
        a.bytes = b;
        if (!p->heap.alloc(b, &a.off)) {
            for (const Alloc &x : s.allocs) p->heap.release(x.off, x.bytes);
            s.allocs.clear();
            return pfail(p, MCINV_E_NOMEM, "the request needs more device memory than the pool has free");
        }
        s.allocs.push_back(a);
    }
    auto at = [&](int k) { return p->arena + s.allocs[k].off; };
    cudaStream_t str = p->stream;
    // uploads (host vectors live until the synchronisation below)
    PCUDA(p, cudaMemcpyAsync(at(0), P.stream.data(), P.stream.size(), cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(1), P.chunks.data(), P.chunks.size() * sizeof(ChunkDesc), cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(2), P.perm.data(), n * 4, cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(3), P.pos.data(), n * 4, cudaMemcpyHostToDevice, str));
    const int gp = (int)parts.size() - kGridParts;  // the flat form's first part
    for (int k = 4; k < gp; ++k) PCUDA(p, cudaMemsetAsync(at(k), 0, parts[k], str));
    // the flat form: records (.row = i K / 4), entries for each cycle parity (.col =
    // vector index of the gathered segment from z[0] / w[0]: this cycle's buffer
    // for j < i, last cycle's for j > i), level starts
    const uint32_t kv = (uint32_t)(p->K / 4), nkv = (uint32_t)n * kv;
    std::vector<GridRow> grow = P.grow;
    for (int64_t q = 0; q < n; ++q) grow[q].row = (int)((uint32_t)P.grow[q].row * kv);
    std::vector<uint8_t> gent[4];
    for (int par = 0; par < 2; ++par) {
        const uint32_t off_new = par ? 0u : nkv, off_old = par ? nkv : 0u;
        gent[par] = P.gzent;
        gent[2 + par] = P.gwent;
        for (int64_t q = 0; q < n; ++q) {
            const int i = P.grow[q].row;
            auto fix = [&](std::vector<uint8_t> &v, int b, int e) {
                for (int x = b; x < e; ++x) {
                    int *c = (int *)(v.data() + (size_t)x * sizeof(EntR));
                    *c = (int)((*c < i ? off_new : off_old) + (uint32_t)*c * kv);
                }
            };
            fix(gent[par], P.grow[q].zb, P.grow[q + 1].zb);
            fix(gent[2 + par], P.grow[q].wb, P.grow[q + 1].wb);
        }
    }
    PCUDA(p, cudaMemcpyAsync(at(gp), grow.data(), grow.size() * sizeof(GridRow), cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(gp + 1), gent[0].data(), gent[0].size(), cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(gp + 2), gent[1].data(), gent[1].size(), cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(gp + 3), gent[2].data(), gent[2].size(), cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(gp + 4), gent[3].data(), gent[3].size(), cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(at(gp + 6), P.lev_ptr.data(), P.lev_ptr.size() * 4, cudaMemcpyHostToDevice, str));
    // constants in FP64 on the GPU, written into the stream
    double *d_diag = nullptr;
    long long *d_at = nullptr;
    int *d_bad = nullptr;
    PCUDA(p, cudaMallocAsync((void **)&d_diag, n * 8, str));
    PCUDA(p, cudaMallocAsync((void **)&d_at, n * 8, str));
    PCUDA(p, cudaMallocAsync((void **)&d_bad, 4, str));
    const int big = 0x7fffffff;
    PCUDA(p, cudaMemcpyAsync(d_diag, P.diag_pos.data(), n * 8, cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(d_at, P.cst_at.data(), n * 8, cudaMemcpyHostToDevice, str));
    PCUDA(p, cudaMemcpyAsync(d_bad, &big, 4, cudaMemcpyHostToDevice, str));
    PCUDA(p, launch_constants((int)n, d_diag, 0, at(0), d_at, d_bad, str));
    // the same constants by position for the ring form
    std::vector<long long> cat((size_t)n);
    for (int64_t q = 0; q < n; ++q) cat[q] = (long long)(q * (int64_t)sizeof(CstR));
    PCUDA(p, cudaMemcpyAsync(d_at, cat.data(), n * 8, cudaMemcpyHostToDevice, str));
    PCUDA(p, launch_constants((int)n, d_diag, 0, at(gp + 5), d_at, d_bad, str));
    int bad = big;
    PCUDA(p, cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, str));
    PCUDA(p, cudaFreeAsync(d_diag, str));
    PCUDA(p, cudaFreeAsync(d_at, str));
    PCUDA(p, cudaFreeAsync(d_bad, str));
    PCUDA(p, cudaStreamSynchronize(str));
    p->launches++;
    if (bad != big) {
        slot_release(p, s);
        return pfail(p, MCINV_E_SINGULAR_DIAG, "diagonal entry of row %d is not usable", P.perm[bad]);
    }
    s.used = true;
    s.ticket = p->next_ticket++;
    s.n = n;
    s.nnz = P.nnz;
    s.nchunks = (int)P.chunks.size();
    s.nlev = P.nlev;
    s.matrix_id = matrix_id;
    s.burnin = burnin;
    s.samples = samples;
    s.inverse = want_inverse ? 1 : 0;
    PoolSlotDev &d = s.dev;
    d.stream = at(0);
    d.chunks = (const ChunkDesc *)at(1);
    d.perm = (const int *)at(2);
    d.pos = (const int *)at(3);
    d.z[0] = (float *)at(4); d.z[1] = d.z[0] + (size_t)n * p->K;
    d.w[0] = (float *)at(5); d.w[1] = d.w[0] + (size_t)n * p->K;
    d.noise = (uint32_t *)at(6);
    d.dpart = (float *)at(7);
    d.dacc = (double *)at(8);
    d.grows = (const GridRow *)at(gp);
    d.gzent[0] = (const EntR *)at(gp + 1);
    d.gzent[1] = (const EntR *)at(gp + 2);
    d.gwent[0] = (const EntR *)at(gp + 3);
    d.gwent[1] = (const EntR *)at(gp + 4);
    d.gcst = (const CstR *)at(gp + 5);
    d.levptr = (const int *)at(gp + 6);
    d.nlev = (int)P.nlev;
    d.n = (int)n;
    d.nchunks = s.nchunks;
    d.matrix_id = matrix_id;
    d.inverse = s.inverse;
    const long long kp = (p->K + 63) / 64 * 64;
    d.kp = kp;
    d.ldsh = (long long)p->B * kp;
    if (s.inverse) {
        d.zsh = (uint16_t *)at(9);
        d.wsh = (uint16_t *)at(10);
        d.D = (float *)at(11);
        d.bsum = (double *)at(12);
        d.bsq = (double *)at(13);
        const char *w = nullptr;
        if (!tc_encode_operand(&s.maps[0], d.zsh, (n + 127) / 128 * 128, d.ldsh, d.ldsh, false, &w) ||
            !tc_encode_operand(&s.maps[1], d.wsh, (n + 255) / 256 * 256, d.ldsh, d.ldsh, true, &w)) {
            slot_release(p, s);
            return pfail(p, MCINV_E_UNSUPPORTED, "%s", w ? w : "tensor map");
        }
        PCUDA(p, cudaMemcpyAsync(p->d_maps + 2 * si, s.maps, sizeof s.maps, cudaMemcpyHostToDevice, str));
        GroupOut go{d.D, (int)n, (int)n, 0, 0};
        PCUDA(p, cudaMemcpyAsync(p->d_outs + si, &go, sizeof go, cudaMemcpyHostToDevice, str));
        PCUDA(p, cudaStreamSynchronize(str));
    }
    p->ticket_slot[s.ticket] = si;
    *ticket = s.ticket;
    return MCINV_OK;
}

template <typename T>
static cudaError_t grow(T **ptr, size_t *cap, size_t need)
{
    if (need <= *cap) return cudaSuccess;
    size_t c = std::max<size_t>(need, *cap * 2 + 64);
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    cudaError_t e = cudaMalloc((void **)ptr, c * sizeof(T));
    if (e == cudaSuccess) *cap = c;
    else *cap = 0;
    return e;
}

// One step's work tables, built on the host.
struct StepTables {
    std::vector<PoolSlotDev> slots;
    std::vector<PoolItem> items;
    std::vector<PoolRB> rbs;
    std::vector<GroupTile> tiles;
    std::vector<GroupOut> outs;
    std::vector<PoolSeg> segs;
    std::vector<char> fold;  // per slot: the block product is folded after this step
};

static void build_tables(mcinv_pool_ctx *p, StepTables &T)
{
    const int lpr = p->LPR;
    const int W = lpr * p->V;
    const int slices = (int)((p->K + W - 1) / W);
    T.slots.assign(p->max_slots, PoolSlotDev{});
    T.items.clear(); T.rbs.clear(); T.tiles.clear(); T.segs.clear();
    T.outs.assign(p->max_slots, GroupOut{});
    T.fold.assign(p->max_slots, 0);
    const long long kp = (p->K + 63) / 64 * 64;
    std::vector<std::pair<double, int>> order;
    for (int si = 0; si < p->max_slots; ++si) {
        HostSlot &s = p->slots[si];
        if (!s.used) continue;
        const int64_t todo = s.burnin + s.samples - s.cycle;
        if (todo <= 0) continue;
        const int64_t nb = std::max<int64_t>(0, std::min<int64_t>(p->B, s.burnin - s.cycle));
        const int64_t ns = std::min<int64_t>(p->B - nb, todo - nb);
        PoolSlotDev d = s.dev;
        d.cycle0 = (uint32_t)s.cycle;
        d.cur = s.cur;
        d.nb = (int)nb;
        d.ns = (int)ns;
        // the block products of F sampling steps (fewer at the member's end) are summed
        // in FP32 by the contraction's epilogue, then folded once: a batch of pend + ns cycles
        const bool fold = ns > 0 && (s.pend_steps + 1 >= p->F || ns == todo - nb);
        d.scale_sq = fold ? 1.0 / ((double)p->K * (double)p->K * (double)(s.pend + ns)) : 0.0;
        T.slots[si] = d;
        T.fold[si] = fold ? 1 : 0;
        order.push_back({(double)(s.nnz + s.n) * (double)(nb + ns), si});
        for (int rb = 0; rb < (s.n + 127) / 128; ++rb) T.rbs.push_back(PoolRB{si, rb});
        if (ns > 0) {
            if (s.inverse) {
                T.outs[si] = GroupOut{d.D, (int)s.n, (int)s.n, (int)((ns * kp + 63) / 64), s.pend > 0 ? 1 : 0};
                for (int m0 = 0; m0 < s.n; m0 += 128)
                    for (int n0 = 0; n0 < s.n; n0 += 256) T.tiles.push_back(GroupTile{si, m0, n0, 0});
                const long long el = (long long)s.n * s.n;
                if (fold)
                    for (long long b = 0; b < el; b += 1 << 16)
                        T.segs.push_back(PoolSeg{si, 0, b, std::min<long long>(1 << 16, el - b)});
            }
            // diagonal segments of 256 positions (a position a thread): the fold of a large
            // matrix spreads over many CTAs instead of one walking it
            for (long long b = 0; b < s.n; b += 256) T.segs.push_back(PoolSeg{si, 1, b, std::min<long long>(256, s.n - b)});
        }
    }
    // most expensive matrices first, so the persistent sweep ends evenly
    std::sort(order.begin(), order.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    for (const auto &o : order)
        for (int sl = 0; sl < slices; ++sl) T.items.push_back(PoolItem{o.second, sl});
}

// One step's kernels on stream s; with ev, the sweep is bracketed by ev[0], ev[1].
static mcinv_status launch_step(mcinv_pool_ctx *p, cudaStream_t s, bool count, cudaEvent_t *ev = nullptr)
{
    PCUDA(p, cudaMemsetAsync(&p->d_cnt->queue, 0, sizeof(int), s));
    pool_noise_kernel<<<4 * 152, 128, 0, s>>>(p->d_slots, p->d_rbs, p->d_cnt, p->seed, (uint64_t)p->chain_base, (int)p->K, p->nw);
    PCUDA(p, cudaGetLastError());
    if (ev) PCUDA(p, cudaEventRecord(ev[0], s));
    PCUDA(p, launch_pool_sweep(p->LPR, p->V, p->d_slots, p->d_items, p->d_cnt, (int)p->K, p->nw, p->blob_max, p->seg,
                               p->d_status, p->grid_sweep, p->threads, s));
    if (ev) PCUDA(p, cudaEventRecord(ev[1], s));
    PCUDA(p, tc_gemm_grouped_run(p->d_tiles, &p->d_cnt->tiles, p->d_maps, p->d_outs, 152, p->d_status, s));
    pool_fold_kernel<<<8 * 152, 256, 0, s>>>(p->d_slots, p->d_segs, p->d_cnt, p->units, p->G);
    PCUDA(p, cudaGetLastError());
    if (count) p->launches += 4;
    return MCINV_OK;
}

// Time the sweep of one step per candidate shape on the pool's current members
// (the results are the same whichever shape runs: same arithmetic per chain);
// the score is the sweep's time per unit of sweep work, so burn-in and sampling
// steps compare alike.
// {32, 384} and {32, 512} are the ring form (a CTA of 12 or 16 warps per 128-chain block),
// {64, 384} the ring form with 256-chain blocks (two vectors a lane)
static const int kTuneL[][2] = {{2, 512}, {4, 512}, {8, 512}, {8, 256}, {16, 256}, {32, 256}, {32, 384}, {32, 512},
                                {64, 384}};

extern "C" mcinv_status mcinv_pool_step(mcinv_pool_t p)
{
    if (!p) return pfail(nullptr, MCINV_E_ARG, "NULL pool");
    // the step's slice shape is fixed before the work items are split by it
    const int nc = (int)(sizeof kTuneL / sizeof kTuneL[0]);
    const bool timed = !p->tuned && !p->fixed_shape;
    int k_tune = -1;
    if (timed) {
        if (p->tune_score.empty()) p->tune_score.assign(nc, 1e300);
        k_tune = p->tune_next;
        p->LPR = kTuneL[k_tune][0];
        p->threads = kTuneL[k_tune][1];
    }
    StepTables T;
    build_tables(p, T);
    if (T.items.empty()) return MCINV_OK;
    // device tables (sizes grow as needed; growing drops the captured graph)
    const size_t before = p->cap_items + p->cap_rbs + p->cap_tiles + p->cap_segs;
    PCUDA(p, grow(&p->d_items, &p->cap_items, T.items.size()));
    PCUDA(p, grow(&p->d_rbs, &p->cap_rbs, T.rbs.size()));
    PCUDA(p, grow(&p->d_tiles, &p->cap_tiles, std::max<size_t>(1, T.tiles.size())));
    PCUDA(p, grow(&p->d_segs, &p->cap_segs, std::max<size_t>(1, T.segs.size())));
    if (p->cap_items + p->cap_rbs + p->cap_tiles + p->cap_segs != before && p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    // stage into pinned memory (the previous step's copy must be done first)
    const size_t b_slots = sizeof(PoolSlotDev) * p->max_slots, b_items = sizeof(PoolItem) * T.items.size(),
                 b_rbs = sizeof(PoolRB) * T.rbs.size(), b_tiles = sizeof(GroupTile) * T.tiles.size(),
                 b_outs = sizeof(GroupOut) * p->max_slots, b_segs = sizeof(PoolSeg) * T.segs.size();
    const size_t need = b_slots + b_items + b_rbs + b_tiles + b_outs + b_segs + sizeof(PoolCounts) + 8 * 256;
    PCUDA(p, cudaEventSynchronize(p->staged));
    if (need > p->stage_bytes) {
        if (p->h_stage) cudaFreeHost(p->h_stage);
        p->h_stage = nullptr;
        p->stage_bytes = 0;
        PCUDA(p, cudaMallocHost((void **)&p->h_stage, need * 2));
        p->stage_bytes = need * 2;
    }
    uint8_t *h = p->h_stage;
    size_t o = 0;
    auto put = [&](const void *src, size_t bytes) {
        uint8_t *dst = h + o;
        if (bytes) std::memcpy(dst, src, bytes);
        o += (bytes + 255) & ~(size_t)255;
        return dst;
    };
    PoolCounts c{};
    c.items = (int)T.items.size();
    c.rbs = (int)T.rbs.size();
    c.tiles = (int)T.tiles.size();
    c.segs = (int)T.segs.size();
    cudaStream_t s = p->stream;
    PCUDA(p, cudaMemcpyAsync(p->d_slots, put(T.slots.data(), b_slots), b_slots, cudaMemcpyHostToDevice, s));
    PCUDA(p, cudaMemcpyAsync(p->d_items, put(T.items.data(), b_items), b_items, cudaMemcpyHostToDevice, s));
    PCUDA(p, cudaMemcpyAsync(p->d_rbs, put(T.rbs.data(), b_rbs), b_rbs, cudaMemcpyHostToDevice, s));
    if (b_tiles) PCUDA(p, cudaMemcpyAsync(p->d_tiles, put(T.tiles.data(), b_tiles), b_tiles, cudaMemcpyHostToDevice, s));
    PCUDA(p, cudaMemcpyAsync(p->d_outs, put(T.outs.data(), b_outs), b_outs, cudaMemcpyHostToDevice, s));
    if (b_segs) PCUDA(p, cudaMemcpyAsync(p->d_segs, put(T.segs.data(), b_segs), b_segs, cudaMemcpyHostToDevice, s));
    PCUDA(p, cudaMemcpyAsync(p->d_cnt, put(&c, sizeof c), sizeof c, cudaMemcpyHostToDevice, s));
    PCUDA(p, cudaEventRecord(p->staged, s));

    if (timed) {
        // autotune on live steps: each candidate shape runs one real step (every
        // shape computes the same values), the fastest per unit of work is kept
        const int k = k_tune;
        p->tune_next++;
        cudaEvent_t ev[2];
        PCUDA(p, cudaEventCreate(&ev[0]));
        PCUDA(p, cudaEventCreate(&ev[1]));
        const mcinv_status st = launch_step(p, s, true, ev);
        PCUDA(p, cudaEventSynchronize(ev[1]));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        if (st != MCINV_OK) return st;
        double work = 0;
        for (int si = 0; si < p->max_slots; ++si)
            work += (double)(T.slots[si].nb + T.slots[si].ns) * (double)(p->slots[si].nnz + p->slots[si].n);
        p->tune_score[k] = ms / std::max(work, 1.0);
        if (p->tune_next == nc) {
            int best = 0;
            for (int q = 1; q < nc; ++q)
                if (p->tune_score[q] < p->tune_score[best]) best = q;
            p->LPR = kTuneL[best][0];
            p->threads = kTuneL[best][1];
            p->tuned = true;
        }
    }
    if (!timed) {
        if (!p->graph || p->graph_LPR != p->LPR || p->graph_threads != p->threads) {
            if (p->graph) cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
            cudaStream_t cs;
            PCUDA(p, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g;
            PCUDA(p, cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
            const mcinv_status st = launch_step(p, cs, false);
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (st != MCINV_OK) return st;
            PCUDA(p, e);
            e = cudaGraphInstantiate(&p->graph, g, 0);
            cudaGraphDestroy(g);
            PCUDA(p, e);
            p->graph_LPR = p->LPR;
            p->graph_threads = p->threads;
        }
        PCUDA(p, cudaGraphLaunch(p->graph, s));
        p->launches += 4;
    }
    for (int si = 0; si < p->max_slots; ++si) {
        const PoolSlotDev &d = T.slots[si];
        if (d.nb + d.ns == 0) continue;
        HostSlot &hs = p->slots[si];
        hs.cycle += d.nb + d.ns;
        hs.cur ^= (d.nb + d.ns) & 1;
        if (d.ns > 0) {
            hs.sampled += d.ns;
            hs.pend += d.ns;
            hs.pend_steps += 1;
            if (T.fold[si]) {
                hs.batches += 1;
                hs.folded += hs.pend;
                hs.pend = 0;
                hs.pend_steps = 0;
            }
        }
    }
    p->steps++;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_pool_poll(mcinv_pool_t p, int64_t ticket, int32_t *done)
{
    if (!p || !done) return pfail(p, MCINV_E_ARG, "NULL argument");
    auto it = p->ticket_slot.find(ticket);
    if (it == p->ticket_slot.end()) return pfail(p, MCINV_E_ARG, "unknown ticket %lld", (long long)ticket);
    const HostSlot &s = p->slots[it->second];
    *done = s.cycle >= s.burnin + s.samples;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_pool_estimate(mcinv_pool_t p, int64_t ticket, mcinv_kind kind, const double *q, double *out,
                                            double *se_out)
{
    if (!p || !out) return pfail(p, MCINV_E_ARG, "NULL argument");
    auto it = p->ticket_slot.find(ticket);
    if (it == p->ticket_slot.end()) return pfail(p, MCINV_E_ARG, "unknown ticket %lld", (long long)ticket);
    HostSlot &s = p->slots[it->second];
    if (s.sampled == 0) return pfail(p, MCINV_E_STATE, "nothing sampled yet");
    cudaStream_t str = p->stream;
    int status = 0;
    PCUDA(p, cudaMemcpyAsync(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, str));
    PCUDA(p, cudaStreamSynchronize(str));
    if (status & 4) return pfail(p, MCINV_E_TIMEOUT, "a bounded wait in the pool's sweep expired");
    if (status & 2) return pfail(p, MCINV_E_TIMEOUT, "a bounded wait in the pool's contraction expired");
    if (status & 1) return pfail(p, MCINV_E_DIVERGED, "a chain in the pool diverged");
    const size_t n = (size_t)s.n;
    size_t elems;
    if (kind == MCINV_EST_DIAG) elems = n;
    else if (kind == MCINV_EST_TRACE) elems = 2;
    else if (kind == MCINV_EST_BLOCK) {
        if (!s.inverse) return pfail(p, MCINV_E_STATE, "the full inverse was not requested for this matrix");
        if (s.folded == 0) return pfail(p, MCINV_E_STATE, "no block batch folded yet");
        elems = n * n;
    } else return pfail(p, MCINV_E_ARG, "unknown estimate kind");
    // scratch for the estimate from the arena (bookkeeping only)
    Alloc a;
    a.bytes = 2 * elems * 8 + (kind == MCINV_EST_TRACE ? n * 8 : 0);
    if (!p->heap.alloc(a.bytes, &a.off)) return pfail(p, MCINV_E_NOMEM, "no arena space for the estimate");
    double *mean = (double *)(p->arena + a.off), *se = mean + elems;
    Alloc g;                   // scratch of the unpermuted inverse, when it fits
    bool unpermuted = false;   // the inverse is in the rows of C already
    mcinv_status st = MCINV_OK;
    cudaError_t e = cudaSuccess;
    if (kind == MCINV_EST_DIAG) {
        e = launch_diag_estimate(0, (int)n, p->G, p->d_counts, (double)s.sampled, s.dev.dacc, mean, se, str);
    } else if (kind == MCINV_EST_TRACE) {
        double *dq = se + elems;
        // q by position (the diagonal's group sums are kept by position)
        std::vector<double> qk;
        if (q) {
            qk.resize(n);
            for (size_t k = 0; k < n; ++k) {
                const int32_t r = s.perm[k];
                qk[k] = q[s.ord.empty() ? r : s.ord[r]];
            }
            q = qk.data();
        }
        if (!q) st = pfail(p, MCINV_E_ARG, "q_diag is NULL");
        else if ((e = cudaMemcpyAsync(dq, q, n * 8, cudaMemcpyHostToDevice, str)) == cudaSuccess &&
                 (e = cudaStreamSynchronize(str)) == cudaSuccess)
            e = launch_trace_estimate(0, (int)n, p->G, p->d_counts, (double)s.sampled, s.dev.dacc, dq, mean, str);
    } else {
        // the samples folded so far (a product still being summed joins at its fold)
        e = launch_block_estimate(0, (long long)(n * n), (double)p->K, (double)s.folded, (double)s.batches, s.dev.bsum,
                                  s.dev.bsq, mean, se, str);
        if (e == cudaSuccess && !s.ord.empty() && p->heap.alloc(2 * elems * 8 + n * 4, &g.off)) {
            // back to the rows and columns of C on the device (else on the host, below)
            g.bytes = 2 * elems * 8 + n * 4;
            double *mc = (double *)(p->arena + g.off), *sc = mc + elems;
            int *dpos = (int *)(sc + elems);
            std::vector<int> pos(n);
            for (size_t k = 0; k < n; ++k) pos[s.ord[k]] = (int)k;
            if ((e = cudaMemcpyAsync(dpos, pos.data(), n * 4, cudaMemcpyHostToDevice, str)) == cudaSuccess &&
                (e = cudaStreamSynchronize(str)) == cudaSuccess) {
                long long blocks = (long long)((elems + 255) / 256);
                if (blocks > 152LL * 16) blocks = 152LL * 16;
                block_unpermute_kernel<<<(unsigned)blocks, 256, 0, str>>>((long long)n, dpos, mean, se, mc, sc);
                e = cudaGetLastError();
            }
            mean = mc;
            se = sc;
            unpermuted = true;
        }
    }
    if (st == MCINV_OK && e == cudaSuccess) {
        if (kind == MCINV_EST_TRACE) {
            e = cudaMemcpyAsync(out, mean, 8, cudaMemcpyDeviceToHost, str);
            if (e == cudaSuccess && se_out) e = cudaMemcpyAsync(se_out, mean + 1, 8, cudaMemcpyDeviceToHost, str);
        } else {
            e = cudaMemcpyAsync(out, mean, elems * 8, cudaMemcpyDeviceToHost, str);
            if (e == cudaSuccess && se_out) e = cudaMemcpyAsync(se_out, se, elems * 8, cudaMemcpyDeviceToHost, str);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(str);
    }
    p->heap.release(a.off, a.bytes);
    if (g.bytes) p->heap.release(g.off, g.bytes);
    if (st != MCINV_OK) return st;
    if (e != cudaSuccess) return pfail(p, MCINV_E_CUDA, "estimate: %s", cudaGetErrorString(e));
    if (kind == MCINV_EST_DIAG) {
        // positions back to the rows of the sampled matrix, and those (colour order) to the rows of C
        for (double *x : {out, se_out}) {
            if (!x) continue;
            std::vector<double> t(x, x + elems);
            for (size_t k = 0; k < n; ++k) {
                const int32_t r = s.perm[k];
                x[s.ord.empty() ? r : s.ord[r]] = t[k];
            }
        }
    } else if (!s.ord.empty() && kind != MCINV_EST_TRACE && !unpermuted) {
        // rows and columns of P C^-1 P^T back to those of C^-1
        for (double *x : {out, se_out}) {
            if (!x) continue;
            std::vector<double> t(x, x + elems);
            for (size_t i = 0; i < n; ++i)
                for (size_t j = 0; j < n; ++j) x[(size_t)s.ord[i] * n + s.ord[j]] = t[i * n + j];
        }
    }
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_pool_get_state(mcinv_pool_t p, int64_t ticket, int64_t chain0, int64_t nchains, double *z,
                                             double *w, int64_t *cycle)
{
    if (!p) return pfail(nullptr, MCINV_E_ARG, "NULL pool");
    auto it = p->ticket_slot.find(ticket);
    if (it == p->ticket_slot.end()) return pfail(p, MCINV_E_ARG, "unknown ticket %lld", (long long)ticket);
    HostSlot &s = p->slots[it->second];
    if (chain0 < 0 || nchains < 0 || chain0 + nchains > p->K) return pfail(p, MCINV_E_ARG, "chain range out of bounds");
    PCUDA(p, cudaStreamSynchronize(p->stream));
    std::vector<float> tmp((size_t)s.n * nchains);
    double *dst[2] = {z, w};
    float *src[2] = {s.dev.z[s.cur], s.dev.w[s.cur]};
    for (int v = 0; v < 2; ++v) {
        if (!dst[v] || nchains == 0) continue;
        PCUDA(p, cudaMemcpy2D(tmp.data(), nchains * 4, src[v] + chain0, p->K * 4, nchains * 4, s.n, cudaMemcpyDeviceToHost));
        if (s.ord.empty()) {
            for (size_t k = 0; k < tmp.size(); ++k) dst[v][k] = tmp[k];
        } else {
            for (int64_t r = 0; r < s.n; ++r)
                for (int64_t c = 0; c < nchains; ++c) dst[v][(size_t)s.ord[r] * nchains + c] = tmp[(size_t)r * nchains + c];
        }
    }
    if (cycle) *cycle = s.cycle;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_pool_release(mcinv_pool_t p, int64_t ticket)
{
    if (!p) return pfail(nullptr, MCINV_E_ARG, "NULL pool");
    auto it = p->ticket_slot.find(ticket);
    if (it == p->ticket_slot.end()) return pfail(p, MCINV_E_ARG, "unknown ticket %lld", (long long)ticket);
    // work of this slot may still be queued: wait for the stream before the memory is reused
    PCUDA(p, cudaStreamSynchronize(p->stream));
    slot_release(p, p->slots[it->second]);
    p->ticket_slot.erase(it);
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_pool_info(mcinv_pool_t p, mcinv_pool_info_t *info)
{
    if (!p || !info) return pfail(p, MCINV_E_ARG, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->K = p->K;
    info->chains_per_cta = p->LPR * p->V;
    info->threads_per_cta = p->threads;
    info->groups = p->G;
    info->batch_cycles = p->B;
    info->fold_steps = p->F;
    info->steps = p->steps;
    info->kernel_launches = p->launches;
    info->arena_bytes = (int64_t)p->arena_bytes;
    info->arena_used = (int64_t)p->heap.used();
    for (const HostSlot &s : p->slots) info->active += s.used ? 1 : 0;
    info->tuned = p->tuned || p->fixed_shape;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_pool_sync(mcinv_pool_t p)
{
    if (!p) return pfail(nullptr, MCINV_E_ARG, "NULL pool");
    PCUDA(p, cudaStreamSynchronize(p->stream));
    return MCINV_OK;
}

extern "C" void mcinv_pool_destroy(mcinv_pool_t p)
{
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->staged) cudaEventDestroy(p->staged);
    if (p->h_stage) cudaFreeHost(p->h_stage);
    cudaFree(p->arena);
    cudaFree(p->d_slots);
    cudaFree(p->d_items);
    cudaFree(p->d_rbs);
    cudaFree(p->d_tiles);
    cudaFree(p->d_outs);
    cudaFree(p->d_segs);
    cudaFree(p->d_cnt);
    cudaFree(p->d_maps);
    cudaFree(p->d_counts);
    cudaFree(p->d_status);
    delete p;
}

extern "C" const char *mcinv_pool_last_error(mcinv_pool_t p)
{
    if (!p) return g_pool_error.c_str();
    return p->err.c_str();
}
