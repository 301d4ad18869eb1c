// sweep_staged.cu -- the coupled sweep (Eqs. 4/5) with the gathers staged in
// shared memory by a producer warp (real matrices, 4 chains per lane).
//
// The row sweep is bound by the latency of its gathers: each lane group keeps
// one work item's z_j and w_j in registers, so a CTA has only as many gathers in
// flight as it has registers for.  Here one producer warp moves the gathered row
// segments (the W chains of a slice of row j: W x 4 bytes, one cp.async.bulk
// each) into per-consumer slots of shared memory ahead of use, completing on the
// slot's mbarrier; eight consumer warps take the values from there and do the
// same arithmetic, in the same order, as the register kernel (so results are
// bit-identical).  Two slots per consumer, each one warp round of work items:
// while a consumer computes one round, the producer fills its next.
//
// Ordering: rows of one dependency level never read each other, so the gathers
// of a level may all be in flight at once; the level ends with the cluster
// barrier (a CTA barrier without clusters), after which the producer fences the
// async proxy against the generic-proxy stores it has just acquired.  Every wait
// is bounded; after an abort every thread still walks the same barrier schedule.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "sweep_core.cuh"

namespace mcinv {

namespace {

constexpr int NCW = 8;                      // consumer warps
constexpr int SU = 8;                       // staged entries per side and item
constexpr int SLOT_BYTES = 32 * 2 * SU * 16;  // one warp round: 32 lanes x 16 entries x 16 B

struct StagedSmem {
    int blob_max;
    __device__ uint8_t *chunk(uint8_t *base, int b) const { return base + (size_t)b * blob_max; }
    __device__ uint8_t *slot(uint8_t *base, int s) const { return base + 2 * (size_t)blob_max + (size_t)s * SLOT_BYTES; }
    __device__ uint64_t *bars(uint8_t *base) const
    {
        return (uint64_t *)(base + 2 * (size_t)blob_max + (size_t)2 * NCW * SLOT_BYTES);
    }
};
// barriers: [0,2) chunk full, [2,4) chunk empty, [4, 4+2NCW) slot full, [4+2NCW, 4+4NCW) slot empty
constexpr int NBARS = 4 + 4 * NCW;

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// bounded wait on an mbarrier phase (wait_chunk's 2 s limit); false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) { return wait_chunk(smem_addr(b), parity); }

__device__ __forceinline__ void level_barrier(bool cluster)
{
    if (cluster) cluster_barrier();
    else __syncthreads();
}

// The staged sweep kernel: LPR lanes x 4 chains per lane (W = 4 LPR chains per
// slice, K a multiple of W), 32 (1 + NCW) threads, Q CTAs per slice.
template <int LPR, bool CLUSTER>
__global__ void __launch_bounds__(32 * (1 + NCW), 1) cc_sweep_staged_kernel(const SweepArgs a)
{
    using P = Prec<false>;
    using L = Lane<false, 4>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    constexpr int V = 4;
    constexpr int RPW = 32 / LPR;        // items per consumer round
    constexpr int SEG = LPR * 16;        // bytes of one gathered row segment (the slice's chains)
    static_assert(RPW * 2 * SU * SEG == SLOT_BYTES, "slot size");
    extern __shared__ __align__(128) uint8_t smem[];
    const StagedSmem L_{a.blob_max};
    uint64_t *bars = L_.bars(smem);
    uint64_t *cfull = bars, *cempty = bars + 2, *sfull = bars + 4, *sempty = bars + 4 + 2 * NCW;
    volatile int *abort_flag = (volatile int *)(bars + NBARS);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;   // 0: producer, 1..NCW: consumers
    const int me = warp - 1;
    const int sub = lane / LPR;
    const int cl = lane % LPR;
    const int Q = CLUSTER ? a.ctas_per_slice : 1;
    const int rank = CLUSTER ? (int)cluster_rank() : 0;
    const int slice = blockIdx.x / Q;
    const int cs = slice * LPR * V;      // first chain of the slice
    const int c0 = cs + cl * V;          // this lane's first chain
    const bool chain_ok = c0 < a.K;
    const size_t K = (size_t)a.K;
    const uint32_t cshift = (uint32_t)(c0 & 31);
    const int seg = a.seg;
    S *dpart = (S *)a.diag_part + (size_t)(c0 / (seg * V)) * a.n;
    const bool dlead = (cl % seg) == 0;
    const int total = a.ncyc * a.nchunks;

    if (threadIdx.x == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(&cfull[k], 1);
            mbar_init(&cempty[k], NCW);
        }
        for (int s = 0; s < 2 * NCW; ++s) {
            mbar_init(&sfull[s], 1);
            mbar_init(&sempty[s], 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int t = 0; t < 2 && t < total; ++t) {
            const ChunkDesc d = a.chunks[t % a.nchunks];
            stage_chunk(smem_addr(L_.chunk(smem, t)), a.stream + d.off, (uint32_t)d.bytes, smem_addr(&cfull[t]));
        }
    }
    __syncthreads();

    bool diverged = false;
    float tsum = 0.f;
    int round = 0;          // consumer: rounds taken so far; producer: per consumer below
    int prounds[NCW];       // producer: rounds filled per consumer
#pragma unroll
    for (int c = 0; c < NCW; ++c) prounds[c] = 0;
    bool level_end = false;

    for (int t = 0; t < total; ++t) {
        const int cyc = t / a.nchunks;
        const int b = t & 1;
        const ChunkDesc d = a.chunks[t - cyc * a.nchunks];
        const int cur = a.cur ^ (cyc & 1);
        const float *zo = (const float *)a.z[cur];
        float *zn = (float *)a.z[cur ^ 1];
        const float *wo = (const float *)a.w[cur];
        float *wn = (float *)a.w[cur ^ 1];
        const uint8_t *buf = L_.chunk(smem, b);
        const RowMeta *meta = (const RowMeta *)buf;
        const int ngroups = (d.items + RPW - 1) / RPW;
        // a new level: everyone's stores of the last one are done and visible
        if (level_end) {
            __threadfence();
            level_barrier(CLUSTER);
        }
        level_end = (d.flags & CHUNK_LEVEL_END) != 0;
        // chunk t's blob has landed (producer and consumers wait on the same phase)
        if (lane == 0 && !*abort_flag && !mbar_wait(&cfull[b], (uint32_t)(t >> 1) & 1u)) *abort_flag = 1;
        __syncwarp();

        if (warp == 0) {
            // ---------------- producer ----------------
            if (!*abort_flag) asm volatile("fence.proxy.async.global;" ::: "memory");
            for (int g = rank; g < ngroups; g += Q) {
                // abort decisions are taken on lane 0's reading, so the warp stays converged
                if (__shfl_sync(0xffffffffu, (int)*abort_flag, 0)) break;
                const int c = (g / Q) % NCW;
                const int r = prounds[c]++;
                const int s = 2 * c + (r & 1);
                // the slot's previous round has been consumed
                if (r >= 2 && lane == 0 && !mbar_wait(&sempty[s], (uint32_t)((r >> 1) - 1) & 1u)) *abort_flag = 1;
                if (__shfl_sync(0xffffffffu, (int)*abort_flag, 0)) break;
                // valid segments of the group's items: lane k < RPW reads item 4g+k's record
                int nz = 0, nw = 0, zb = 0, wb = 0, row = 0;
                const int it = g * RPW + (lane % RPW);
                if (lane < RPW && it < d.items) {
                    const RowMeta m = meta[it], m1 = meta[it + 1];
                    zb = m.zoff; wb = m.woff; row = m.row;
                    nz = min(m1.zoff - m.zoff, SU);
                    nw = min(m1.woff - m.woff, SU);
                }
                int cnt = nz + nw;
#pragma unroll
                for (int o = 1; o < RPW; o <<= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                uint8_t *slot = L_.slot(smem, s);
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (cnt > 0) mbar_expect(&sfull[s], (uint32_t)(cnt * SEG));
                    else mbar_arrive(&sfull[s]);
                }
                __syncwarp();
                // position q = item x 16 + entry (z: 0..7, w: 8..15); two per lane
                const Ent *zs = (const Ent *)(buf + d.zent_off);
                const Ent *ws = (const Ent *)(buf + d.went_off);
#pragma unroll
                for (int h = 0; h < 2 * RPW * SU / 32; ++h) {
                    const int q = lane + 32 * h;
                    const int item = q / (2 * SU), e = q % (2 * SU);
                    const int izb = __shfl_sync(0xffffffffu, zb, item), inz = __shfl_sync(0xffffffffu, nz, item);
                    const int iwb = __shfl_sync(0xffffffffu, wb, item), inw = __shfl_sync(0xffffffffu, nw, item);
                    const int irow = __shfl_sync(0xffffffffu, row, item);
                    const float *src = nullptr;
                    if (e < SU) {
                        if (e < inz) {
                            const int j = zs[izb + e].col;
                            src = (j < irow ? zn : zo) + (size_t)j * K + cs;
                        }
                    } else if (e - SU < inw) {
                        const int j = ws[iwb + e - SU].col;
                        src = (j < irow ? wn : wo) + (size_t)j * K + cs;
                    }
                    if (src) bulk_g2s(slot + (size_t)q * SEG, src, SEG, &sfull[s]);
                }
            }
            // chunk t-1's buffer is free again (every consumer finished it): stage chunk t+1
            if (t >= 1 && t + 1 < total) {
                if (lane == 0 && !*abort_flag && !mbar_wait(&cempty[(t + 1) & 1], (uint32_t)((t - 1) >> 1) & 1u))
                    *abort_flag = 1;
                if (lane == 0 && !*abort_flag) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    const ChunkDesc dn = a.chunks[(t + 1) % a.nchunks];
                    stage_chunk(smem_addr(L_.chunk(smem, (t + 1) & 1)), a.stream + dn.off, (uint32_t)dn.bytes,
                                smem_addr(&cfull[(t + 1) & 1]));
                }
                __syncwarp();
            }
            if (a.tpart && (t + 1) % a.nchunks == 0 && lane == 0)
                a.tpart[((size_t)cyc * gridDim.x + blockIdx.x) * (blockDim.x >> 5)] = 0.f;
        } else {
            // ---------------- consumers ----------------
            const Cst *cstv = (const Cst *)(buf + d.cst_off);
            const Ent *zs = (const Ent *)(buf + d.zent_off);
            const Ent *ws = (const Ent *)(buf + d.went_off);
            const uint32_t *__restrict__ noise =
                a.noise ? a.noise + ((size_t)cyc * a.nw + (size_t)(c0 >> 5)) * (size_t)a.n : nullptr;
            const int shcol = a.cyc0_in_batch + cyc;
            const bool split = (d.flags & CHUNK_SPLIT) != 0;
            for (int g = rank + Q * me; g < ngroups; g += Q * NCW) {
                const int s = 2 * me + (round & 1);
                const uint32_t par = (uint32_t)(round >> 1) & 1u;
                ++round;
                if (lane == 0 && !*abort_flag && !mbar_wait(&sfull[s], par)) *abort_flag = 1;
                __syncwarp();
                const uint8_t *slot = L_.slot(smem, s);
                const int it = g * RPW + sub;
                const bool live = chain_ok && it < d.items && !*abort_flag;
                RowMeta m{0, 0, 0, 0}, m1{0, 0, 0, 0};
                if (it < d.items) { m = meta[it]; m1 = meta[it + 1]; }
                const int i = m.row, pk = m.info & 3, np = 1 << ((m.info >> 2) & 3), r = m.info >> 4;
                const bool ok = live && pk == 0;
                const int p = d.pb + r;
                uint32_t bits = 0u;
                S dold = P::zero();
                int rp = -1, sp = -1;
                if (ok) {
                    bits = noise ? __ldg(&noise[p]) >> cshift : 0u;
                    if (a.diag_part && dlead) dold = dpart[p];
                    if (a.rpos) { rp = __ldg(&a.rpos[p]); sp = __ldg(&a.spos[p]); }
                }
                T sz = L::zero(), sw = L::zero();
                if (live) {
                    const int zb = m.zoff, zeN = m1.zoff, wb = m.woff, weN = m1.woff;
                    const uint8_t *mine = slot + (size_t)sub * 2 * SU * SEG + (size_t)cl * 16;
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        if (zb + u < zeN) L::fma(sz, zs[zb + u], *(const T *)(mine + (size_t)u * SEG));
                        if (wb + u < weN) L::fma(sw, ws[wb + u], *(const T *)(mine + (size_t)(SU + u) * SEG));
                    }
                    // entries beyond the staged ones (slices longer than SU are rare): plain gathers
                    for (int ez = zb + SU, ew = wb + SU; ez < zeN || ew < weN; ez += SU, ew += SU) {
                        T xz[SU], xw[SU];
#pragma unroll
                        for (int u = 0; u < SU; ++u) {
                            xz[u] = L::zero();
                            xw[u] = L::zero();
                            if (ez + u < zeN) {
                                const int j = zs[ez + u].col;
                                xz[u] = ld_state<true>((const T *)((j < i ? zn : zo) + (size_t)j * K + c0));
                            }
                            if (ew + u < weN) {
                                const int j = ws[ew + u].col;
                                xw[u] = ld_state<true>((const T *)((j < i ? wn : wo) + (size_t)j * K + c0));
                            }
                        }
#pragma unroll
                        for (int u = 0; u < SU; ++u) {
                            if (ez + u < zeN) L::fma(sz, zs[ez + u], xz[u]);
                            if (ew + u < weN) L::fma(sw, ws[ew + u], xw[u]);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sempty[s]);  // the slot's values are in registers now
                // pieces of a split row: the first piece's lanes fold in the others, in order
#pragma unroll
                for (int q = 1; q < 4 && q < RPW; ++q) {
                    const T oz = L::shfl_down(sz, q * LPR), ow = L::shfl_down(sw, q * LPR);
                    if (split && pk == 0 && q < np) { sz = L::add(sz, oz); sw = L::add(sw, ow); }
                }
                S prod = P::zero();
                if (ok) {
                    const float phi_scale = noise ? 1.f : 0.f;
                    const Cst k = cstv[r];
                    T zv, wv;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const float phi = phi_scale * (((bits >> v) & 1u) ? -1.f : 1.f);
                        const S zsc = P::zrow(k, phi, L::get(sz, v));
                        const S wsc = P::wrow(k, phi, L::get(sw, v));
                        L::set(zv, v, zsc);
                        L::set(wv, v, wsc);
                        diverged |= !(P::finite_bounded(zsc) && P::finite_bounded(wsc));
                        prod = P::add(prod, P::mulconj(zsc, wsc));
                    }
                    if (a.tq) tsum = __fmaf_rn(__ldg(&a.tq[p]), prod, tsum);
                    *(T *)(zn + (size_t)i * K + c0) = zv;
                    *(T *)(wn + (size_t)i * K + c0) = wv;
                    if (rp >= 0 || sp >= 0) {
                        const size_t o = (size_t)shcol * a.kp + (size_t)c0;
                        if (rp >= 0) store_bf16<4>(a.zsh + (size_t)rp * a.ldsh + o, L::f(zv));
                        if (sp >= 0) store_bf16<4>(a.wsh + (size_t)sp * a.ldsh + o, L::f(wv));
                    }
                }
                if (a.diag_part) {
#pragma unroll
                    for (int o = 1; o < LPR; o <<= 1)
                        if (o < seg) prod = P::add(prod, P::shfl_xor(prod, o));
                    if (ok && dlead) dpart[p] = P::add(dold, prod);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&cempty[b]);  // this consumer is done with chunk t
            if (a.tpart && (t + 1) % a.nchunks == 0) {
                float v = tsum;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0) a.tpart[((size_t)cyc * gridDim.x + blockIdx.x) * (blockDim.x >> 5) + warp] = v;
                tsum = 0.f;
            }
        }
    }
    __threadfence();
    level_barrier(CLUSTER);  // the last level's rows are done before anyone leaves
    if (diverged) atomicOr(a.status, 1);
    if (threadIdx.x == 0 && *abort_flag) {
        atomicOr(a.status, 4);
        const uint64_t t0 = gtimer();  // let copies still in flight land before exit
        while (gtimer() - t0 < 10000000ull) {
        }
    }
}

size_t staged_smem(int blob_max) { return 2 * (size_t)blob_max + (size_t)2 * NCW * SLOT_BYTES + NBARS * 8 + 16; }

template <int LPR, bool CL>
cudaError_t staged_launch(const SweepArgs &a, int slices, cudaStream_t s)
{
    auto kern = cc_sweep_staged_kernel<LPR, CL>;
    const size_t smem = staged_smem(a.blob_max);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && CL && a.ctas_per_slice > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(slices * (CL ? a.ctas_per_slice : 1)));
    cfg.blockDim = dim3(32 * (1 + NCW));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL ? (unsigned)a.ctas_per_slice : 1u;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = CL ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace

// 4 or 8 lanes per row: a consumer round holds 8 or 4 items, so the (at most 4) pieces
// of a split row are always in one round and are folded by shuffles
bool staged_supported(int cplx, int lanes_per_row, int chains_per_lane, int64_t K, int blob_max)
{
    return !cplx && chains_per_lane == 4 && (lanes_per_row == 4 || lanes_per_row == 8) &&
           K % (4 * lanes_per_row) == 0 && staged_smem(blob_max) <= 227 * 1024;
}

cudaError_t launch_sweep_staged(const SweepArgs &a, int lanes_per_row, int slices, cudaStream_t s)
{
    const bool cl = a.ctas_per_slice > 1;
    switch (lanes_per_row) {
    case 4: return cl ? staged_launch<4, true>(a, slices, s) : staged_launch<4, false>(a, slices, s);
    case 8: return cl ? staged_launch<8, true>(a, slices, s) : staged_launch<8, false>(a, slices, s);
    default: return cudaErrorInvalidValue;
    }
}

int staged_threads() { return 32 * (1 + NCW); }

}  // namespace mcinv
