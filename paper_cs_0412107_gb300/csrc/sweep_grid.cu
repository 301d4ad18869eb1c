// sweep_grid.cu -- the coupled sweep (Eqs. 4 and 5) as one cooperative grid
// over every SM.
//
// The chain-sliced kernel (sweep.cu) gives each slice of 16-128 chains its own
// CTA or cluster, which walks every row of the matrix for those chains.  Here
// the unit of work is a (row, chain block) pair, a chain block being the
// 32 x V chains of one warp (a 512-byte segment of z or w per gathered row),
// and all CTAs of one cooperative launch share every dependency level:
//   * warp g keeps one chain block, g mod nblk, for the whole launch and takes
//     the rows g / nblk, g / nblk + R, g / nblk + 2R, ... of every level
//     (R = warps / nblk), so everything that depends on the chains (noise
//     column, diagonal unit, trace lane) is set up once;
//   * a grid-wide barrier ends every level (rows of a level never read each
//     other through C or C^dagger; a row reads z_j, j < i, written at an earlier
//     level from this cycle's buffer and z_j, j > i, from last cycle's buffer,
//     which is the in-place ascending sweep of Eqs. 4/5);
//   * each entry holds the gathered vector's index from the base of the two
//     state buffers for one cycle parity (the host resolves "j < i: this
//     cycle's buffer" into the index), so a gather is one shuffle, one address
//     and one 16-byte load;
//   * the next row's record and entries are loaded while the current row's
//     gathers are in flight, so the gathers are the only round trip on the path.
// The arithmetic is that of the chain-sliced kernel in the same order (the
// pieces of long rows summed as ((p0 + p1) + p2) + p3, explicit round-to-
// nearest FMAs), so both kernels give the same bits for z, w, the diagonal
// partials and the BF16 shadows.  Every wait is bounded (2 s of globaltimer);
// a CTA whose wait expires sets bit 2 of the status word and stops working.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "sweep_core.cuh"
#include "sweep_ring.cuh"

namespace mcinv {

namespace {

// Arrive at the next grid barrier and wait until every CTA of the grid has: the
// counter was zeroed before the launch and counts arrivals (target = barriers
// so far x CTAs).  Thread 0 releases the CTA's writes (ordered before it by the
// CTA barrier) and acquires everyone else's; the closing CTA barrier passes
// that on to the whole CTA.
__device__ __forceinline__ void grid_barrier(unsigned *bar, unsigned target, volatile int *abort_flag)
{
    __syncthreads();
    if (threadIdx.x == 0 && !*abort_flag) {
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        const uint64_t t0 = gtimer();
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if ((int)(v - target) >= 0) break;
            if (gtimer() - t0 > 2000000000ull) {
                *abort_flag = 1;
                break;
            }
            __nanosleep(32);
        }
    }
    __syncthreads();
}

using namespace ring;

constexpr int BULK_THREADS = 384;
constexpr int PAIR_THREADS = 512;
// slots of one warp's ring.  Separate z and w buffers: RING with 12 / G warps
// a CTA, RING16 with 16 warps.  The pair layout: PAIR_RN slots of 1 KB with 16
// warps (G = 1); with G = 2 (two adjacent blocks a warp, 2 KB slots) 9 slots
// with 12 warps or 13 with 8.
template <int NT, int G, bool PAIR>
constexpr int ring_slots()
{
    return PAIR ? (G == 1 ? PAIR_RN : NT == 384 ? 9 : 13) : NT == 512 ? RING16 : RING;
}
// ring bytes of one warp: slots of G x 512 bytes, or of G x 1 KB on the pair layout
template <int NT, int G, bool PAIR>
constexpr int ring_bytes() { return ring_slots<NT, G, PAIR>() * (PAIR ? 2 : 1) * SEGB * G; }
template <int NT, int G, bool PAIR>
constexpr size_t bulk_smem() { return (size_t)(NT / 32) * (ring_bytes<NT, G, PAIR>() + NBAR * sizeof(uint64_t)); }
// the threads of a CTA and the vectors a lane of the bulk-staged forms
constexpr int bulk_g(int threads, bool pair)
{
    return pair ? (threads == PAIR_THREADS ? 1 : 2) : threads <= BULK_THREADS ? BULK_THREADS / threads : 1;
}

// The grid-wide sweep: warp g keeps the chain block g mod nblk for the whole
// launch and takes the rows g / nblk, g / nblk + R, ... of every level (R =
// warps / nblk); a grid barrier ends each level.  G: vectors per lane (BULK
// only; 1 with register gathers).
template <bool CPLX, int V, int NT, bool BULK, int G, bool PAIR = false>
__global__ void __launch_bounds__(NT, 1) cc_sweep_grid_kernel(const SweepArgs a, const GridArgs g)
{
    static_assert(BULK || G == 1, "register gathers take one vector per lane");
    static_assert(!PAIR || (BULK && G <= 2), "the pair layout is read with bulk copies, one or two vectors a lane");
    static_assert(!BULK || bulk_smem<NT, G, PAIR>() <= 227u * 1024u, "rings fit the shared memory of a CTA");
    extern __shared__ __align__(128) uint8_t gsm[];
    __shared__ int abort_s;
    volatile int *abort_flag = &abort_s;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (NT / 32) + warp;
    const int tw = gridDim.x * (NT / 32);
    const int kv = g.kv;  // vectors per row of z (or of w)
    const int nblk = (kv + 32 * G - 1) / (32 * G);
    const int rstep = tw / nblk;       // warps per chain block
    const int r0 = gw / nblk;          // this warp's first row of every level
    const int blk = gw - r0 * nblk;    // and its chain block
    const bool active = r0 < rstep;
    Lanes<CPLX, V, G> w;
    const uint32_t ring0 = smem_addr(gsm) + (uint32_t)(warp * ring_bytes<NT, G, PAIR>());
    const uint32_t bar0 = smem_addr(gsm) + (uint32_t)((NT / 32) * ring_bytes<NT, G, PAIR>() + warp * NBAR * sizeof(uint64_t));
    w.init(lane, blk, kv, a.K, a.n, a.seg, a.diag_part, a.noise, ring0, bar0, PAIR);
    if (threadIdx.x == 0) abort_s = 0;
    if (BULK && lane == 0) {
        for (int b = 0; b < NBAR; ++b) mbar_init1(bar0 + 8u * b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    Mat<CPLX> m;
    m.rows = g.rows;
    m.cst = (const typename Prec<CPLX>::Cst *)g.cst;
    m.z0 = a.z[0];
    m.w0 = PAIR ? a.z[0] : a.w[0];  // the pair layout holds w beside z
    m.has_noise = a.noise != nullptr;
    m.rpos = a.rpos;
    m.spos = a.spos;
    m.zsh = a.zsh;
    m.wsh = a.wsh;
    m.ldsh = a.ldsh;
    m.kp = a.kp;
    m.tq = a.tq;
    bool diverged = false;
    unsigned target = 0;
    const int nlev = g.nlev;
    for (int cyc = 0; cyc < a.ncyc; ++cyc) {
        const int cur = a.cur ^ (cyc & 1);
        m.zn_off = cur ? 0u : g.nkv;  // this cycle's buffer: the other one
        m.zent = (const typename Prec<CPLX>::Ent *)(cur ? g.zent[1] : g.zent[0]);
        m.went = (const typename Prec<CPLX>::Ent *)(cur ? g.went[1] : g.went[0]);
        m.noise_cyc = (size_t)cyc * a.nw * (size_t)a.n;
        m.shcol = a.cyc0_in_batch + cyc;
        m.check_div = cyc == a.ncyc - 1;
        float tsum = 0.f;  // this lane's share of the cycle's trace series value
        for (int l = 0; l < nlev; ++l) {
            const int lb = __ldg(&g.lev_ptr[l]), le = __ldg(&g.lev_ptr[l + 1]);
            if (!*abort_flag && active) {
                if constexpr (BULK) {
                    // the bulk copies read rows that other CTAs wrote before the grid barrier
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    level_bulk<CPLX, V, G, PAIR, ring_slots<NT, G, PAIR>()>(w, m, lb + r0, le, rstep, tsum, diverged, abort_flag);
                } else {
                    level_regs<CPLX, V>(w, m, lb + r0, le, rstep, tsum, diverged);
                }
            }
            // the level's rows are written before any CTA reads them (none after the last)
            if (!(cyc == a.ncyc - 1 && l == nlev - 1)) {
                target += gridDim.x;
                grid_barrier(g.bar, target, abort_flag);
            }
        }
        if (a.tpart && !*abort_flag) {
            // this warp's partial of the cycle's trace series, reduced in a fixed order
            float v = tsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) a.tpart[((size_t)cyc * gridDim.x + blockIdx.x) * (NT / 32) + warp] = v;
        }
    }
    if (diverged) atomicOr(a.status, 1);
    if (threadIdx.x == 0 && *abort_flag) {
        atomicOr(a.status, 4);
        const uint64_t t0 = gtimer();  // let copies still in flight land before exit
        while (gtimer() - t0 < 10000000ull) {
        }
    }
}

template <bool CPLX, int V, int NT, bool BULK, int G, bool PAIR = false>
cudaError_t launch_grid_v(const SweepArgs &a, const GridArgs &g, int ctas, cudaStream_t s)
{
    auto kern = cc_sweep_grid_kernel<CPLX, V, NT, BULK, G, PAIR>;
    const size_t smem = BULK ? bulk_smem<NT, G, PAIR>() : 0;
    if (BULK) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3((unsigned)NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, g);
}

template <bool CPLX, int V, int NT, bool BULK, int G, bool PAIR = false>
int grid_blocks_per_sm()
{
    auto kern = cc_sweep_grid_kernel<CPLX, V, NT, BULK, G, PAIR>;
    const size_t smem = BULK ? bulk_smem<NT, G, PAIR>() : 0;
    int per_sm = 0;
    if ((BULK && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

// The pair layout of the state: row j, chain block k (32 vectors of 16 bytes:
// V chains each) holds the block's z vectors, then the same chains' w vectors;
// rows are nblk x 64 vectors (the last block padded).  Pack: canonical z, w
// ([n][kv] vectors each) -> x; unpack: x -> z, w.
__global__ void pair_pack_kernel(const float4 *__restrict__ z, const float4 *__restrict__ w, float4 *__restrict__ x,
                                 long long n, int kv, int kvp, int unpack)
{
    const long long total = n * (long long)kvp;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long j = t / kvp;
        const int v = (int)(t - j * kvp);
        const long long xo = j * 2 * kvp + (v >> 5) * 64 + (v & 31);
        if (!unpack) {
            x[xo] = v < kv ? z[j * kv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[xo + 32] = v < kv ? w[j * kv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (v < kv) {
            ((float4 *)z)[j * kv + v] = x[xo];
            ((float4 *)w)[j * kv + v] = x[xo + 32];
        }
    }
}

}  // namespace

cudaError_t launch_pair_pack(const void *z, const void *w, void *x, long long n, int kv, int unpack, cudaStream_t s)
{
    const int kvp = (kv + 31) / 32 * 32;
    long long blocks = (n * kvp + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (blocks < 1) blocks = 1;
    pair_pack_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float4 *)z, (const float4 *)w, (float4 *)x, n, kv, kvp, unpack);
    return cudaGetLastError();
}

static_assert(bulk_smem<PAIR_THREADS, 1, true>() == bulk_smem<PAIR_THREADS, 1, false>(),
              "the 16-warp forms share one occupancy");

bool grid_supported(int cplx, int chains_per_lane, int64_t K, int threads, bool bulk)
{
    const int v = cplx ? 2 : 4;
    if (chains_per_lane != v || K % v != 0) return false;
    if (bulk)
        return threads == BULK_THREADS || threads == BULK_THREADS / 2 || threads == BULK_THREADS / 4 ||
               threads == PAIR_THREADS;
    return threads == 384 || threads == 512;
}

int grid_ctas(int cplx, int threads, bool bulk, bool pair)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (bulk && pair && threads != PAIR_THREADS) {
        if (threads == 384)
            per_sm = cplx ? grid_blocks_per_sm<true, 2, 384, true, 2, true>() : grid_blocks_per_sm<false, 4, 384, true, 2, true>();
        else if (threads == 256)
            per_sm = cplx ? grid_blocks_per_sm<true, 2, 256, true, 2, true>() : grid_blocks_per_sm<false, 4, 256, true, 2, true>();
    } else if (bulk) {
        if (threads == PAIR_THREADS)  // the pair and the 16-warp separate forms: the same 12 KB rings
            per_sm = cplx ? grid_blocks_per_sm<true, 2, PAIR_THREADS, true, 1, true>()
                          : grid_blocks_per_sm<false, 4, PAIR_THREADS, true, 1, true>();
        else if (threads == BULK_THREADS)
            per_sm = cplx ? grid_blocks_per_sm<true, 2, BULK_THREADS, true, 1>() : grid_blocks_per_sm<false, 4, BULK_THREADS, true, 1>();
        else if (threads == BULK_THREADS / 2)
            per_sm = cplx ? grid_blocks_per_sm<true, 2, BULK_THREADS / 2, true, 2>()
                          : grid_blocks_per_sm<false, 4, BULK_THREADS / 2, true, 2>();
        else if (threads == BULK_THREADS / 4)
            per_sm = cplx ? grid_blocks_per_sm<true, 2, BULK_THREADS / 4, true, 4>()
                          : grid_blocks_per_sm<false, 4, BULK_THREADS / 4, true, 4>();
    } else if (threads == 384) {
        per_sm = cplx ? grid_blocks_per_sm<true, 2, 384, false, 1>() : grid_blocks_per_sm<false, 4, 384, false, 1>();
    } else if (threads == 512) {
        per_sm = cplx ? grid_blocks_per_sm<true, 2, 512, false, 1>() : grid_blocks_per_sm<false, 4, 512, false, 1>();
    }
    return per_sm * sms;
}

cudaError_t launch_sweep_grid(const SweepArgs &a, const GridArgs &g, int cplx, int ctas, int threads, bool bulk,
                              cudaStream_t s)
{
    if (ctas < 1 || threads < 32) return cudaErrorInvalidConfiguration;
    // rows of a level plus two prefetch strides stay in int; state indices in uint32
    if ((long long)a.n + 2LL * ctas * (threads / 32) >= (1LL << 31) || 2ull * g.nkv >= (1ull << 32))
        return cudaErrorInvalidValue;
    const int G = bulk ? bulk_g(threads, g.pair != 0) : 1;
    if ((long long)ctas * (threads / 32) < (g.nblk + G - 1) / G) return cudaErrorInvalidConfiguration;
    // the barrier counter starts at zero in every launch
    cudaError_t e = cudaMemsetAsync(g.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (bulk) {
        if (g.pair) {
            if (threads == 384)
                return cplx ? launch_grid_v<true, 2, 384, true, 2, true>(a, g, ctas, s)
                            : launch_grid_v<false, 4, 384, true, 2, true>(a, g, ctas, s);
            if (threads == 256)
                return cplx ? launch_grid_v<true, 2, 256, true, 2, true>(a, g, ctas, s)
                            : launch_grid_v<false, 4, 256, true, 2, true>(a, g, ctas, s);
            if (threads != PAIR_THREADS) return cudaErrorInvalidValue;
            return cplx ? launch_grid_v<true, 2, PAIR_THREADS, true, 1, true>(a, g, ctas, s)
                        : launch_grid_v<false, 4, PAIR_THREADS, true, 1, true>(a, g, ctas, s);
        }
        if (threads == PAIR_THREADS)  // 16 warps of RING16 slots
            return cplx ? launch_grid_v<true, 2, PAIR_THREADS, true, 1>(a, g, ctas, s)
                        : launch_grid_v<false, 4, PAIR_THREADS, true, 1>(a, g, ctas, s);
        if (threads == BULK_THREADS)
            return cplx ? launch_grid_v<true, 2, BULK_THREADS, true, 1>(a, g, ctas, s)
                        : launch_grid_v<false, 4, BULK_THREADS, true, 1>(a, g, ctas, s);
        if (threads == BULK_THREADS / 2)
            return cplx ? launch_grid_v<true, 2, BULK_THREADS / 2, true, 2>(a, g, ctas, s)
                        : launch_grid_v<false, 4, BULK_THREADS / 2, true, 2>(a, g, ctas, s);
        if (threads == BULK_THREADS / 4)
            return cplx ? launch_grid_v<true, 2, BULK_THREADS / 4, true, 4>(a, g, ctas, s)
                        : launch_grid_v<false, 4, BULK_THREADS / 4, true, 4>(a, g, ctas, s);
        return cudaErrorInvalidValue;
    }
    if (threads == 384) return cplx ? launch_grid_v<true, 2, 384, false, 1>(a, g, ctas, s) : launch_grid_v<false, 4, 384, false, 1>(a, g, ctas, s);
    if (threads == 512) return cplx ? launch_grid_v<true, 2, 512, false, 1>(a, g, ctas, s) : launch_grid_v<false, 4, 512, false, 1>(a, g, ctas, s);
    return cudaErrorInvalidValue;
}

}  // namespace mcinv
