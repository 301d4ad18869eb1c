// sweep_tiled.cu -- the coupled sweep (Eqs. 4 and 5) of a structurally symmetric
// matrix whose dependency levels cut into short tiles of positions that name few
// distinct neighbours: the lattice operators in the colour order.
//
// The row pipeline of sweep_ring.cuh copies every row's neighbours for itself
// (one bulk copy a neighbour, a ring slot, a queue of rows in flight): on a
// stencil each site is copied again for each of its 4 or 8 neighbours, and the
// per-row bookkeeping makes the sweep issue-bound.  Here a CTA takes a tile of
// consecutive positions of one level and one 32-vector chain block, copies the
// tile's distinct neighbours (its staged list, at most TILE_CAP slabs of 1 KB:
// the block's z and w vectors of one row) into shared memory once, and its 16
// warps update the tile's rows from there: an entry is a slot index, a
// coefficient and two shared-memory loads.  The state is kept block-major
// (block, row, z and w), so each run of consecutive staged rows is one bulk
// copy: a tile of a 2D lattice stages about 97 rows in 3 or 4 copies.  Two
// stage buffers alternate, so the next tile's copies run while this one is
// computed.  The rows' sums take the entries in their order and the epilogue
// is the ring path's `finish`, so the values are the same bits as every other
// sweep kernel's.  A grid barrier ends each level; every wait is bounded (2 s
// of globaltimer).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "internal.h"
#include "sweep_core.cuh"
#include "sweep_ring.cuh"
#include "sweep_tiled.h"

namespace mcinv {

bool build_tiles(const std::vector<GridRow> &rows, const std::vector<uint8_t> &zent, size_t ent_bytes,
                 const std::vector<int32_t> &lev_ptr, int tile, std::vector<int> &tile_ptr,
                 std::vector<int> &tile_slots, std::vector<int> &lev_tile, std::vector<int> &run_ptr,
                 std::vector<int> &run_row, std::vector<int> &run_len, std::vector<uint16_t> &slot)
{
    const int nlev = (int)lev_ptr.size() - 1;
    tile_ptr.assign(1, 0);
    tile_slots.clear();
    lev_tile.assign(1, 0);
    run_ptr.assign(1, 0);
    run_row.clear();
    run_len.clear();
    slot.assign(zent.size() / ent_bytes, 0);
    std::vector<long long> keys;
    // key: (read from this cycle's buffer, row j): the rows of one buffer ascending
    auto key_of = [](int i, int j) { return ((long long)(j < i ? 1 : 0) << 32) | (long long)(uint32_t)j; };
    for (int l = 0; l < nlev; ++l) {
        for (int p0 = lev_ptr[l]; p0 < lev_ptr[l + 1]; p0 += tile) {
            const int p1 = std::min(p0 + tile, (int)lev_ptr[l + 1]);
            keys.clear();
            for (int p = p0; p < p1; ++p) {
                if (rows[p].info & 3) return false;                              // a row cut into pieces
                if (rows[p + 1].zb - rows[p].zb > SPLIT_ENTRIES) return false;  // (implied by the above)
                const int i = rows[p].row;
                for (int e = rows[p].zb; e < rows[p + 1].zb; ++e)
                    keys.push_back(key_of(i, *(const int *)(zent.data() + (size_t)e * ent_bytes)));
            }
            std::sort(keys.begin(), keys.end());
            keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
            if ((int)keys.size() > TILE_CAP) return false;
            // runs of consecutive rows of one buffer; a key's slot is its rank in `keys`
            for (size_t k = 0; k < keys.size();) {
                size_t e = k + 1;
                while (e < keys.size() && keys[e] == keys[e - 1] + 1) ++e;  // same buffer, next row
                const int j0 = (int)(uint32_t)keys[k];
                run_row.push_back(j0 | ((keys[k] >> 32) ? (int)0x80000000u : 0));
                run_len.push_back((int)(e - k) | ((int)k << 16));
                k = e;
            }
            for (int p = p0; p < p1; ++p) {
                const int i = rows[p].row;
                for (int e = rows[p].zb; e < rows[p + 1].zb; ++e) {
                    const long long k = key_of(i, *(const int *)(zent.data() + (size_t)e * ent_bytes));
                    slot[e] = (uint16_t)(std::lower_bound(keys.begin(), keys.end(), k) - keys.begin());
                }
            }
            tile_ptr.push_back(p1);
            tile_slots.push_back((int)keys.size());
            run_ptr.push_back((int)run_row.size());
        }
        lev_tile.push_back((int)tile_ptr.size() - 1);
    }
    return true;
}

std::vector<uint8_t> build_tile_rows(const std::vector<GridRow> &rows, const std::vector<uint8_t> &zent,
                                     const std::vector<uint8_t> &went, const std::vector<uint16_t> &slot, int cplx)
{
    const size_t n = rows.size() - 1;
    const size_t rb = cplx ? sizeof(TileRow<true>) : sizeof(TileRow<false>);
    const size_t eb = cplx ? sizeof(EntC) : sizeof(EntR);
    std::vector<uint8_t> out(n * rb, 0);
    for (size_t p = 0; p < n; ++p) {
        const int d = rows[p + 1].zb - rows[p].zb;
        uint8_t *r = out.data() + p * rb;
        if (cplx) {
            TileRow<true> t{};
            t.iv = rows[p].row * 64;
            t.d = d;
            for (int u = 0; u < d && u < 8; ++u) {
                const EntC ez = *(const EntC *)(zent.data() + (size_t)(rows[p].zb + u) * eb);
                const EntC ew = *(const EntC *)(went.data() + (size_t)(rows[p].wb + u) * eb);
                t.slot[u] = slot[rows[p].zb + u];
                t.zc[u] = make_float2(ez.re, ez.im);
                t.wc[u] = make_float2(ew.re, ew.im);
            }
            std::memcpy(r, &t, rb);
        } else {
            TileRow<false> t{};
            t.iv = rows[p].row * 64;
            t.d = d;
            for (int u = 0; u < d && u < 8; ++u) {
                const EntR ez = *(const EntR *)(zent.data() + (size_t)(rows[p].zb + u) * eb);
                const EntR ew = *(const EntR *)(went.data() + (size_t)(rows[p].wb + u) * eb);
                t.slot[u] = slot[rows[p].zb + u];
                t.zc[u] = ez.val;
                t.wc[u] = ew.val;
            }
            std::memcpy(r, &t, rb);
        }
    }
    return out;
}

namespace {

using namespace ring;

static_assert(SPLIT_ENTRIES == 8, "a tiled row record holds the entries of an unsplit row");

constexpr int TILE_THREADS = 512;         // 16 warps, one CTA an SM
constexpr int TNW = TILE_THREADS / 32;
constexpr int SLAB = 2 * SEGB;            // a row's z and w vectors of one 32-vector block: 1 KB
// a stage buffer's tile metadata: the rows' records and constants (complex sizes)
constexpr int META = TILE_MAX_ROWS * ((int)sizeof(TileRow<true>) + (int)sizeof(CstC));
constexpr size_t TILE_SMEM = 2 * (size_t)TILE_CAP * SLAB + 2 * (size_t)META + 2 * sizeof(uint64_t);
static_assert(TILE_SMEM <= 227u * 1024u, "two stage buffers fit the shared memory of a CTA");

// Arrive at the next grid barrier and wait until every CTA of the grid has (the
// counter was zeroed before the launch; target = barriers so far x CTAs).
// Thread 0 releases the CTA's writes and acquires everyone else's; the closing
// CTA barrier passes that on to the whole CTA.  Bounded: 2 s.
__device__ __forceinline__ void tile_grid_barrier(unsigned *bar, unsigned target, volatile int *abort_flag)
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

template <bool CPLX, int V>
__global__ void __launch_bounds__(TILE_THREADS, 1)
    cc_sweep_tiled_kernel(const SweepArgs a, const GridArgs g, const TileArgs t)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    extern __shared__ __align__(128) uint8_t tsm[];
    __shared__ int abort_s;
    volatile int *abort_flag = &abort_s;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t stage0 = smem_addr(tsm);
    const uint32_t meta0 = stage0 + 2u * TILE_CAP * SLAB;  // the stage buffers' row records and constants
    const uint32_t bar0 = meta0 + 2u * META;               // one mbarrier per stage buffer
    constexpr uint32_t RB = sizeof(TileRow<CPLX>), CB = sizeof(Cst);
    const uint32_t bstride = 64u * (uint32_t)a.n;        // vectors of one chain block, block-major
    Lanes<CPLX, V, 1> w;
    w.init(lane, 0, g.kv, a.K, a.n, a.seg, a.diag_part, a.noise, 0u, 0u, true);
    if (threadIdx.x == 0) {
        abort_s = 0;
        mbar_init1(bar0);
        mbar_init1(bar0 + 8u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    Mat<CPLX> m;
    m.rows = g.rows;  // (not read: the tiled records carry what a row needs)
    m.cst = (const Cst *)g.cst;
    m.z0 = a.z[0];
    m.w0 = a.z[0];  // the pair layout holds w beside z
    m.has_noise = a.noise != nullptr;
    m.rpos = a.rpos;
    m.spos = a.spos;
    m.zsh = a.zsh;
    m.wsh = a.wsh;
    m.ldsh = a.ldsh;
    m.kp = a.kp;
    m.tq = a.tq;
    const float4 *x0 = (const float4 *)a.z[0];
    bool diverged = false;
    unsigned target = 0;
    uint32_t uses = 0;  // tiles this CTA has staged: buffer uses & 1, its phase (uses >> 1) & 1
    for (int cyc = 0; cyc < a.ncyc; ++cyc) {
        const int cur = a.cur ^ (cyc & 1);
        m.zn_off = cur ? 0u : g.nkv;                  // this cycle's buffer: the other one
        const uint32_t old_off = cur ? g.nkv : 0u;    // last cycle's
        m.noise_cyc = (size_t)cyc * a.nw * (size_t)a.n;
        m.shcol = a.cyc0_in_batch + cyc;
        m.check_div = cyc == a.ncyc - 1;
        float tsum = 0.f;
        for (int l = 0; l < g.nlev; ++l) {
            const int t0 = __ldg(&t.lev_tile[l]);
            const int nitems = (__ldg(&t.lev_tile[l + 1]) - t0) * g.nblk;
            // stage item it (tile, chain block) into buffer b: warp 0 issues one bulk copy a
            // run of the tile's staged rows (contiguous in the block-major layout), all
            // completing on the buffer's mbarrier
            auto issue = [&](int it, uint32_t b) {
                if (warp != 0) return;
                const int tile = t0 + it / g.nblk, blk = it - (it / g.nblk) * g.nblk;
                const int r0 = __ldg(&t.run_ptr[tile]), nr = __ldg(&t.run_ptr[tile + 1]) - r0;
                const int ns = min(__ldg(&t.tile_slots[tile]), TILE_CAP);  // (the host keeps it <= TILE_CAP)
                const int p0 = __ldg(&t.tile_ptr[tile]);
                const int np = min(__ldg(&t.tile_ptr[tile + 1]) - p0, TILE_MAX_ROWS);
                const uint32_t bar = bar0 + 8u * b;
                // the slots' earlier generic-proxy reads before these async-proxy writes
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (lane == 0) {
                    mbar_expect(bar, (uint32_t)ns * SLAB + (uint32_t)np * (RB + CB));
                    // the tile's row records and constants (contiguous by position)
                    const uint32_t mb = meta0 + b * (uint32_t)META;
                    bulk_g2s(mb, (const uint8_t *)t.trow + (size_t)p0 * RB, (uint32_t)np * RB, bar);
                    bulk_g2s(mb + TILE_MAX_ROWS * RB, (const uint8_t *)g.cst + (size_t)p0 * CB, (uint32_t)np * CB, bar);
                }
                __syncwarp();
                for (int r = lane; r < nr; r += 32) {
                    const int code = __ldg(&t.run_row[r0 + r]);
                    const int ls = __ldg(&t.run_len[r0 + r]);
                    const uint32_t len = (uint32_t)ls & 0xffffu, s0 = (uint32_t)ls >> 16;
                    const uint32_t j0 = (uint32_t)code & 0x7fffffffu;
                    const uint32_t off = (code < 0 ? m.zn_off : old_off) + (uint32_t)blk * bstride + j0 * 64u;
                    if (s0 + len <= (uint32_t)TILE_CAP)
                        bulk_g2s(stage0 + (b * TILE_CAP + s0) * SLAB, x0 + off, len * SLAB, bar);
                }
            };
            if (!*abort_flag && nitems > 0) {
                // the copies read rows that other CTAs wrote before the grid barrier
                asm volatile("fence.proxy.async.global;" ::: "memory");
                int it = blockIdx.x;
                if (it < nitems) issue(it, uses & 1u);
                for (; it < nitems; it += gridDim.x) {
                    const uint32_t b = uses & 1u;
                    const int nxt = it + gridDim.x;
                    if (nxt < nitems) issue(nxt, b ^ 1u);  // that buffer was released at the last CTA barrier
                    // a stage that did not land (an expired wait) leaves its rows alone: its records,
                    // and so their slots, may never have been written
                    const bool landed = __all_sync(0xffffffffu, ring_wait(bar0 + 8u * b, (uses >> 1) & 1u));
                    if (!landed) *abort_flag = 1;
                    ++uses;
                    const int tile = t0 + it / g.nblk, blk = it - (it / g.nblk) * g.nblk;
                    w.set_block(blk, g.kv, a.K, a.n, a.diag_part, a.noise, true);
                    w.zo[0] = (uint32_t)blk * bstride + (uint32_t)lane;  // the block-major layout
                    w.wo[0] = w.zo[0] + 32u;
                    const uint32_t base = stage0 + b * TILE_CAP * SLAB + (uint32_t)lane * 16u;
                    const int p1 = __ldg(&t.tile_ptr[tile + 1]);
                    const int pb = __ldg(&t.tile_ptr[tile]);
                    const uint32_t mb = meta0 + b * (uint32_t)META;
                    // a row's noise word, diagonal partial and shadow indices, loaded one row ahead
                    uint32_t nbits = 0u;
                    S ndold = P::zero();
                    int nrp = -1, nsp = -1;
                    auto prefetch = [&](int q) {
                        nbits = w.bits(0, q, m.noise_cyc);
                        ndold = w.dlead[0] ? w.dpart[0][q] : P::zero();
                        if (m.rpos) { nrp = __ldg(&m.rpos[q]); nsp = __ldg(&m.spos[q]); }
                    };
                    if (pb + warp < p1) prefetch(pb + warp);
                    for (int p = pb + warp; landed && p < p1; p += TNW) {
                        const uint32_t bits = nbits;
                        const S dold = ndold;
                        const int rp = nrp, sp = nsp;
                        if (p + TNW < p1) prefetch(p + TNW);
                        // the row's record and constants, staged with the tile
                        TileRow<CPLX> r;
#pragma unroll
                        for (int q = 0; q < (int)(RB / 16); ++q)
                            ((float4 *)&r)[q] = lds_vec<float4>(mb + (uint32_t)(p - pb) * RB + 16u * q);
                        Cst k;
#pragma unroll
                        for (int q = 0; q < (int)(CB / 16); ++q)
                            ((float4 *)&k)[q] = lds_vec<float4>(mb + TILE_MAX_ROWS * RB + (uint32_t)(p - pb) * CB + 16u * q);
                        // the sums in entry order (rows of the tiled form have at most 8 entries)
                        T sz = L::zero(), sw = L::zero();
#pragma unroll
                        for (int u = 0; u < SPLIT_ENTRIES; ++u) {
                            if (u < r.d) {
                                Ent ez, ew;
                                ez.col = ew.col = 0;
                                if constexpr (CPLX) {
                                    ez.re = r.zc[u].x; ez.im = r.zc[u].y; ez.pad = 0;
                                    ew.re = r.wc[u].x; ew.im = r.wc[u].y; ew.pad = 0;
                                } else {
                                    ez.val = r.zc[u];
                                    ew.val = r.wc[u];
                                }
                                const uint32_t sl = r.slot[u];
                                L::fma(sz, ez, lds_vec<T>(base + sl * SLAB));
                                L::fma(sw, ew, lds_vec<T>(base + sl * SLAB + SEGB));
                            }
                        }
                        const S pr = finish<CPLX, V, 1>(w, m, 0, p, (uint32_t)r.iv, sz, sw, k, bits, dold, rp, sp, tsum,
                                                         diverged);
                        diag_one(w, 0, p, pr, dold);
                    }
                    // every warp is done with buffer b before it is staged again; an expired wait
                    // ends the level's items for the whole CTA at once (the same answer in every thread)
                    if (__syncthreads_or(*abort_flag)) break;
                }
            }
            // the level's rows are written before any CTA reads them (none after the last)
            if (!(cyc == a.ncyc - 1 && l == g.nlev - 1)) {
                target += gridDim.x;
                tile_grid_barrier(g.bar, target, abort_flag);
            }
        }
        if (a.tpart && !*abort_flag) {
            // this warp's partial of the cycle's trace series, reduced in a fixed order
            float v = tsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) a.tpart[((size_t)cyc * gridDim.x + blockIdx.x) * TNW + warp] = v;
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

// canonical z, w ([n][kv] vectors each) <-> the block-major pair layout x with
// blocks of bw = 2^lg vectors: block b, row j at vector b n 2bw + j 2bw (z), + bw
// (w); vectors past kv are zero
__global__ void tile_pack_kernel(const float4 *__restrict__ z, const float4 *__restrict__ w, float4 *__restrict__ x,
                                 long long n, int kv, int kvp, int lg, int unpack)
{
    const long long total = n * (long long)kvp;
    const int bw = 1 << lg;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long j = t / kvp;
        const int v = (int)(t - j * kvp);
        const long long xo = ((long long)(v >> lg) * n + j) * 2 * bw + (v & (bw - 1));
        if (!unpack) {
            x[xo] = v < kv ? z[j * kv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
            x[xo + bw] = v < kv ? w[j * kv + v] : make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (v < kv) {
            ((float4 *)z)[j * kv + v] = x[xo];
            ((float4 *)w)[j * kv + v] = x[xo + bw];
        }
    }
}

}  // namespace

cudaError_t launch_tile_pack(const void *z, const void *w, void *x, long long n, int kv, int unpack, cudaStream_t s,
                             int bw)
{
    int lg = 0;
    while ((1 << lg) < bw) ++lg;
    if (bw < 1 || bw > 32 || (1 << lg) != bw) return cudaErrorInvalidValue;
    const int kvp = (kv + bw - 1) / bw * bw;
    long long blocks = (n * kvp + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (blocks < 1) blocks = 1;
    tile_pack_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float4 *)z, (const float4 *)w, (float4 *)x, n, kv, kvp, lg,
                                                      unpack);
    return cudaGetLastError();
}

int tiled_ctas(int cplx)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    auto kern = cplx ? cc_sweep_tiled_kernel<true, 2> : cc_sweep_tiled_kernel<false, 4>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TILE_THREADS, TILE_SMEM) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

cudaError_t launch_sweep_tiled(const SweepArgs &a, const GridArgs &g, const TileArgs &t, int cplx, int ctas,
                               cudaStream_t s)
{
    if (ctas < 1 || !g.pair) return cudaErrorInvalidConfiguration;
    if ((long long)a.n + (long long)ctas >= (1LL << 31) || 2ull * g.nkv >= (1ull << 32)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(g.bar, 0, sizeof(unsigned), s);  // the barrier counter starts at zero
    if (e != cudaSuccess) return e;
    auto kern = cplx ? cc_sweep_tiled_kernel<true, 2> : cc_sweep_tiled_kernel<false, 4>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3((unsigned)TILE_THREADS);
    cfg.dynamicSmemBytes = TILE_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, g, t);
}

}  // namespace mcinv
