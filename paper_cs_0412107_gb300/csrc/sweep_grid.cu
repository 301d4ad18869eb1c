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

__device__ __forceinline__ int4 ldnc4(const void *p) { return __ldg((const int4 *)p); }
__device__ __forceinline__ EntR ldg_ent(const EntR *p)
{
    const int2 v = __ldg((const int2 *)p);
    return EntR{v.x, __int_as_float(v.y)};
}
__device__ __forceinline__ EntC ldg_ent(const EntC *p)
{
    const int4 v = ldnc4(p);
    return EntC{v.x, __int_as_float(v.y), __int_as_float(v.z), v.w};
}
__device__ __forceinline__ CstR ldg_cst(const CstR *p)
{
    const float4 v = __ldg((const float4 *)p);
    return CstR{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ CstC ldg_cst(const CstC *p)
{
    const float4 u = __ldg((const float4 *)p), v = __ldg((const float4 *)p + 1);
    CstC k;
    k.alpha = make_float2(u.x, u.y);
    k.beta = make_float2(u.z, u.w);
    k.inv_d = make_float2(v.x, v.y);
    k.pad = make_float2(v.z, v.w);
    return k;
}

template <typename Ent>
__device__ __forceinline__ Ent ent_none()
{
    Ent e;
    e.col = 0;
    if constexpr (sizeof(Ent) == 8) e.val = 0.f;
    else { e.re = 0.f; e.im = 0.f; e.pad = 0; }
    return e;
}

template <typename Ent>
__device__ __forceinline__ Ent shfl_val(const Ent &m, int src)
{
    Ent e;
    e.col = 0;
    if constexpr (sizeof(Ent) == 8) {
        e.val = __shfl_sync(0xffffffffu, m.val, src);
    } else {
        e.re = __shfl_sync(0xffffffffu, m.re, src);
        e.im = __shfl_sync(0xffffffffu, m.im, src);
        e.pad = 0;
    }
    return e;
}

// Entry e (warp-uniform) of a side in the piece path: the first 32 come from the
// lanes' registers, later ones (rows of more than 32 entries) from L1/L2;
// `valid` says e is inside the row.
template <typename Ent>
__device__ __forceinline__ uint32_t ent_off(const Ent &m, const Ent *__restrict__ all, int base, int e, bool valid)
{
    if (e < 32) return (uint32_t)__shfl_sync(0xffffffffu, m.col, e);
    return valid ? (uint32_t)__ldg((const int *)&all[base + e]) : 0u;
}
template <typename Ent>
__device__ __forceinline__ Ent ent_val(const Ent &m, const Ent *__restrict__ all, int base, int e, bool valid)
{
    if (e < 32) return shfl_val(m, e);
    return valid ? ldg_ent(&all[base + e]) : ent_none<Ent>();
}

// The bulk-staged variant keeps, per warp, two stages of NSLOT 512-byte
// segments in shared memory: while one row's gathers land in one stage (one
// cp.async.bulk per gathered segment, completing on the stage's mbarrier), the
// warp computes the previous row from the other.  The gathers then take no
// registers, and every warp has two rows of gathers in flight.
constexpr int NSLOT = 2 * SPLIT_ENTRIES;  // segments of a row with one piece (<= 8 a side)
constexpr int SEGB = 512;                 // 32 lanes x 16 bytes
constexpr int BULK_THREADS = 384;
constexpr size_t BULK_SMEM = (size_t)(BULK_THREADS / 32) * 2 * NSLOT * SEGB + (BULK_THREADS / 32) * 3 * sizeof(uint64_t);

__device__ __forceinline__ void mbar_init1(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// one lane's 16 bytes of a staged segment
template <typename T>
__device__ __forceinline__ T lds_vec(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return *reinterpret_cast<T *>(&v);
}

// The offset held by entry e of a side, e differing from lane to lane; every
// lane of the warp calls it.  Entries past the first 32 come from L1/L2 (only
// when `valid`, i.e. e is inside the row).
template <typename Ent>
__device__ __forceinline__ uint32_t ent_off_lane(const Ent &m, const Ent *__restrict__ all, int base, int e, bool valid)
{
    const uint32_t r = (uint32_t)__shfl_sync(0xffffffffu, m.col, e & 31);
    if (e < 32) return r;
    return valid ? (uint32_t)__ldg((const int *)&all[base + e]) : 0u;
}

// The sum over one side's entries of a row cut into np = 2^lg pieces, the
// entries added one at a time in order: piece k covers entries
// [min(d, k c), min(d, (k+1) c)) with c = ceil(d / np); each piece is summed
// from zero and the pieces are joined in order, ((p0 + p1) + p2) + p3 -- the
// order of the chain-sliced kernel, whose lane groups sum the pieces side by side.
template <typename L>
struct PieceSum {
    using T = typename L::T;
    T acc, tot;
    int k, next, c, d, np;
    __device__ __forceinline__ PieceSum(int d_, int lg) : k(0), d(d_), np(1 << lg)
    {
        c = (d + np - 1) >> lg;
        next = min(d, c);
        acc = L::zero();
        tot = L::zero();
    }
    __device__ __forceinline__ void join()
    {
        if (k == 0) tot = acc;
        else tot = L::add(tot, acc);
        acc = L::zero();
        ++k;
        next = min(d, (k + 1) * c);
    }
    template <typename Ent>
    __device__ __forceinline__ void add(int e, const Ent &en, const T &x)
    {
        while (e >= next && k < np - 1) join();
        L::fma(acc, en, x);
    }
    __device__ __forceinline__ T total()
    {
        while (k < np) join();
        return tot;
    }
};

template <bool CPLX, int V, int NT, bool BULK>
__global__ void __launch_bounds__(NT, 1) cc_sweep_grid_kernel(const SweepArgs a, const GridArgs g)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    constexpr int U1 = 8;  // one batch of a whole row (at most SPLIT_ENTRIES entries a side)
    constexpr int UP = 4;  // batches of a piece of a long row
    extern __shared__ __align__(128) uint8_t gsm[];
    __shared__ int abort_s;
    volatile int *abort_flag = &abort_s;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (NT / 32) + warp;
    const int tw = gridDim.x * (NT / 32);
    const int nblk = g.nblk;
    const int rstep = tw / nblk;       // warps per chain block
    const int r0 = gw / nblk;          // this warp's first row of every level
    const int blk = gw - r0 * nblk;    // and its chain block
    const bool active = r0 < rstep;
    const int c0 = (blk * 32 + lane) * V;
    const bool chain_ok = c0 < a.K;
    const uint32_t cv = (uint32_t)(c0 / V);  // the lane's vector within a row
    const int seg = a.seg;
    const size_t nsz = (size_t)a.n;
    S *dpart = (S *)a.diag_part + (size_t)(c0 / (seg * V)) * nsz;
    const bool dlead = ((lane % seg) == 0) && chain_ok && a.diag_part;
    const uint32_t *noise_col = a.noise ? a.noise + (size_t)(c0 >> 5) * nsz : nullptr;
    const uint32_t cshift = (uint32_t)(c0 & 31);
    const GridRow *__restrict__ rows = g.rows;
    const Cst *__restrict__ cstv = (const Cst *)g.cst;
    T *const z0 = (T *)a.z[0];
    T *const w0 = (T *)a.w[0];
    // bulk-staged variant: this warp's two stages and their barriers; a segment is
    // the block's vectors of one row (fewer than 32 in a last, partial block)
    const uint32_t stage0 = smem_addr(gsm) + (uint32_t)(warp * 2 * NSLOT * SEGB);
    const uint32_t bar0 = smem_addr(gsm) + (uint32_t)((NT / 32) * 2 * NSLOT * SEGB + warp * 3 * sizeof(uint64_t));
    const uint32_t cvb = (uint32_t)(blk * 32);
    const uint32_t seg_bytes = (uint32_t)min(32, (int)(g.nkv / (uint32_t)a.n) - blk * 32) * 16u;
    if (threadIdx.x == 0) abort_s = 0;
    if (BULK && lane == 0) {
        mbar_init1(bar0);
        mbar_init1(bar0 + 8);
        mbar_init1(bar0 + 16);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    bool diverged = false;
    unsigned target = 0;
    uint32_t kk = 0;  // short bulk-staged rows of this warp so far: stage kk & 1, phase (kk >> 1) & 1
    uint32_t kb = 0;  // rounds of long rows so far: phase kb & 1 of the third barrier
    const int nlev = g.nlev;
    for (int cyc = 0; cyc < a.ncyc; ++cyc) {
        const int cur = a.cur ^ (cyc & 1);
        const uint32_t zn_off = cur ? 0u : g.nkv;  // this cycle's buffer: the other one
        const Ent *__restrict__ zent = (const Ent *)(cur ? g.zent[1] : g.zent[0]);
        const Ent *__restrict__ went = (const Ent *)(cur ? g.went[1] : g.went[0]);
        const uint32_t *noise = noise_col ? noise_col + (size_t)cyc * a.nw * nsz : nullptr;
        const int shcol = a.cyc0_in_batch + cyc;
        float tsum = 0.f;  // this lane's share of the cycle's trace series value

        // this lane's share of row i's entries: lane e holds entry e of each side
        auto load_ents = [&](const int4 &rec, Ent &mz, Ent &mw) {
            const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
            mz = lane < dz ? ldg_ent(&zent[rec.y + lane]) : ent_none<Ent>();
            mw = lane < dw ? ldg_ent(&went[rec.z + lane]) : ent_none<Ent>();
        };
        // Eqs. 4/5 for the lane's V chains from the sums over the row's entries, the
        // stores, the shadows and the z_i conj(w_i) partials
        auto finish = [&](int p, const int4 &rec, const T &sz, const T &sw, const Cst &k, uint32_t bits, S dold, int rp,
                          int sp) {
            const uint32_t iv = (uint32_t)rec.x;  // the row's first vector: i * K / V
            S prod = P::zero();
            if (chain_ok) {
                const float phi_scale = noise ? 1.f : 0.f;
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
                if (a.tq) {
                    float re;
                    if constexpr (CPLX) re = prod.x;
                    else re = prod;
                    tsum = __fmaf_rn(__ldg(&a.tq[p]), re, tsum);
                }
                z0[zn_off + iv + cv] = zv;
                w0[zn_off + iv + cv] = wv;
                if (rp >= 0 || sp >= 0) {
                    const size_t o = (size_t)shcol * a.kp + (size_t)c0 * (CPLX ? 2 : 1);
                    constexpr int NF = L::NF;
                    if (rp >= 0) store_bf16<NF>(a.zsh + (size_t)rp * a.ldsh + o, L::f(zv));
                    if (sp >= 0) {
                        if constexpr (!CPLX) {
                            store_bf16<NF>(a.wsh + (size_t)sp * a.ldsh + o, L::f(wv));
                        } else {
                            // rows 2s = [wr, wi] and 2s+1 = [-wi, wr]: one real
                            // contraction gives Re and Im of z conj(w) interleaved
                            uint16_t *wr0 = a.wsh + (size_t)(2 * sp) * a.ldsh + o;
                            float f0[2 * V], f1[2 * V];
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const S x = L::get(wv, v);
                                f0[2 * v] = x.x;
                                f0[2 * v + 1] = x.y;
                                f1[2 * v] = -x.y;
                                f1[2 * v + 1] = x.x;
                            }
                            store_bf16<2 * V>(wr0, f0);
                            store_bf16<2 * V>(wr0 + a.ldsh, f1);
                        }
                    }
                }
            }
            if (a.diag_part) {
                // the unit's sum over its seg lanes; the leader adds it to the running partial
#pragma unroll
                for (int o = 1; o < 32; o <<= 1)
                    if (o < seg) prod = P::add(prod, P::shfl_xor(prod, o));
                if (dlead) dpart[p] = P::add(dold, prod);
            }
        };
        // one row with register gathers: one batch of every gather before any FMA
        // when it has one piece, else its 2 or 4 pieces, each a sequential sum from
        // zero, joined in order
        auto row_regs = [&](int p, const int4 &rec, const Ent &mz, const Ent &mw) {
            const int lg = rec.w & 3;
            const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
            // the epilogue's operands (their latency hides behind the gathers)
            const Cst k = ldg_cst(&cstv[p]);
            const uint32_t bits = (noise && chain_ok) ? __ldg(&noise[p]) >> cshift : 0u;
            S dold = P::zero();
            if (dlead) dold = dpart[p];
            int rp = -1, sp = -1;
            if (a.rpos && chain_ok) { rp = __ldg(&a.rpos[p]); sp = __ldg(&a.spos[p]); }
            T sz = L::zero(), sw = L::zero();
            if (lg == 0) {
                T xz[U1], xw[U1];
#pragma unroll
                for (int u = 0; u < U1; ++u) {
                    const uint32_t oz = (uint32_t)__shfl_sync(0xffffffffu, mz.col, u);
                    const uint32_t ow = (uint32_t)__shfl_sync(0xffffffffu, mw.col, u);
                    xz[u] = L::zero();
                    xw[u] = L::zero();
                    if (u < dz && chain_ok) xz[u] = __ldcg(&z0[oz + cv]);
                    if (u < dw && chain_ok) xw[u] = __ldcg(&w0[ow + cv]);
                }
#pragma unroll
                for (int u = 0; u < U1; ++u) {
                    if (u < dz) L::fma(sz, shfl_val(mz, u), xz[u]);
                    if (u < dw) L::fma(sw, shfl_val(mw, u), xw[u]);
                }
            } else {
                const int np = 1 << lg;
                const int cz = (dz + np - 1) >> lg, cw = (dw + np - 1) >> lg;
#pragma unroll 1
                for (int pk = 0; pk < np; ++pk) {
                    const int zb = min(dz, pk * cz), zeN = min(dz, (pk + 1) * cz);
                    const int wb = min(dw, pk * cw), weN = min(dw, (pk + 1) * cw);
                    T pz = L::zero(), pw = L::zero();
#pragma unroll 1
                    for (int ez = zb, ew = wb; ez < zeN || ew < weN; ez += UP, ew += UP) {
                        T xz[UP], xw[UP];
#pragma unroll
                        for (int u = 0; u < UP; ++u) {
                            const bool vz = ez + u < zeN, vw = ew + u < weN;
                            const uint32_t oz = ent_off(mz, zent, rec.y, ez + u, vz);
                            const uint32_t ow = ent_off(mw, went, rec.z, ew + u, vw);
                            xz[u] = L::zero();
                            xw[u] = L::zero();
                            if (vz && chain_ok) xz[u] = __ldcg(&z0[oz + cv]);
                            if (vw && chain_ok) xw[u] = __ldcg(&w0[ow + cv]);
                        }
#pragma unroll
                        for (int u = 0; u < UP; ++u) {
                            const bool vz = ez + u < zeN, vw = ew + u < weN;
                            const Ent ez_ = ent_val(mz, zent, rec.y, ez + u, vz);
                            const Ent ew_ = ent_val(mw, went, rec.z, ew + u, vw);
                            if (vz) L::fma(pz, ez_, xz[u]);
                            if (vw) L::fma(pw, ew_, xw[u]);
                        }
                    }
                    if (pk == 0) { sz = pz; sw = pw; }
                    else { sz = L::add(sz, pz); sw = L::add(sw, pw); }
                }
            }
            finish(p, rec, sz, sw, k, bits, dold, rp, sp);
        };
        // bulk-staged rows: start the gathers of a one-piece row into stage st
        auto issue = [&](const int4 &rec, const Ent &mz, const Ent &mw, uint32_t st) {
            const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
            const uint32_t bar = bar0 + st * 8u;
            const uint32_t wo = (uint32_t)__shfl_sync(0xffffffffu, mw.col, (lane - dz) & 31);
            // every lane is done reading this stage's previous row; order those
            // generic-proxy reads before the async-proxy writes below
            __syncwarp();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (lane == 0) mbar_expect(bar, (uint32_t)(dz + dw) * seg_bytes);
            if (lane < dz + dw) {
                const T *src = lane < dz ? z0 + (uint32_t)mz.col + cvb : w0 + wo + cvb;
                bulk_g2s(stage0 + (st * NSLOT + lane) * SEGB, src, seg_bytes, bar);
            }
        };

        for (int l = 0; l < nlev; ++l) {
            const int lb = __ldg(&g.lev_ptr[l]), le = __ldg(&g.lev_ptr[l + 1]);
            int p = lb + r0;
            if (BULK && !*abort_flag && active && p < le) {
                // the bulk copies read rows that other CTAs wrote before the grid barrier
                asm volatile("fence.proxy.async.global;" ::: "memory");
                // Rows of at most NSLOT segments are pipelined through the two stages,
                // two in flight; a longer row waits for the one in flight, then takes
                // both stages (all 2 NSLOT slots) per round of gathers.
                int4 rec = ldnc4(&rows[p]);
                int4 rnext = p + rstep < le ? ldnc4(&rows[p + rstep]) : make_int4(0, 0, 0, 0);
                bool have_a = false;  // a short row in flight, number ka of this warp's short rows
                uint32_t ka = 0;
                int pa = 0;
                int4 ra = make_int4(0, 0, 0, 0);
                Ent az = ent_none<Ent>(), aw = ent_none<Ent>();
                // compute the row in flight from its stage
                auto finish_a = [&]() {
                    const uint32_t st = ka & 1u;
                    const Cst k = ldg_cst(&cstv[pa]);
                    const uint32_t bits = (noise && chain_ok) ? __ldg(&noise[pa]) >> cshift : 0u;
                    S dold = P::zero();
                    if (dlead) dold = dpart[pa];
                    int rp = -1, sp = -1;
                    if (a.rpos && chain_ok) { rp = __ldg(&a.rpos[pa]); sp = __ldg(&a.spos[pa]); }
                    if (!wait_chunk(bar0 + st * 8u, (ka >> 1) & 1u)) *abort_flag = 1;
                    const uint32_t sa = stage0 + st * NSLOT * SEGB + lane * 16u;
                    const int dz = (ra.w >> 2) & 0x7fff, dw = (ra.w >> 17) & 0x7fff;
                    T sz = L::zero(), sw = L::zero();
                    if ((ra.w & 3) == 0) {
#pragma unroll
                        for (int u = 0; u < U1; ++u)
                            if (u < dz) L::fma(sz, shfl_val(az, u), lds_vec<T>(sa + u * SEGB));
#pragma unroll
                        for (int u = 0; u < U1; ++u)
                            if (u < dw) L::fma(sw, shfl_val(aw, u), lds_vec<T>(sa + (dz + u) * SEGB));
                    } else {
                        PieceSum<L> pzs(dz, ra.w & 3), pws(dw, ra.w & 3);
                        for (int e = 0; e < dz; ++e) pzs.add(e, shfl_val(az, e), lds_vec<T>(sa + e * SEGB));
                        for (int e = 0; e < dw; ++e) pws.add(e, shfl_val(aw, e), lds_vec<T>(sa + (dz + e) * SEGB));
                        sz = pzs.total();
                        sw = pws.total();
                    }
                    finish(pa, ra, sz, sw, k, bits, dold, rp, sp);
                    have_a = false;
                };
                for (; p < le; p += rstep) {
                    Ent mz, mw;
                    load_ents(rec, mz, mw);
                    const int4 rnn = p + 2 * rstep < le ? ldnc4(&rows[p + 2 * rstep]) : make_int4(0, 0, 0, 0);
                    const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
                    if (dz + dw <= NSLOT) {
                        // start this row's gathers, then finish the one in flight
                        const uint32_t kn = kk++;
                        issue(rec, mz, mw, kn & 1u);
                        if (have_a) finish_a();
                        have_a = true;
                        ka = kn;
                        pa = p;
                        ra = rec;
                        az = mz;
                        aw = mw;
                    } else {
                        if (have_a) finish_a();
                        const Cst k = ldg_cst(&cstv[p]);
                        const uint32_t bits = (noise && chain_ok) ? __ldg(&noise[p]) >> cshift : 0u;
                        S dold = P::zero();
                        if (dlead) dold = dpart[p];
                        int rp = -1, sp = -1;
                        if (a.rpos && chain_ok) { rp = __ldg(&a.rpos[p]); sp = __ldg(&a.spos[p]); }
                        PieceSum<L> pzs(dz, rec.w & 3), pws(dw, rec.w & 3);
                        for (int ez = 0, ew = 0; ez < dz || ew < dw;) {
                            // one round: up to 2 NSLOT segments over both stages
                            int mzr = min(dz - ez, NSLOT);
                            const int mwr = min(dw - ew, 2 * NSLOT - mzr);
                            mzr = min(dz - ez, 2 * NSLOT - mwr);
                            const uint32_t bar = bar0 + 16u;
                            const uint32_t oz = ent_off_lane(mz, zent, rec.y, ez + lane, lane < mzr);
                            const uint32_t ow = ent_off_lane(mw, went, rec.z, ew + lane - mzr, lane >= mzr && lane < mzr + mwr);
                            __syncwarp();
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            if (lane == 0) mbar_expect(bar, (uint32_t)(mzr + mwr) * seg_bytes);
                            if (lane < mzr + mwr) {
                                const T *src = lane < mzr ? z0 + oz + cvb : w0 + ow + cvb;
                                bulk_g2s(stage0 + lane * SEGB, src, seg_bytes, bar);
                            }
                            if (!wait_chunk(bar, kb & 1u)) *abort_flag = 1;
                            ++kb;
                            const uint32_t sa = stage0 + lane * 16u;
                            for (int e = 0; e < mzr; ++e)
                                pzs.add(ez + e, ent_val(mz, zent, rec.y, ez + e, true), lds_vec<T>(sa + e * SEGB));
                            for (int e = 0; e < mwr; ++e)
                                pws.add(ew + e, ent_val(mw, went, rec.z, ew + e, true), lds_vec<T>(sa + (mzr + e) * SEGB));
                            ez += mzr;
                            ew += mwr;
                        }
                        finish(p, rec, pzs.total(), pws.total(), k, bits, dold, rp, sp);
                    }
                    rec = rnext;
                    rnext = rnn;
                }
                if (have_a) finish_a();
            } else if (!BULK && !*abort_flag && active && p < le) {
                // pipeline: this row's record and entries, the next row's record
                int4 rec = ldnc4(&rows[p]);
                Ent mz, mw;
                load_ents(rec, mz, mw);
                int4 nrec = p + rstep < le ? ldnc4(&rows[p + rstep]) : make_int4(0, 0, 0, 0);
                for (; p < le; p += rstep) {
                    // the next row's entries and the one after's record
                    Ent nz, nw;
                    const bool more = p + rstep < le;
                    if (more) load_ents(nrec, nz, nw);
                    const int4 nnrec = p + 2 * rstep < le ? ldnc4(&rows[p + 2 * rstep]) : make_int4(0, 0, 0, 0);
                    row_regs(p, rec, mz, mw);
                    if (more) { rec = nrec; mz = nz; mw = nw; }
                    nrec = nnrec;
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

template <bool CPLX, int V, int NT, bool BULK>
cudaError_t launch_grid_v(const SweepArgs &a, const GridArgs &g, int ctas, cudaStream_t s)
{
    auto kern = cc_sweep_grid_kernel<CPLX, V, NT, BULK>;
    const size_t smem = BULK ? BULK_SMEM : 0;
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

template <bool CPLX, int V, int NT, bool BULK>
int grid_blocks_per_sm()
{
    auto kern = cc_sweep_grid_kernel<CPLX, V, NT, BULK>;
    const size_t smem = BULK ? BULK_SMEM : 0;
    int per_sm = 0;
    if ((BULK && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

}  // namespace

bool grid_supported(int cplx, int chains_per_lane, int64_t K, int threads)
{
    const int v = cplx ? 2 : 4;
    return chains_per_lane == v && K % v == 0 && (threads == 384 || threads == 512);
}

int grid_ctas(int cplx, int threads, bool bulk)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (bulk) {
        if (threads == BULK_THREADS)
            per_sm = cplx ? grid_blocks_per_sm<true, 2, BULK_THREADS, true>() : grid_blocks_per_sm<false, 4, BULK_THREADS, true>();
    } else if (threads == 384) {
        per_sm = cplx ? grid_blocks_per_sm<true, 2, 384, false>() : grid_blocks_per_sm<false, 4, 384, false>();
    } else if (threads == 512) {
        per_sm = cplx ? grid_blocks_per_sm<true, 2, 512, false>() : grid_blocks_per_sm<false, 4, 512, false>();
    }
    return per_sm * sms;
}

cudaError_t launch_sweep_grid(const SweepArgs &a, const GridArgs &g, int cplx, int ctas, int threads, bool bulk,
                              cudaStream_t s)
{
    const int nt = threads;
    if (ctas < 1 || (long long)ctas * (nt / 32) < g.nblk) return cudaErrorInvalidConfiguration;
    // rows of a level plus two prefetch strides stay in int; state indices in uint32
    if ((long long)a.n + 2LL * ctas * (nt / 32) >= (1LL << 31) || 2ull * g.nkv >= (1ull << 32))
        return cudaErrorInvalidValue;
    // the barrier counter starts at zero in every launch
    cudaError_t e = cudaMemsetAsync(g.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (bulk) {
        if (threads != BULK_THREADS) return cudaErrorInvalidValue;
        return cplx ? launch_grid_v<true, 2, BULK_THREADS, true>(a, g, ctas, s)
                    : launch_grid_v<false, 4, BULK_THREADS, true>(a, g, ctas, s);
    }
    if (threads == 384) return cplx ? launch_grid_v<true, 2, 384, false>(a, g, ctas, s) : launch_grid_v<false, 4, 384, false>(a, g, ctas, s);
    if (threads == 512) return cplx ? launch_grid_v<true, 2, 512, false>(a, g, ctas, s) : launch_grid_v<false, 4, 512, false>(a, g, ctas, s);
    return cudaErrorInvalidValue;
}

}  // namespace mcinv
