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

// The bulk-staged variant gives each warp a ring of RING 512-byte slots in
// shared memory.  A row's gathered segments go to consecutive slots of the
// ring (never across its end), one cp.async.bulk each, completing on one of
// QMAX + 1 mbarriers; up to QMAX rows are in flight while the warp computes the
// oldest, so the gathers take no registers and a warp keeps about RING segments
// in flight.  A row of more than RING segments waits for the ring to drain and
// then runs in rounds of RING segments on a barrier of its own.
constexpr int RING = 32;                  // slots per warp (a power of two)
constexpr int QMAX = 3;                   // rows in flight per warp
constexpr int NBAR = QMAX + 2;            // QMAX + 1 for the ring rows, one for long rows
constexpr int SEGB = 512;                 // 32 lanes x 16 bytes
constexpr int BULK_THREADS = 384;
// per CTA: 12 / G warps, each a ring of RING slots of G x 512 bytes (192 KB in all)
template <int G>
constexpr size_t bulk_smem() { return (size_t)(BULK_THREADS / G / 32) * RING * SEGB * G + (BULK_THREADS / G / 32) * NBAR * sizeof(uint64_t); }

// A row in flight in a warp's ring: its position, first vector i K / V, packed
// counts, first slot, barrier use number, and the lane's values of its entries
// (lane e holds entry e of each side; the offsets were used when issued).
template <bool CPLX>
struct RingRow {
    int p, info;
    uint32_t vslot;  // first slot, counted from the warp's start (slot vslot mod RING)
    uint32_t iv, use;
    float zr, zi, wr, wi;
};

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

// Wait for a phase of a ring barrier: try_wait with a suspend-time hint, so the
// warp sleeps in the barrier until the bytes land instead of polling; false
// after 2 s (globaltimer).
__device__ __forceinline__ bool ring_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (int it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(20000u)
            : "memory");
        if (ok) return true;
        if (it == 0) t0 = gtimer();
        else if (gtimer() - t0 > 2000000000ull) return false;
    }
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
    PieceSum() = default;
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

// G: vectors per lane (BULK only; 1 with register gathers).  A warp's chain block
// is G x 32 vectors, i.e. G x 512 contiguous bytes of a row: lane l handles the
// vectors l, l + 32, ... of the block, each exactly as the G = 1 kernel's lane l
// of the 32-vector block it falls in (same diagonal units, same bits).
template <bool CPLX, int V, int NT, bool BULK, int G>
__global__ void __launch_bounds__(NT, 1) cc_sweep_grid_kernel(const SweepArgs a, const GridArgs g)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    static_assert(BULK || G == 1, "register gathers take one vector per lane");
    constexpr int U1 = 8;  // one batch of a whole row (at most SPLIT_ENTRIES entries a side)
    constexpr int UP = 4;  // batches of a piece of a long row
    constexpr int SEGG = SEGB * G;  // bytes of one gathered segment (one ring slot)
    extern __shared__ __align__(128) uint8_t gsm[];
    __shared__ int abort_s;
    volatile int *abort_flag = &abort_s;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (NT / 32) + warp;
    const int tw = gridDim.x * (NT / 32);
    const int kv = (int)(g.nkv / (uint32_t)a.n);  // vectors per row
    const int nblk = (kv + 32 * G - 1) / (32 * G);
    const int rstep = tw / nblk;       // warps per chain block
    const int r0 = gw / nblk;          // this warp's first row of every level
    const int blk = gw - r0 * nblk;    // and its chain block
    const bool active = r0 < rstep;
    const int seg = a.seg;
    const size_t nsz = (size_t)a.n;
    // per vector of the lane: its first chain, the diagonal unit, the noise word
    int c0[G];
    bool chain_ok[G], dlead[G];
    uint32_t cv[G], cshift[G];
    S *dpart[G];
    const uint32_t *noise_col[G];
#pragma unroll
    for (int q = 0; q < G; ++q) {
        cv[q] = (uint32_t)(blk * 32 * G + q * 32 + lane);
        c0[q] = (int)cv[q] * V;
        chain_ok[q] = c0[q] < a.K;
        dpart[q] = (S *)a.diag_part + (size_t)(c0[q] / (seg * V)) * nsz;
        dlead[q] = ((lane % seg) == 0) && chain_ok[q] && a.diag_part;
        noise_col[q] = a.noise ? a.noise + (size_t)(c0[q] >> 5) * nsz : nullptr;
        cshift[q] = (uint32_t)(c0[q] & 31);
    }
    const GridRow *__restrict__ rows = g.rows;
    const Cst *__restrict__ cstv = (const Cst *)g.cst;
    T *const z0 = (T *)a.z[0];
    T *const w0 = (T *)a.w[0];
    // bulk staging: this warp's ring of RING slots of SEGG bytes and its barriers;
    // a segment is the block's vectors of one row (fewer in a last, partial block)
    const uint32_t ring0 = smem_addr(gsm) + (uint32_t)(warp * RING * SEGG);
    const uint32_t bar0 = smem_addr(gsm) + (uint32_t)((NT / 32) * RING * SEGG + warp * NBAR * sizeof(uint64_t));
    const uint32_t bar_long = bar0 + (NBAR - 1) * 8u;
    const uint32_t cvb = (uint32_t)(blk * 32 * G);
    const uint32_t seg_bytes = (uint32_t)min(32 * G, kv - blk * 32 * G) * 16u;
    if (threadIdx.x == 0) abort_s = 0;
    if (BULK && lane == 0) {
        for (int b = 0; b < NBAR; ++b) mbar_init1(bar0 + 8u * b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    bool diverged = false;
    unsigned target = 0;
    uint32_t ic = 0;    // ring rows issued by this warp: row c waits on barrier c % (QMAX + 1), phase (c / (QMAX + 1)) & 1
    uint32_t kb = 0;    // rounds of long rows so far: phase kb & 1 of bar_long
    uint32_t vhead = 0; // the ring's next free slot, counted from the warp's start
    const int nlev = g.nlev;
    for (int cyc = 0; cyc < a.ncyc; ++cyc) {
        const int cur = a.cur ^ (cyc & 1);
        const uint32_t zn_off = cur ? 0u : g.nkv;  // this cycle's buffer: the other one
        const Ent *__restrict__ zent = (const Ent *)(cur ? g.zent[1] : g.zent[0]);
        const Ent *__restrict__ went = (const Ent *)(cur ? g.went[1] : g.went[0]);
        const bool has_noise = a.noise != nullptr;
        const size_t noise_cyc = (size_t)cyc * a.nw * nsz;
        const int shcol = a.cyc0_in_batch + cyc;
        float tsum = 0.f;  // this lane's share of the cycle's trace series value

        // this lane's share of row i's entries: lane e holds entry e of each side
        auto load_ents = [&](const int4 &rec, Ent &mz, Ent &mw) {
            const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
            mz = lane < dz ? ldg_ent(&zent[rec.y + lane]) : ent_none<Ent>();
            mw = lane < dw ? ldg_ent(&went[rec.z + lane]) : ent_none<Ent>();
        };
        auto noise_bits = [&](int q, int p) -> uint32_t {
            return (has_noise && chain_ok[q]) ? __ldg(&noise_col[q][noise_cyc + p]) >> cshift[q] : 0u;
        };
        // Eqs. 4/5 for the V chains of the lane's vector q from the sums over the row's
        // entries, the stores, the shadows and the z_i conj(w_i) partials
        auto finish = [&](int q, int p, uint32_t iv, const T &sz, const T &sw, const Cst &k, uint32_t bits, S dold,
                          int rp, int sp) {
            S prod = P::zero();
            if (chain_ok[q]) {
                const float phi_scale = has_noise ? 1.f : 0.f;
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
                z0[zn_off + iv + cv[q]] = zv;
                w0[zn_off + iv + cv[q]] = wv;
                if (rp >= 0 || sp >= 0) {
                    const size_t o = (size_t)shcol * a.kp + (size_t)c0[q] * (CPLX ? 2 : 1);
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
                if (dlead[q]) dpart[q][p] = P::add(dold, prod);
            }
        };
        // one row with register gathers (G = 1): one batch of every gather before any
        // FMA when it has one piece, else its 2 or 4 pieces, each a sequential sum
        // from zero, joined in order
        auto row_regs = [&](int p, const int4 &rec, const Ent &mz, const Ent &mw) {
            const int lg = rec.w & 3;
            const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
            // the epilogue's operands (their latency hides behind the gathers)
            const Cst k = ldg_cst(&cstv[p]);
            const uint32_t bits = noise_bits(0, p);
            S dold = P::zero();
            if (dlead[0]) dold = dpart[0][p];
            int rp = -1, sp = -1;
            if (a.rpos && chain_ok[0]) { rp = __ldg(&a.rpos[p]); sp = __ldg(&a.spos[p]); }
            T sz = L::zero(), sw = L::zero();
            if (lg == 0) {
                T xz[U1], xw[U1];
#pragma unroll
                for (int u = 0; u < U1; ++u) {
                    const uint32_t oz = (uint32_t)__shfl_sync(0xffffffffu, mz.col, u);
                    const uint32_t ow = (uint32_t)__shfl_sync(0xffffffffu, mw.col, u);
                    xz[u] = L::zero();
                    xw[u] = L::zero();
                    if (u < dz && chain_ok[0]) xz[u] = __ldcg(&z0[oz + cv[0]]);
                    if (u < dw && chain_ok[0]) xw[u] = __ldcg(&w0[ow + cv[0]]);
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
                            if (vz && chain_ok[0]) xz[u] = __ldcg(&z0[oz + cv[0]]);
                            if (vw && chain_ok[0]) xw[u] = __ldcg(&w0[ow + cv[0]]);
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
            finish(0, p, (uint32_t)rec.x, sz, sw, k, bits, dold, rp, sp);
        };

        for (int l = 0; l < nlev; ++l) {
            const int lb = __ldg(&g.lev_ptr[l]), le = __ldg(&g.lev_ptr[l + 1]);
            int p = lb + r0;
            if (BULK && !*abort_flag && active && p < le) {
                // the bulk copies read rows that other CTAs wrote before the grid barrier
                asm volatile("fence.proxy.async.global;" ::: "memory");
                static_assert(QMAX >= 2 && QMAX <= 4, "queue registers");
                RingRow<CPLX> q0{}, q1{}, q2{}, q3{};  // rows in flight, oldest first
                int qn = 0;
                // the oldest row's epilogue operands, loaded as soon as it becomes the oldest
                Cst ek{};
                uint32_t ebits[G];
                S edold[G];
                int erp = -1, esp = -1;
                auto load_ep = [&](int pp) {
                    ek = ldg_cst(&cstv[pp]);
#pragma unroll
                    for (int q = 0; q < G; ++q) {
                        ebits[q] = noise_bits(q, pp);
                        edold[q] = P::zero();
                        if (dlead[q]) edold[q] = dpart[q][pp];
                    }
                    erp = -1;
                    esp = -1;
                    if (a.rpos) { erp = __ldg(&a.rpos[pp]); esp = __ldg(&a.spos[pp]); }
                };
#pragma unroll
                for (int q = 0; q < G; ++q) { ebits[q] = 0u; edold[q] = P::zero(); }
                // compute the oldest row in flight from its slots, which are then free
                auto pop = [&]() {
                    const RingRow<CPLX> r = q0;
                    const Cst k = ek;
                    uint32_t bits[G];
                    S dold[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) { bits[q] = ebits[q]; dold[q] = edold[q]; }
                    const int rp = erp, sp = esp;
                    q0 = q1;
                    q1 = q2;
                    q2 = q3;
                    --qn;
                    if (qn > 0) load_ep(q0.p);
                    const int dz = (r.info >> 2) & 0x7fff, dw = (r.info >> 17) & 0x7fff;
                    if (!ring_wait(bar0 + 8u * (r.use % (QMAX + 1)), (r.use / (QMAX + 1)) & 1u)) *abort_flag = 1;
                    Ent az, aw;
                    az.col = 0; aw.col = 0;
                    if constexpr (CPLX) { az.re = r.zr; az.im = r.zi; aw.re = r.wr; aw.im = r.wi; az.pad = aw.pad = 0; }
                    else { az.val = r.zr; aw.val = r.wr; }
                    const uint32_t zb = ring0 + (r.vslot & (RING - 1)) * SEGG + lane * 16u;
                    const uint32_t wb = zb + (uint32_t)dz * SEGG;
                    T sz[G], sw[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) { sz[q] = L::zero(); sw[q] = L::zero(); }
                    if ((r.info & 3) == 0) {
#pragma unroll
                        for (int u = 0; u < U1; ++u)
                            if (u < dz) {
                                const Ent e = shfl_val(az, u);
#pragma unroll
                                for (int q = 0; q < G; ++q) L::fma(sz[q], e, lds_vec<T>(zb + u * SEGG + q * SEGB));
                            }
#pragma unroll
                        for (int u = 0; u < U1; ++u)
                            if (u < dw) {
                                const Ent e = shfl_val(aw, u);
#pragma unroll
                                for (int q = 0; q < G; ++q) L::fma(sw[q], e, lds_vec<T>(wb + u * SEGG + q * SEGB));
                            }
                    } else {
#pragma unroll
                        for (int q = 0; q < G; ++q) {
                            PieceSum<L> pzs(dz, r.info & 3), pws(dw, r.info & 3);
                            for (int e = 0; e < dz; ++e) pzs.add(e, shfl_val(az, e), lds_vec<T>(zb + e * SEGG + q * SEGB));
                            for (int e = 0; e < dw; ++e) pws.add(e, shfl_val(aw, e), lds_vec<T>(wb + e * SEGG + q * SEGB));
                            sz[q] = pzs.total();
                            sw[q] = pws.total();
                        }
                    }
#pragma unroll
                    for (int q = 0; q < G; ++q) finish(q, r.p, r.iv, sz[q], sw[q], k, bits[q], dold[q], rp, sp);
                };
                // pipeline: this row's record and entries, the next row's record
                int4 rec = ldnc4(&rows[p]);
                Ent mz, mw;
                load_ents(rec, mz, mw);
                int4 rnext = p + rstep < le ? ldnc4(&rows[p + rstep]) : make_int4(0, 0, 0, 0);
                for (; p < le; p += rstep) {
                    // the next row's entries and the record of the one after
                    Ent nz, nw;
                    const bool more = p + rstep < le;
                    if (more) load_ents(rnext, nz, nw);
                    const int4 rnn = p + 2 * rstep < le ? ldnc4(&rows[p + 2 * rstep]) : make_int4(0, 0, 0, 0);
                    const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
                    const int nseg = dz + dw;
                    if (nseg <= RING) {
                        // the row's slots, not across the ring's end; wait for room and a barrier
                        uint32_t v = vhead;
                        if ((v & (RING - 1)) + nseg > RING) v = (v + RING - 1) & ~(uint32_t)(RING - 1);
                        while (qn == QMAX || (qn > 0 && v + nseg - q0.vslot > (uint32_t)RING)) pop();
                        const uint32_t bar = bar0 + 8u * (ic % (QMAX + 1));
                        const uint32_t wo = (uint32_t)__shfl_sync(0xffffffffu, mw.col, (lane - dz) & 31);
                        // every lane is done reading the slots freed above; order those
                        // generic-proxy reads before the async-proxy writes below
                        __syncwarp();
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        if (lane == 0) mbar_expect(bar, (uint32_t)nseg * seg_bytes);
                        if (lane < nseg) {
                            const T *src = lane < dz ? z0 + (uint32_t)mz.col + cvb : w0 + wo + cvb;
                            bulk_g2s(ring0 + ((v & (RING - 1)) + lane) * SEGG, src, seg_bytes, bar);
                        }
                        RingRow<CPLX> r;
                        r.p = p;
                        r.info = rec.w;
                        r.vslot = v;
                        r.iv = (uint32_t)rec.x;
                        r.use = ic;
                        if constexpr (CPLX) { r.zr = mz.re; r.zi = mz.im; r.wr = mw.re; r.wi = mw.im; }
                        else { r.zr = mz.val; r.zi = 0.f; r.wr = mw.val; r.wi = 0.f; }
                        if (qn == 0) {
                            q0 = r;
                            load_ep(p);
                        } else if (qn == 1) {
                            q1 = r;
                        } else if (QMAX == 3 || qn == 2) {
                            q2 = r;
                        } else {
                            q3 = r;
                        }
                        ++qn;
                        ++ic;
                        vhead = v + nseg;
                    } else {
                        // a long row: drain the ring, then rounds of up to RING segments
                        while (qn > 0) pop();
                        const Cst k = ldg_cst(&cstv[p]);
                        uint32_t bits[G];
                        S dold[G];
#pragma unroll
                        for (int q = 0; q < G; ++q) {
                            bits[q] = noise_bits(q, p);
                            dold[q] = P::zero();
                            if (dlead[q]) dold[q] = dpart[q][p];
                        }
                        int rp = -1, sp = -1;
                        if (a.rpos) { rp = __ldg(&a.rpos[p]); sp = __ldg(&a.spos[p]); }
                        PieceSum<L> pzs[G], pws[G];
#pragma unroll
                        for (int q = 0; q < G; ++q) { pzs[q] = PieceSum<L>(dz, rec.w & 3); pws[q] = PieceSum<L>(dw, rec.w & 3); }
                        for (int ez = 0, ew = 0; ez < dz || ew < dw;) {
                            int mzr = min(dz - ez, RING / 2);
                            const int mwr = min(dw - ew, RING - mzr);
                            mzr = min(dz - ez, RING - mwr);
                            const uint32_t oz = ent_off_lane(mz, zent, rec.y, ez + lane, lane < mzr);
                            const uint32_t ow = ent_off_lane(mw, went, rec.z, ew + lane - mzr, lane >= mzr && lane < mzr + mwr);
                            __syncwarp();
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            if (lane == 0) mbar_expect(bar_long, (uint32_t)(mzr + mwr) * seg_bytes);
                            if (lane < mzr + mwr) {
                                const T *src = lane < mzr ? z0 + oz + cvb : w0 + ow + cvb;
                                bulk_g2s(ring0 + lane * SEGG, src, seg_bytes, bar_long);
                            }
                            if (!ring_wait(bar_long, kb & 1u)) *abort_flag = 1;
                            ++kb;
                            const uint32_t sa = ring0 + lane * 16u;
                            for (int e = 0; e < mzr; ++e) {
                                const Ent en = ent_val(mz, zent, rec.y, ez + e, true);
#pragma unroll
                                for (int q = 0; q < G; ++q) pzs[q].add(ez + e, en, lds_vec<T>(sa + e * SEGG + q * SEGB));
                            }
                            for (int e = 0; e < mwr; ++e) {
                                const Ent en = ent_val(mw, went, rec.z, ew + e, true);
#pragma unroll
                                for (int q = 0; q < G; ++q) pws[q].add(ew + e, en, lds_vec<T>(sa + (mzr + e) * SEGG + q * SEGB));
                            }
                            ez += mzr;
                            ew += mwr;
                        }
#pragma unroll
                        for (int q = 0; q < G; ++q)
                            finish(q, p, (uint32_t)rec.x, pzs[q].total(), pws[q].total(), k, bits[q], dold[q], rp, sp);
                    }
                    if (more) { rec = rnext; mz = nz; mw = nw; }
                    rnext = rnn;
                }
                while (qn > 0) pop();
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

template <bool CPLX, int V, int NT, bool BULK, int G>
cudaError_t launch_grid_v(const SweepArgs &a, const GridArgs &g, int ctas, cudaStream_t s)
{
    auto kern = cc_sweep_grid_kernel<CPLX, V, NT, BULK, G>;
    const size_t smem = BULK ? bulk_smem<G>() : 0;
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

template <bool CPLX, int V, int NT, bool BULK, int G>
int grid_blocks_per_sm()
{
    auto kern = cc_sweep_grid_kernel<CPLX, V, NT, BULK, G>;
    const size_t smem = BULK ? bulk_smem<G>() : 0;
    int per_sm = 0;
    if ((BULK && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

}  // namespace

bool grid_supported(int cplx, int chains_per_lane, int64_t K, int threads, bool bulk)
{
    const int v = cplx ? 2 : 4;
    if (chains_per_lane != v || K % v != 0) return false;
    if (bulk) return threads == BULK_THREADS || threads == BULK_THREADS / 2 || threads == BULK_THREADS / 4;
    return threads == 384 || threads == 512;
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
    const int G = bulk ? BULK_THREADS / threads : 1;
    if ((long long)ctas * (threads / 32) < (g.nblk + G - 1) / G) return cudaErrorInvalidConfiguration;
    // the barrier counter starts at zero in every launch
    cudaError_t e = cudaMemsetAsync(g.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (bulk) {
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
