// sweep_ring.cuh -- the row pipeline of the row-per-warp sweeps (Eqs. 4 and 5).
//
// A warp updates one row for a block of 32 x V x G chains (G 32-vector blocks,
// G x 512 contiguous bytes of z or w per gathered row), gathering the
// neighbours' segments either into registers or, with bulk staging, into a ring
// of shared-memory slots with cp.async.bulk, several rows in flight.  Used by
// the grid-wide sweep of one matrix (sweep_grid.cu: all CTAs share each
// dependency level, a grid barrier between levels) and by the pool's sweep
// (pool.cu: a CTA owns one matrix's chain block, a CTA barrier between levels).
// Entries carry the gathered vector's index from the base of the two state
// buffers for one cycle parity (this cycle's buffer for j < i, last cycle's for
// j > i: the in-place ascending sweep), so a gather is a shuffle, an address
// and a load.  The arithmetic is that of the chain-sliced kernel in the same
// order (pieces of long rows summed as ((p0 + p1) + p2) + p3, explicit
// round-to-nearest FMAs), so every kernel gives the same bits.  Every wait is
// bounded (2 s of globaltimer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "sweep_core.cuh"

namespace mcinv {
namespace ring {

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

// The bulk-staged variant gives each warp a ring of 512-byte slots (RING or RING16) in
// shared memory.  A row's gathered segments go to consecutive slots of the
// ring (never across its end), one cp.async.bulk each, completing on one of
// QMAX + 1 mbarriers; up to QMAX rows are in flight while the warp computes the
// oldest, so the gathers take no registers and a warp keeps about a ring of
// segments in flight.  A row of more segments than the ring has slots waits for
// the ring to drain and then runs in rounds of a ring each on a barrier of its
// own.  Every slot index is taken modulo the ring's slot count.
constexpr int RING = 32;                  // slots per warp (12 warps a CTA)
constexpr int RING16 = 24;                // slots per warp with 16 warps a CTA (same 12 KB a warp as PAIR_RN)
constexpr int QMAX = 3;                   // rows in flight per warp
constexpr int NBAR = QMAX + 2;            // QMAX + 1 for the ring rows, one for long rows
constexpr int SEGB = 512;                 // 32 lanes x 16 bytes
constexpr int PAIR_RN = 12;               // 1 KB slots per warp on the pair layout with 16 warps a CTA

// A row in flight in a warp's ring: its position, first vector i K / V, packed
// counts, first slot, barrier use number, and the lane's values of its entries
// (lane e holds entry e of each side; the offsets were used when issued).
template <bool CPLX>
struct RingRow {
    int p, info;
    uint32_t vslot;  // first slot, counted from the warp's start (slot vslot mod the ring's slots)
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


// The lane's share of a warp's chain block: G vectors l, l + 32, ..., each
// handled exactly as the one-vector kernel's lane l of the 32-vector block it
// falls in (same diagonal units, same bits); plus the warp's ring in shared
// memory and its running state.
template <bool CPLX, int V, int G>
struct Lanes {
    using S = typename Prec<CPLX>::T;
    int lane, seg;
    bool diag;                      // diagonal partials on
    int c0[G];
    bool ok[G], dlead[G];
    uint32_t cv[G], cshift[G];
    S *dpart[G];
    const uint32_t *noise_col[G];   // the lane's noise words of cycle 0, by position, or null
    uint32_t zo[G], wo[G];          // the lane's z and w vectors within a row of the state
    uint32_t ring0, bar0, bar_long; // the ring and its barriers (bulk staging)
    uint32_t cvb, seg_bytes;        // the block's first vector in a row; bytes of one segment
    uint32_t ic, kb, vhead;         // ring rows issued, long-row rounds, next free slot

    // blk: the warp's chain block (G x 32 vectors); kv: vectors per row; K chains;
    // dp: diagonal partials [units][n] by position, or null; noise: [cycle][nw][n]
    // by position, or null
    // pair: the state is in the pair layout (see PairLayout below; G = 1)
    __device__ __forceinline__ void init(int lane_, int blk, int kv, int K, int n, int seg_, void *dp,
                                         const uint32_t *noise, uint32_t ring0_, uint32_t bar0_, bool pair = false)
    {
        lane = lane_;
        seg = seg_;
        ring0 = ring0_;
        bar0 = bar0_;
        bar_long = bar0 + (NBAR - 1) * 8u;
        ic = kb = vhead = 0;
        set_block(blk, kv, K, n, dp, noise, pair);
    }
    // the chain block, the diagonal partials and the noise plane (the ring and its
    // state are kept)
    __device__ __forceinline__ void set_block(int blk, int kv, int K, int n, void *dp, const uint32_t *noise,
                                              bool pair = false)
    {
        diag = dp != nullptr;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            cv[q] = (uint32_t)(blk * 32 * G + q * 32 + lane);
            c0[q] = (int)cv[q] * V;
            ok[q] = c0[q] < K;
            dpart[q] = (S *)dp + (size_t)(c0[q] / (seg * V)) * (size_t)n;
            // the lane that adds the unit's sum to its partial: the unit's first lane; with
            // two vectors a lane and units of two or more lanes, vector 1's unit sum ends in
            // the unit's second lane (diag_pair), which stores it if the unit has chains
            if (G == 2 && q == 1 && seg >= 2)
                dlead[q] = ((lane % seg) == 1) && (c0[q] - V < K) && diag;
            else
                dlead[q] = ((lane % seg) == 0) && ok[q] && diag;
            noise_col[q] = noise ? noise + (size_t)(c0[q] >> 5) * (size_t)n : nullptr;
            cshift[q] = (uint32_t)(c0[q] & 31);
        }
        if (pair) {
            // a row's 32-vector block b: 32 z vectors, then the same chains' 32 w
            // vectors; the warp's G blocks are adjacent (the last may be past the row)
#pragma unroll
            for (int q = 0; q < G; ++q) {
                zo[q] = (uint32_t)((blk * G + q) * 64 + lane);
                wo[q] = zo[q] + 32u;
            }
            cvb = (uint32_t)(blk * G * 64);
            seg_bytes = (uint32_t)min(G, (kv + 31) / 32 - blk * G) * 2u * SEGB;
        } else {
#pragma unroll
            for (int q = 0; q < G; ++q) zo[q] = wo[q] = cv[q];
            cvb = (uint32_t)(blk * 32 * G);
            seg_bytes = (uint32_t)min(32 * G, kv - blk * 32 * G) * 16u;
        }
    }
    // the noise word of vector q at position p in the cycle starting noise_cyc words in
    __device__ __forceinline__ uint32_t bits(int q, int p, size_t noise_cyc) const
    {
        return (noise_col[q] && ok[q]) ? __ldg(&noise_col[q][noise_cyc + p]) >> cshift[q] : 0u;
    }
};

// One matrix in one cycle, as the row pipeline reads and writes it.
template <bool CPLX>
struct Mat {
    using P = Prec<CPLX>;
    const GridRow *rows;                  // by position; .row holds i K / V
    const typename P::Ent *zent, *went;   // this cycle parity's entries (.col: vector index from z0 / w0)
    const typename P::Cst *cst;           // by position
    void *z0, *w0;                        // the two state buffers of z: z0 and z0 + nkv vectors (same for w)
    uint32_t zn_off;                      // this cycle's buffer, in vectors from z0
    size_t noise_cyc;                     // this cycle's noise words, from the lanes' noise_col
    bool has_noise;
    bool check_div;                       // this cycle checks for diverged chains (the launch's last)
    const int *rpos, *spos;               // BF16 shadows: by position, index in R / S or -1; or null
    uint16_t *zsh, *wsh;
    long long ldsh, kp;
    int shcol;
    const float *tq;                      // trace weights by position, or null
};

// Eqs. 4/5 for the V chains of the lane's vector q from the sums over the row's
// entries, the stores, the shadows and the trace term; returns the lane's
// z_i conj(w_i) partial for the diagonal (diag_one / diag_pair) and leaves the
// new values in zv, wv (unset when the lane's chains are past K).
template <bool CPLX, int V, int G>
__device__ __forceinline__ typename Prec<CPLX>::T finish_keep(const Lanes<CPLX, V, G> &w, const Mat<CPLX> &m, int q, int p,
                                            uint32_t iv, const typename Lane<CPLX, V>::T &sz,
                                            const typename Lane<CPLX, V>::T &sw, const typename Prec<CPLX>::Cst &k,
                                            uint32_t bits, typename Prec<CPLX>::T dold, int rp, int sp, float &tsum,
                                            bool &diverged, typename Lane<CPLX, V>::T &zv, typename Lane<CPLX, V>::T &wv)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    S prod = P::zero();
    if (w.ok[q]) {
        // phi alpha and phi beta (Eq. 5): phi = +-1 flips the sign bit; no noise: phi = +0
        const S a0 = m.has_noise ? k.alpha : P::times_zero(k.alpha);
        const S b0 = m.has_noise ? k.beta : P::times_zero(k.beta);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t sign = ((bits >> v) & 1u) << 31;
            L::set(zv, v, P::zrow_a(k, P::flip(a0, sign), L::get(sz, v)));
            L::set(wv, v, P::wrow_a(k, P::flip(b0, sign), L::get(sw, v)));
        }
        // a diverging chain stays beyond the bound, so the launch's last cycle tells
        if (m.check_div) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                diverged |= !(P::finite_bounded(L::get(zv, v)) && P::finite_bounded(L::get(wv, v)));
        }
        if (w.diag || m.tq) {
#pragma unroll
            for (int v = 0; v < V; ++v) prod = P::add(prod, P::mulconj(L::get(zv, v), L::get(wv, v)));
        }
        if (m.tq) {
            float re;
            if constexpr (CPLX) re = prod.x;
            else re = prod;
            tsum = __fmaf_rn(__ldg(&m.tq[p]), re, tsum);
        }
        ((T *)m.z0)[m.zn_off + iv + w.zo[q]] = zv;
        ((T *)m.w0)[m.zn_off + iv + w.wo[q]] = wv;
        if (rp >= 0 || sp >= 0) {
            const size_t o = (size_t)m.shcol * m.kp + (size_t)w.c0[q] * (CPLX ? 2 : 1);
            constexpr int NF = L::NF;
            if (rp >= 0) store_bf16<NF>(m.zsh + (size_t)rp * m.ldsh + o, L::f(zv));
            if (sp >= 0) {
                if constexpr (!CPLX) {
                    store_bf16<NF>(m.wsh + (size_t)sp * m.ldsh + o, L::f(wv));
                } else {
                    // rows 2s = [wr, wi] and 2s+1 = [-wi, wr]: one real
                    // contraction gives Re and Im of z conj(w) interleaved
                    uint16_t *wr0 = m.wsh + (size_t)(2 * sp) * m.ldsh + o;
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
                    store_bf16<2 * V>(wr0 + m.ldsh, f1);
                }
            }
        }
    }
    return prod;
}

template <bool CPLX, int V, int G>
__device__ __forceinline__ typename Prec<CPLX>::T finish(const Lanes<CPLX, V, G> &w, const Mat<CPLX> &m, int q, int p, uint32_t iv,
                                       const typename Lane<CPLX, V>::T &sz, const typename Lane<CPLX, V>::T &sw,
                                       const typename Prec<CPLX>::Cst &k, uint32_t bits, typename Prec<CPLX>::T dold,
                                       int rp, int sp, float &tsum, bool &diverged)
{
    typename Lane<CPLX, V>::T zv, wv;
    return finish_keep<CPLX, V, G>(w, m, q, p, iv, sz, sw, k, bits, dold, rp, sp, tsum, diverged, zv, wv);
}

// The unit's sum of the lanes' z_i conj(w_i) over its seg lanes (xor butterfly:
// every lane of the unit ends with the same sum); its leader adds it to the
// running partial.
template <bool CPLX, int V, int G>
__device__ __forceinline__ void diag_one(const Lanes<CPLX, V, G> &w, int q, int p, typename Prec<CPLX>::T prod,
                                         typename Prec<CPLX>::T dold)
{
    using P = Prec<CPLX>;
    if (!w.diag) return;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1)
        if (o < w.seg) prod = P::add(prod, P::shfl_xor(prod, o));
    if (w.dlead[q]) w.dpart[q][p] = P::add(dold, prod);
}

// The same for both vectors of a two-vector lane at once: at the first level
// even lanes keep vector 0's pair sum and odd lanes vector 1's (each lane sends
// the other), then one butterfly over the unit's lanes of the same parity.  The
// additions are those of two separate butterflies (a + b = b + a), so the unit
// sums are the same bits, in the unit's even lanes for vector 0 and odd lanes
// for vector 1.
template <bool CPLX, int V>
__device__ __forceinline__ void diag_pair(const Lanes<CPLX, V, 2> &w, int p, typename Prec<CPLX>::T pr0,
                                          typename Prec<CPLX>::T pr1, typename Prec<CPLX>::T dold0,
                                          typename Prec<CPLX>::T dold1)
{
    using P = Prec<CPLX>;
    using S = typename P::T;
    if (!w.diag) return;
    if (w.seg == 1) {
        if (w.dlead[0]) w.dpart[0][p] = P::add(dold0, pr0);
        if (w.dlead[1]) w.dpart[1][p] = P::add(dold1, pr1);
        return;
    }
    const bool odd = (w.lane & 1) != 0;
    S keep = odd ? pr1 : pr0;
    keep = P::add(keep, P::shfl_xor(odd ? pr0 : pr1, 1));
#pragma unroll
    for (int o = 2; o < 32; o <<= 1)
        if (o < w.seg) keep = P::add(keep, P::shfl_xor(keep, o));
    if (w.dlead[0]) w.dpart[0][p] = P::add(dold0, keep);
    if (w.dlead[1]) w.dpart[1][p] = P::add(dold1, keep);
}

// this lane's share of row p's entries: lane e holds entry e of each side
template <bool CPLX>
__device__ __forceinline__ void load_ents(const Mat<CPLX> &m, int lane, const int4 &rec, typename Prec<CPLX>::Ent &mz,
                                          typename Prec<CPLX>::Ent &mw)
{
    using Ent = typename Prec<CPLX>::Ent;
    const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
    mz = lane < dz ? ldg_ent(&m.zent[rec.y + lane]) : ent_none<Ent>();
    mw = lane < dw ? ldg_ent(&m.went[rec.z + lane]) : ent_none<Ent>();
}

// One row with register gathers (G = 1): one batch of every gather before any
// FMA when it has one piece, else its 2 or 4 pieces, each a sequential sum from
// zero, joined in order.
template <bool CPLX, int V>
__device__ __forceinline__ void row_regs(const Lanes<CPLX, V, 1> &w, const Mat<CPLX> &m, int p, const int4 &rec,
                                         const typename Prec<CPLX>::Ent &mz, const typename Prec<CPLX>::Ent &mw,
                                         float &tsum, bool &diverged)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    constexpr int U1 = 8;  // a whole row (at most SPLIT_ENTRIES entries a side)
    constexpr int UP = 4;  // batches of a piece of a long row
    const T *z0 = (const T *)m.z0, *w0 = (const T *)m.w0;
    const int lg = rec.w & 3;
    const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
    // the epilogue's operands (their latency hides behind the gathers)
    const typename P::Cst k = ldg_cst(&m.cst[p]);
    const uint32_t bits = w.bits(0, p, m.noise_cyc);
    S dold = P::zero();
    if (w.dlead[0]) dold = w.dpart[0][p];
    int rp = -1, sp = -1;
    if (m.rpos && w.ok[0]) { rp = __ldg(&m.rpos[p]); sp = __ldg(&m.spos[p]); }
    T sz = L::zero(), sw = L::zero();
    if (lg == 0) {
        T xz[U1], xw[U1];
#pragma unroll
        for (int u = 0; u < U1; ++u) {
            const uint32_t oz = (uint32_t)__shfl_sync(0xffffffffu, mz.col, u);
            const uint32_t ow = (uint32_t)__shfl_sync(0xffffffffu, mw.col, u);
            xz[u] = L::zero();
            xw[u] = L::zero();
            if (u < dz && w.ok[0]) xz[u] = __ldcg(&z0[oz + w.zo[0]]);
            if (u < dw && w.ok[0]) xw[u] = __ldcg(&w0[ow + w.wo[0]]);
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
                    const uint32_t oz = ent_off(mz, m.zent, rec.y, ez + u, vz);
                    const uint32_t ow = ent_off(mw, m.went, rec.z, ew + u, vw);
                    xz[u] = L::zero();
                    xw[u] = L::zero();
                    if (vz && w.ok[0]) xz[u] = __ldcg(&z0[oz + w.zo[0]]);
                    if (vw && w.ok[0]) xw[u] = __ldcg(&w0[ow + w.wo[0]]);
                }
#pragma unroll
                for (int u = 0; u < UP; ++u) {
                    const bool vz = ez + u < zeN, vw = ew + u < weN;
                    const Ent ez_ = ent_val(mz, m.zent, rec.y, ez + u, vz);
                    const Ent ew_ = ent_val(mw, m.went, rec.z, ew + u, vw);
                    if (vz) L::fma(pz, ez_, xz[u]);
                    if (vw) L::fma(pw, ew_, xw[u]);
                }
            }
            if (pk == 0) { sz = pz; sw = pw; }
            else { sz = L::add(sz, pz); sw = L::add(sw, pw); }
        }
    }
    diag_one(w, 0, p, finish<CPLX, V, 1>(w, m, 0, p, (uint32_t)rec.x, sz, sw, k, bits, dold, rp, sp, tsum, diverged), dold);
}

// The rows p, p + rstep, ... (< le) of one level with register gathers, the next
// row's record and entries loaded while this row's gathers are in flight.
template <bool CPLX, int V>
__device__ __forceinline__ void level_regs(const Lanes<CPLX, V, 1> &w, const Mat<CPLX> &m, int p, int le, int rstep,
                                           float &tsum, bool &diverged)
{
    using Ent = typename Prec<CPLX>::Ent;
    if (p >= le) return;
    int4 rec = ldnc4(&m.rows[p]);
    Ent mz, mw;
    load_ents(m, w.lane, rec, mz, mw);
    int4 nrec = p + rstep < le ? ldnc4(&m.rows[p + rstep]) : make_int4(0, 0, 0, 0);
    for (; p < le; p += rstep) {
        Ent nz, nw;
        const bool more = p + rstep < le;
        if (more) load_ents(m, w.lane, nrec, nz, nw);
        const int4 nnrec = p + 2 * rstep < le ? ldnc4(&m.rows[p + 2 * rstep]) : make_int4(0, 0, 0, 0);
        row_regs<CPLX, V>(w, m, p, rec, mz, mw, tsum, diverged);
        if (more) { rec = nrec; mz = nz; mw = nw; }
        nrec = nnrec;
    }
}

// The rows p, p + rstep, ... (< le) of one level with bulk-staged gathers: a row
// of at most RNS segments goes to consecutive slots of the warp's ring of RNS
// slots (never across its end), its segments one cp.async.bulk each, completing
// on one of QMAX + 1 barriers; up to QMAX rows are in flight while the oldest is
// computed.  A longer row drains the ring and runs in rounds of RNS segments.  The caller
// has ordered the last level's state stores before these async-proxy reads
// (fence.proxy.async after the level barrier).  On an expired wait *abort_flag
// is set and the rows are finished with whatever landed.
//
// PAIR: the state is in the pair layout (the chain block's z vectors of a row
// followed by its w vectors, one allocation for both) and the matrix is
// structurally symmetric (row i of C and of C^dagger name the same j, in the
// same order), so z_j and w_j of a neighbour's 32-vector block are one 1 KB
// segment, and the G adjacent blocks of the warp one G KB copy into one slot.
template <bool CPLX, int V, int G, bool PAIR = false, int RNS = RING>
__device__ __forceinline__ void level_bulk(Lanes<CPLX, V, G> &w, const Mat<CPLX> &m, int p, int le, int rstep,
                                           float &tsum, bool &diverged, volatile int *abort_flag)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    constexpr int U1 = 8;
    constexpr int SEGG = PAIR ? 2 * SEGB * G : SEGB * G;  // bytes of one slot
    constexpr int RN = RNS;                               // slots of the warp's ring
    constexpr int WOFF = PAIR ? SEGB : 0;                 // the w half of a block's pair
    constexpr int QOFF = PAIR ? 2 * SEGB : SEGB;          // vector q of a lane, from vector 0
    static_assert(QMAX >= 2 && QMAX <= 4, "queue registers");
    static_assert(RN >= 2 && RN <= 32, "a ring's copies take a lane each");
    if (p >= le) return;
    const int lane = w.lane;
    T *const z0 = (T *)m.z0;
    T *const w0 = (T *)m.w0;
    RingRow<CPLX> q0{}, q1{}, q2{}, q3{};  // rows in flight, oldest first
    int qn = 0;
    // the oldest row's epilogue operands, loaded as soon as it becomes the oldest
    Cst ek{};
    uint32_t ebits[G];
    S edold[G];
    int erp = -1, esp = -1;
#pragma unroll
    for (int q = 0; q < G; ++q) { ebits[q] = 0u; edold[q] = P::zero(); }
    auto load_ep = [&](int pp) {
        ek = ldg_cst(&m.cst[pp]);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            ebits[q] = w.bits(q, pp, m.noise_cyc);
            edold[q] = P::zero();
            if (w.dlead[q]) edold[q] = w.dpart[q][pp];
        }
        erp = -1;
        esp = -1;
        if (m.rpos) { erp = __ldg(&m.rpos[pp]); esp = __ldg(&m.spos[pp]); }
    };
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
        if (!ring_wait(w.bar0 + 8u * (r.use % (QMAX + 1)), (r.use / (QMAX + 1)) & 1u)) *abort_flag = 1;
        Ent az, aw;
        az.col = 0; aw.col = 0;
        if constexpr (CPLX) { az.re = r.zr; az.im = r.zi; aw.re = r.wr; aw.im = r.wi; az.pad = aw.pad = 0; }
        else { az.val = r.zr; aw.val = r.wr; }
        const uint32_t zb = w.ring0 + (r.vslot % RN) * SEGG + lane * 16u;
        const uint32_t wb = PAIR ? zb + WOFF : zb + (uint32_t)dz * SEGG;
        T sz[G], sw[G];
#pragma unroll
        for (int q = 0; q < G; ++q) { sz[q] = L::zero(); sw[q] = L::zero(); }
        if ((r.info & 3) == 0) {
            // entries 0..3, then 4..7 where the row has them (one branch for both sides)
#pragma unroll
            for (int u = 0; u < U1 / 2; ++u)
                if (u < dz) {
                    const Ent e = shfl_val(az, u);
#pragma unroll
                    for (int q = 0; q < G; ++q) L::fma(sz[q], e, lds_vec<T>(zb + u * SEGG + q * QOFF));
                }
#pragma unroll
            for (int u = 0; u < U1 / 2; ++u)
                if (u < dw) {
                    const Ent e = shfl_val(aw, u);
#pragma unroll
                    for (int q = 0; q < G; ++q) L::fma(sw[q], e, lds_vec<T>(wb + u * SEGG + q * QOFF));
                }
            if (dz > U1 / 2 || dw > U1 / 2) {
#pragma unroll
                for (int u = U1 / 2; u < U1; ++u)
                    if (u < dz) {
                        const Ent e = shfl_val(az, u);
#pragma unroll
                        for (int q = 0; q < G; ++q) L::fma(sz[q], e, lds_vec<T>(zb + u * SEGG + q * QOFF));
                    }
#pragma unroll
                for (int u = U1 / 2; u < U1; ++u)
                    if (u < dw) {
                        const Ent e = shfl_val(aw, u);
#pragma unroll
                        for (int q = 0; q < G; ++q) L::fma(sw[q], e, lds_vec<T>(wb + u * SEGG + q * QOFF));
                    }
            }
        } else {
#pragma unroll
            for (int q = 0; q < G; ++q) {
                PieceSum<L> pzs(dz, r.info & 3), pws(dw, r.info & 3);
                for (int e = 0; e < dz; ++e) pzs.add(e, shfl_val(az, e), lds_vec<T>(zb + e * SEGG + q * QOFF));
                for (int e = 0; e < dw; ++e) pws.add(e, shfl_val(aw, e), lds_vec<T>(wb + e * SEGG + q * QOFF));
                sz[q] = pzs.total();
                sw[q] = pws.total();
            }
        }
#pragma unroll
        S pr[G];
#pragma unroll
        for (int q = 0; q < G; ++q)
            pr[q] = finish<CPLX, V, G>(w, m, q, r.p, r.iv, sz[q], sw[q], k, bits[q], dold[q], rp, sp, tsum, diverged);
        if constexpr (G == 2) {
            diag_pair<CPLX, V>(w, r.p, pr[0], pr[1], dold[0], dold[1]);
        } else {
#pragma unroll
            for (int q = 0; q < G; ++q) diag_one(w, q, r.p, pr[q], dold[q]);
        }
    };
    // pipeline: this row's record and entries, the next row's record
    int4 rec = ldnc4(&m.rows[p]);
    Ent mz, mw;
    load_ents(m, lane, rec, mz, mw);
    int4 rnext = p + rstep < le ? ldnc4(&m.rows[p + rstep]) : make_int4(0, 0, 0, 0);
    for (; p < le; p += rstep) {
        // the next row's entries and the record of the one after
        Ent nz, nw;
        const bool more = p + rstep < le;
        if (more) load_ents(m, lane, rnext, nz, nw);
        const int4 rnn = p + 2 * rstep < le ? ldnc4(&m.rows[p + 2 * rstep]) : make_int4(0, 0, 0, 0);
        const int dz = (rec.w >> 2) & 0x7fff, dw = (rec.w >> 17) & 0x7fff;
        const int nseg = PAIR ? dz : dz + dw;
        if (nseg <= RN) {
            // the row's slots, not across the ring's end; wait for room and a barrier
            uint32_t v = w.vhead;
            if ((v % RN) + nseg > RN) v = (v / RN + 1) * RN;
            while (qn == QMAX || (qn > 0 && v + nseg - q0.vslot > (uint32_t)RN)) pop();
            const uint32_t bar = w.bar0 + 8u * (w.ic % (QMAX + 1));
            const uint32_t wo = (uint32_t)__shfl_sync(0xffffffffu, mw.col, (lane - dz) & 31);
            // every lane is done reading the slots freed above; order those
            // generic-proxy reads before the async-proxy writes below
            __syncwarp();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (lane == 0) mbar_expect(bar, (uint32_t)nseg * w.seg_bytes);
            if (lane < nseg) {
                const T *src = (PAIR || lane < dz) ? z0 + (uint32_t)mz.col + w.cvb : w0 + wo + w.cvb;
                bulk_g2s(w.ring0 + ((v % RN) + lane) * SEGG, src, w.seg_bytes, bar);
            }
            RingRow<CPLX> r;
            r.p = p;
            r.info = rec.w;
            r.vslot = v;
            r.iv = (uint32_t)rec.x;
            r.use = w.ic;
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
            ++w.ic;
            w.vhead = v + nseg;
        } else {
            // a long row: drain the ring, then rounds of up to RN segments
            while (qn > 0) pop();
            const Cst k = ldg_cst(&m.cst[p]);
            uint32_t bits[G];
            S dold[G];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                bits[q] = w.bits(q, p, m.noise_cyc);
                dold[q] = P::zero();
                if (w.dlead[q]) dold[q] = w.dpart[q][p];
            }
            int rp = -1, sp = -1;
            if (m.rpos) { rp = __ldg(&m.rpos[p]); sp = __ldg(&m.spos[p]); }
            PieceSum<L> pzs[G], pws[G];
#pragma unroll
            for (int q = 0; q < G; ++q) { pzs[q] = PieceSum<L>(dz, rec.w & 3); pws[q] = PieceSum<L>(dw, rec.w & 3); }
            for (int ez = 0, ew = 0; ez < dz || ew < dw;) {
                // one round: z and w segments (or pairs) of the next entries
                int mzr, mwr;
                if constexpr (PAIR) {
                    mzr = mwr = min(dz - ez, RN);
                } else {
                    mzr = min(dz - ez, RN / 2);
                    mwr = min(dw - ew, RN - mzr);
                    mzr = min(dz - ez, RN - mwr);
                }
                const int ncp = PAIR ? mzr : mzr + mwr;
                const uint32_t oz = ent_off_lane(mz, m.zent, rec.y, ez + lane, lane < mzr);
                const uint32_t ow = PAIR ? 0u : ent_off_lane(mw, m.went, rec.z, ew + lane - mzr, lane >= mzr && lane < mzr + mwr);
                __syncwarp();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (lane == 0) mbar_expect(w.bar_long, (uint32_t)ncp * w.seg_bytes);
                if (lane < ncp) {
                    const T *src = (PAIR || lane < mzr) ? z0 + oz + w.cvb : w0 + ow + w.cvb;
                    bulk_g2s(w.ring0 + lane * SEGG, src, w.seg_bytes, w.bar_long);
                }
                if (!ring_wait(w.bar_long, w.kb & 1u)) *abort_flag = 1;
                ++w.kb;
                const uint32_t sa = w.ring0 + lane * 16u;
                for (int e = 0; e < mzr; ++e) {
                    const Ent en = ent_val(mz, m.zent, rec.y, ez + e, true);
#pragma unroll
                    for (int q = 0; q < G; ++q) pzs[q].add(ez + e, en, lds_vec<T>(sa + e * SEGG + q * QOFF));
                }
                for (int e = 0; e < mwr; ++e) {
                    const Ent en = ent_val(mw, m.went, rec.z, ew + e, true);
#pragma unroll
                    for (int q = 0; q < G; ++q)
                        pws[q].add(ew + e, en, lds_vec<T>(sa + (PAIR ? e * SEGG + WOFF : (mzr + e) * SEGG) + q * QOFF));
                }
                ez += mzr;
                ew += mwr;
            }
            S pr[G];
#pragma unroll
            for (int q = 0; q < G; ++q)
                pr[q] = finish<CPLX, V, G>(w, m, q, p, (uint32_t)rec.x, pzs[q].total(), pws[q].total(), k, bits[q],
                                           dold[q], rp, sp, tsum, diverged);
            if constexpr (G == 2) {
                diag_pair<CPLX, V>(w, p, pr[0], pr[1], dold[0], dold[1]);
            } else {
#pragma unroll
                for (int q = 0; q < G; ++q) diag_one(w, q, p, pr[q], dold[q]);
            }
        }
        if (more) { rec = rnext; mz = nz; mw = nw; }
        rnext = rnn;
    }
    while (qn > 0) pop();
}

}  // namespace ring
}  // namespace mcinv
