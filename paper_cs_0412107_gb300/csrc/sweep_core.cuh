// sweep_core.cuh -- the row arithmetic of the coupled sweep (Eqs. 4 and 5)
// and the staging of the chunk stream, shared by the single-matrix sweep
// (sweep.cu) and the pool's persistent sweep (pool.cu), so both compute the
// same values in the same order.
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace mcinv {

// ---------------------------------------------------------------------------
// Scalar helpers for the two sweep precisions.
// ---------------------------------------------------------------------------
template <bool CPLX> struct Prec;
template <> struct Prec<false> {
    using T = float;
    using Ent = EntR;
    using Cst = CstR;
    static __device__ __forceinline__ T zero() { return 0.f; }
    static __device__ __forceinline__ void fma(T &acc, const Ent &e, T x) { acc = __fmaf_rn(e.val, x, acc); }
    // Eq. 4 / Eq. 5 right-hand sides
    // every operation is an explicit fmaf / mul / add with round-to-nearest, so
    // all template instantiations (any slice shape) give the same bits
    static __device__ __forceinline__ T zrow(const Cst &k, float phi, T s) { return __fmaf_rn(-k.inv_d, s, phi * k.alpha); }
    static __device__ __forceinline__ T wrow(const Cst &k, float phi, T s) { return __fmaf_rn(-k.inv_d, s, phi * k.beta); }
    // the same with phi * alpha (phi * beta) given: phi = +-1 only flips the sign bit
    static __device__ __forceinline__ T zrow_a(const Cst &k, T pa, T s) { return __fmaf_rn(-k.inv_d, s, pa); }
    static __device__ __forceinline__ T wrow_a(const Cst &k, T pb, T s) { return __fmaf_rn(-k.inv_d, s, pb); }
    static __device__ __forceinline__ T flip(T a, uint32_t sign) { return __int_as_float(__float_as_int(a) ^ (int)sign); }
    static __device__ __forceinline__ T times_zero(T a) { return 0.f * a; }
    static __device__ __forceinline__ T mulconj(T a, T b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ T add(T a, T b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ T shfl_xor(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    static __device__ __forceinline__ bool finite_bounded(T v) { return fabsf(v) <= 1e30f; }
};
template <> struct Prec<true> {
    using T = float2;
    using Ent = EntC;
    using Cst = CstC;
    static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ void fma(T &acc, const Ent &e, T x)
    {
        acc.x = __fmaf_rn(e.re, x.x, __fmaf_rn(-e.im, x.y, acc.x));
        acc.y = __fmaf_rn(e.re, x.y, __fmaf_rn(e.im, x.x, acc.y));
    }
    static __device__ __forceinline__ T zrow(const Cst &k, float phi, T s)
    {   // phi alpha - inv_d s   (phi = +-1, so phi*alpha is exact)
        const float re = __fmaf_rn(-k.inv_d.y, s.y, __fmul_rn(k.inv_d.x, s.x));
        const float im = __fmaf_rn(k.inv_d.y, s.x, __fmul_rn(k.inv_d.x, s.y));
        return make_float2(__fsub_rn(phi * k.alpha.x, re), __fsub_rn(phi * k.alpha.y, im));
    }
    static __device__ __forceinline__ T wrow(const Cst &k, float phi, T s)
    {   // phi beta - conj(inv_d) s
        const float re = __fmaf_rn(k.inv_d.y, s.y, __fmul_rn(k.inv_d.x, s.x));
        const float im = __fmaf_rn(-k.inv_d.y, s.x, __fmul_rn(k.inv_d.x, s.y));
        return make_float2(__fsub_rn(phi * k.beta.x, re), __fsub_rn(phi * k.beta.y, im));
    }
    // the same with phi * alpha (phi * beta) given
    static __device__ __forceinline__ T zrow_a(const Cst &k, T pa, T s)
    {
        const float re = __fmaf_rn(-k.inv_d.y, s.y, __fmul_rn(k.inv_d.x, s.x));
        const float im = __fmaf_rn(k.inv_d.y, s.x, __fmul_rn(k.inv_d.x, s.y));
        return make_float2(__fsub_rn(pa.x, re), __fsub_rn(pa.y, im));
    }
    static __device__ __forceinline__ T wrow_a(const Cst &k, T pb, T s)
    {
        const float re = __fmaf_rn(k.inv_d.y, s.y, __fmul_rn(k.inv_d.x, s.x));
        const float im = __fmaf_rn(-k.inv_d.y, s.x, __fmul_rn(k.inv_d.x, s.y));
        return make_float2(__fsub_rn(pb.x, re), __fsub_rn(pb.y, im));
    }
    static __device__ __forceinline__ T flip(T a, uint32_t sign)
    {
        return make_float2(__int_as_float(__float_as_int(a.x) ^ (int)sign), __int_as_float(__float_as_int(a.y) ^ (int)sign));
    }
    static __device__ __forceinline__ T times_zero(T a) { return make_float2(0.f * a.x, 0.f * a.y); }
    static __device__ __forceinline__ T mulconj(T a, T b)
    {   // a conj(b)
        return make_float2(__fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)), __fmaf_rn(-a.x, b.y, __fmul_rn(a.y, b.x)));
    }
    static __device__ __forceinline__ T add(T a, T b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
    static __device__ __forceinline__ T shfl_xor(T v, int o)
    {
        return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
    }
    static __device__ __forceinline__ bool finite_bounded(T v) { return fabsf(v.x) <= 1e30f && fabsf(v.y) <= 1e30f; }
};

__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// NF BF16 values to dst.  Four of them are 8 bytes at an 8-byte boundary (shadow rows
// are padded to 64 elements and a lane's chain offset is a multiple of 4 elements)
// and go out as one 64-bit store.
template <int NF>
__device__ __forceinline__ void store_bf16(uint16_t *dst, const float *v)
{
    if constexpr (NF == 4) {
        const uint32_t lo = (uint32_t)bf16_bits(v[0]) | ((uint32_t)bf16_bits(v[1]) << 16);
        const uint32_t hi = (uint32_t)bf16_bits(v[2]) | ((uint32_t)bf16_bits(v[3]) << 16);
        *(uint2 *)dst = make_uint2(lo, hi);
    } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) dst[q] = bf16_bits(v[q]);
    }
}

// V chains of one lane as a single vector: V consecutive chains of one row are
// contiguous in the [n][K] layout, so each gather is one 4-, 8- or 16-byte load.
template <bool CPLX, int V> struct Vec;
template <> struct Vec<false, 1> { using T = float; };
template <> struct Vec<false, 4> { using T = float4; };
template <> struct Vec<true, 1> { using T = float2; };
template <> struct Vec<true, 2> { using T = float4; };

template <bool CPLX, int V>
struct Lane {
    using P = Prec<CPLX>;
    using S = typename P::T;                 // one chain's scalar (float or float2)
    using T = typename Vec<CPLX, V>::T;      // the lane's V chains
    static constexpr int NF = (CPLX ? 2 : 1) * V;  // floats per lane vector
    static __device__ __forceinline__ float *f(T &v) { return reinterpret_cast<float *>(&v); }
    static __device__ __forceinline__ const float *f(const T &v) { return reinterpret_cast<const float *>(&v); }
    static __device__ __forceinline__ T zero()
    {
        T v;
#pragma unroll
        for (int k = 0; k < NF; ++k) f(v)[k] = 0.f;
        return v;
    }
    static __device__ __forceinline__ S get(const T &v, int k)
    {
        if constexpr (CPLX) return make_float2(f(v)[2 * k], f(v)[2 * k + 1]);
        else return f(v)[k];
    }
    static __device__ __forceinline__ void set(T &v, int k, S x)
    {
        if constexpr (CPLX) { f(v)[2 * k] = x.x; f(v)[2 * k + 1] = x.y; }
        else f(v)[k] = x;
    }
    // acc += c * x for each of the V chains
    static __device__ __forceinline__ void fma(T &acc, const typename P::Ent &e, const T &x)
    {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            S s = get(acc, k);
            P::fma(s, e, get(x, k));
            set(acc, k, s);
        }
    }
    // a + b, component by component (joins the partial sums of a split row)
    static __device__ __forceinline__ T add(const T &a, const T &b)
    {
        T v;
#pragma unroll
        for (int k = 0; k < NF; ++k) f(v)[k] = __fadd_rn(f(a)[k], f(b)[k]);
        return v;
    }
    static __device__ __forceinline__ T shfl_down(const T &a, int o)
    {
        T v;
#pragma unroll
        for (int k = 0; k < NF; ++k) f(v)[k] = __shfl_down_sync(0xffffffffu, f(a)[k], o);
        return v;
    }
};

// State reads of the cluster variant go to L2 (ld.global.cg): rows written by
// another CTA of the cluster are seen after the cluster barrier, never a stale
// L1 line.
template <bool CG, typename T>
__device__ __forceinline__ T ld_state(const T *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// ---------------------------------------------------------------------------
// Staging of the chunk stream: one elected thread moves each chunk's blob into
// one of two shared-memory buffers with a bulk async copy that completes on
// the buffer's mbarrier; every wait is bounded (2 s of globaltimer).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void stage_chunk(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool wait_chunk(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = gtimer();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (gtimer() - t0 > 2000000000ull) return false;
    }
}

// ---------------------------------------------------------------------------
// The coupled sweep.  A chain slice = LPR lanes x V chains per lane; Q CTAs
// (one thread-block cluster, Q = 1 without) share a slice and split each
// chunk's rows.  Chains are independent, so slices never communicate.  Per
// cycle the CTA walks the chunk stream; a block barrier ends every chunk (its
// buffer is recycled) and a cluster barrier ends every level.  State is
// double-buffered: a row reads z_j (j < i) from the buffer being written this
// cycle and z_j (j > i) from last cycle's buffer, exactly the in-place
// semantics of Eq. 4 (and of Eq. 5 for w).
//
// Per work item (a row, or one of the 2 or 4 pieces of a long row): the item
// record, constants and entries come from shared memory; the row's first
// piece loads the noise word and the diagonal partial first (they depend only
// on the position); then all 2U gathers of z and w are issued before any FMA
// consumes them.  The gathers are the only round trip to memory on the path.
// Splitting a long row over sibling lane groups keeps the chunk's slowest
// item, which everyone waits for at the chunk barrier, to about one round
// trip: rows are sorted by decreasing length, so without it the first warp
// of every chunk walks the level's longest rows U entries at a time.
// ---------------------------------------------------------------------------
// The rows of one staged chunk for one lane's chains (shared by the
// single-matrix sweep and the pool's persistent sweep, so both compute the
// same arithmetic in the same order).
struct ChunkWork {
    const uint8_t *buf;        // the chunk's blob in shared memory
    ChunkDesc d;
    const void *zo, *wo;       // last cycle's state [n][K]
    void *zn, *wn;             // this cycle's state
    const uint32_t *noise;     // noise words of this cycle and this lane's chain word, by position;
                               // null: no noise (phi = 0), the difference of two coupled paths (Eq. 12)
    void *dpart;               // this lane's unit of diagonal partials (by position), or null
    bool diag, dlead;
    int seg;
    const int *rpos, *spos;    // by position, or null
    uint16_t *zsh, *wsh;
    long long ldsh, kp;
    int shcol;
    size_t K;
    int c0, first, stride, sub;
    bool chain_ok;
    uint32_t cshift;
    const float *tq;           // trace weights q_i by position, or null
};

// Returns whether a chain left the finite bound; adds q_i Re(sum over this
// lane's chains of z_i conj(w_i)) of its rows to *tsum when w.tq is set.
template <bool CPLX, int LPR, int V, int U, bool CLUSTER>
__device__ __forceinline__ bool sweep_chunk_rows(const ChunkWork &w, float *tsum)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    const uint8_t *buf = w.buf;
    const ChunkDesc &d = w.d;
    const T *zo = (const T *)w.zo;
    T *zn = (T *)w.zn;
    const T *wo = (const T *)w.wo;
    T *wn = (T *)w.wn;
    const size_t K = w.K;
    const int c0 = w.c0, first = w.first, stride = w.stride, sub = w.sub, seg = w.seg;
    const bool chain_ok = w.chain_ok, dlead = w.dlead;
    const uint32_t cshift = w.cshift;
    S *dpart = (S *)w.dpart;
    bool diverged = false;

    constexpr int RPW = 32 / LPR;  // lane groups (items) per warp
    const bool split = (d.flags & CHUNK_SPLIT) != 0;
    const RowMeta *meta = (const RowMeta *)buf;
    const Cst *cstv = (const Cst *)(buf + d.cst_off);
    const Ent *zs = (const Ent *)(buf + d.zent_off);
    const Ent *ws = (const Ent *)(buf + d.went_off);
    const uint32_t *__restrict__ noise = w.noise;
    const int shcol = w.shcol;
    // this lane's partial sums over item q's slices of the C and C^dagger entries of row i
    auto piece = [&](int q, int i, T &sz, T &sw) {
        const int zb = meta[q].zoff, zeN = meta[q + 1].zoff;
        const int wb = meta[q].woff, weN = meta[q + 1].woff;
        for (int ez = zb, ew = wb; ez < zeN || ew < weN; ez += U, ew += U) {
            // issue every gather before any FMA consumes one; real entries
            // (8 B) stay in registers, complex ones (16 B) are re-read from
            // shared memory by the FMA pass to keep the register budget
            constexpr bool KEEP = !CPLX;
            Ent enz[KEEP ? U : 1], enw[KEEP ? U : 1];
            T xz[U], xw[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                xz[u] = L::zero();
                xw[u] = L::zero();
                if (ez + u < zeN) {
                    const Ent e = zs[ez + u];
                    if constexpr (KEEP) enz[u] = e;
                    const T *src = e.col < i ? zn : zo;
                    xz[u] = ld_state<CLUSTER>(&src[((size_t)e.col * K + c0) / V]);
                }
                if (ew + u < weN) {
                    const Ent e = ws[ew + u];
                    if constexpr (KEEP) enw[u] = e;
                    const T *src = e.col < i ? wn : wo;
                    xw[u] = ld_state<CLUSTER>(&src[((size_t)e.col * K + c0) / V]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (KEEP) {
                    if (ez + u < zeN) L::fma(sz, enz[u], xz[u]);
                    if (ew + u < weN) L::fma(sw, enw[u], xw[u]);
                } else {
                    if (ez + u < zeN) L::fma(sz, zs[ez + u], xz[u]);
                    if (ew + u < weN) L::fma(sw, ws[ew + u], xw[u]);
                }
            }
        }
    };
    for (int base = first; base < d.items; base += stride) {
        const int it = base + sub;
        const bool live = chain_ok && it < d.items;
        const RowMeta m = it < d.items ? meta[it] : RowMeta{0, 0, 0, 0};
        const int i = m.row;
        const int pk = m.info & 3;              // this item's piece
        const int np = 1 << ((m.info >> 2) & 3);  // pieces of its row
        const int r = m.info >> 4;              // the row within the chunk
        // the pieces of a row run on sibling lane groups of this warp when they fit
        // in it (they start at a multiple of np, so they do); otherwise the first
        // piece's lanes run them one after another.  Either way the partial sums
        // are added in piece order, ((p0 + p1) + p2) + p3.
        const bool par = np <= RPW;
        const bool ok = live && pk == 0;  // the row's update is made by its first piece
        S prod = P::zero();
        S dold = P::zero();
        const int p = d.pb + r;
        uint32_t bits = 0u;
        int rp = -1, sp = -1;
        if (ok) {
            bits = noise ? __ldg(&noise[p]) >> cshift : 0u;
            if (w.diag && dlead) dold = dpart[p];
            if (w.rpos) { rp = __ldg(&w.rpos[p]); sp = __ldg(&w.spos[p]); }
        }
        T sz = L::zero(), sw = L::zero();
        if constexpr (RPW >= 4) {
            if (live) piece(it, i, sz, sw);  // np <= 4 <= RPW: always on sibling lane groups
        } else if (!split) {
            if (live) piece(it, i, sz, sw);  // every item is a whole row
        } else if (live && (par || ok)) {
            const int nq = par ? 1 : np;
#pragma unroll 1
            for (int q = 0; q < nq; ++q) {
                T pz = L::zero(), pw = L::zero();
                piece(it + q, i, pz, pw);
                if (q == 0) { sz = pz; sw = pw; }
                else { sz = L::add(sz, pz); sw = L::add(sw, pw); }
            }
        }
        // the first piece's lanes fold in the others' partial sums; only they add,
        // so every shuffle reads a piece's own partial sum
#pragma unroll
        for (int q = 1; q < 4 && q < RPW && split; ++q) {
            const T oz = L::shfl_down(sz, q * LPR), ow = L::shfl_down(sw, q * LPR);
            if (par && pk == 0 && q < np) { sz = L::add(sz, oz); sw = L::add(sw, ow); }
        }
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
            if (w.tq) {
                float re;
                if constexpr (CPLX) re = prod.x;
                else re = prod;
                *tsum = __fmaf_rn(__ldg(&w.tq[p]), re, *tsum);
            }
            zn[((size_t)i * K + c0) / V] = zv;
            wn[((size_t)i * K + c0) / V] = wv;
            if (rp >= 0 || sp >= 0) {
                // shadow column of (cycle, chain): cycle block of kp elements, then
                // the chain (x2 for re,im); blocks are padded to 64 and the pad
                // stays zero
                const size_t o = (size_t)shcol * w.kp + (size_t)c0 * (CPLX ? 2 : 1);
                constexpr int NF = L::NF;
                if (rp >= 0) store_bf16<NF>(w.zsh + (size_t)rp * w.ldsh + o, L::f(zv));
                if (sp >= 0) {
                    if constexpr (!CPLX) {
                        store_bf16<NF>(w.wsh + (size_t)sp * w.ldsh + o, L::f(wv));
                    } else {
                        // row 2s = [wr, wi] contracts to Re(z conj w), row 2s+1 =
                        // [-wi, wr] to Im(z conj w), so the product comes out
                        // interleaved re,im
                        uint16_t *w0 = w.wsh + (size_t)(2 * sp) * w.ldsh + o;
                        float f0[2 * V], f1[2 * V];
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const S x = L::get(wv, v);
                            f0[2 * v] = x.x;
                            f0[2 * v + 1] = x.y;
                            f1[2 * v] = -x.y;
                            f1[2 * v + 1] = x.x;
                        }
                        store_bf16<2 * V>(w0, f0);
                        store_bf16<2 * V>(w0 + w.ldsh, f1);
                    }
                }
            }
        }
        if (w.diag) {
            // sum over the seg lanes of a unit (all lanes shuffle); the leader
            // adds the running partial it loaded at the start of the row
#pragma unroll
            for (int o = 1; o < LPR; o <<= 1)
                if (o < seg) prod = P::add(prod, P::shfl_xor(prod, o));
            if (ok && dlead) dpart[p] = P::add(dold, prod);
        }
    }
    return diverged;
}

}  // namespace mcinv
