// sweep_wave.cu -- the coupled sweep (Eqs. 4 and 5) of a matrix in the colour
// order whose two colours are banded: a lattice operator, a red site touching
// only the black sites of the neighbouring lattice rows.
//
// Chains are independent, so a CTA can own a slice of them (sv vectors of 16
// bytes: 32 complex or 64 real chains at sv = 16) for whole cycles and never
// wait for another CTA.  It walks the two colours as a wavefront over chunks of
// S consecutive positions.  At step t one half of its warps updates red chunk t
// from black chunks t-B .. t+B (last cycle's values, copied in from HBM once
// each, one step ahead of use) and keeps the new values in a ring of shared
// memory, while the other half updates black chunk t-B-1 from red chunks
// t-2B-1 .. t-1, all new by then; one CTA barrier ends the step.  The black
// chunks whose bands wrap around the level's end, and the last regular one, are
// updated after the last red chunk, with the first 2B red chunks read back from
// the new buffer.  So a cycle reads each black value once, writes each value
// once, and reads nothing of the red half but 2B chunks: about 3/4 of the bytes
// of reading and writing the whole state.  Two state buffers alternate between
// cycles (the new values never overwrite what this cycle still reads).
//
// A lane updates two vectors of a row (j and j + sv/2), so the row's record is
// loaded once for both and the lane has two independent chains of FMAs.  The
// sums take the entries in their order, the epilogue is the ring path's
// `finish`, and the diagonal partial of a unit is reduced over the same binary
// tree as the other kernels' butterfly, so the values are the same bits as every
// other sweep kernel's.  Every wait is bounded (2 s of globaltimer).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "sweep_core.cuh"
#include "sweep_ring.cuh"
#include "sweep_wave.h"

namespace mcinv {

namespace {

constexpr int WAVE_THREADS = 512;  // two groups of 8 warps (red, black), one CTA an SM
constexpr int WNW = WAVE_THREADS / 32;
constexpr size_t WAVE_SMEM_MAX = 227u * 1024u;

size_t row_bytes(int cplx, int D)
{
    return cplx ? (D == 4 ? sizeof(WaveRow<true, 4>) : sizeof(WaveRow<true, 8>))
                : (D == 4 ? sizeof(WaveRow<false, 4>) : sizeof(WaveRow<false, 8>));
}

// shared memory of one CTA: the black ring and the red ring (2B + 2 chunks each), two
// stage buffers of two record chunks each (records, constants and noise words of S
// positions), two mbarriers
size_t smem_for(int S, int B, int sv, int cplx, int D)
{
    const int V = cplx ? 2 : 4;
    const size_t chb = (size_t)S * 2 * sv * 16;
    const size_t cb = cplx ? sizeof(CstC) : sizeof(CstR);
    const size_t nws = std::max(1, sv * V / 32);
    const size_t rcb = (size_t)S * (row_bytes(cplx, D) + cb) + nws * S * 4;
    return (size_t)(4 * B + 4) * chb + 4 * rcb + 16;
}

template <bool CPLX, int D>
void put_row(uint8_t *dst, int d, const uint16_t *code, const std::vector<uint8_t> &zent,
             const std::vector<uint8_t> &went, size_t eb, int zb, int wb)
{
    WaveRow<CPLX, D> t{};
    t.d = d;
    for (int u = 0; u < d; ++u) {
        t.code[u] = code[u];
        if constexpr (CPLX) {
            const EntC ez = *(const EntC *)(zent.data() + (size_t)(zb + u) * eb);
            const EntC ew = *(const EntC *)(went.data() + (size_t)(wb + u) * eb);
            t.zc[u] = make_float2(ez.re, ez.im);
            t.wc[u] = make_float2(ew.re, ew.im);
        } else {
            const EntR ez = *(const EntR *)(zent.data() + (size_t)(zb + u) * eb);
            const EntR ew = *(const EntR *)(went.data() + (size_t)(wb + u) * eb);
            t.zc[u] = ez.val;
            t.wc[u] = ew.val;
        }
    }
    std::memcpy(dst, &t, sizeof(t));
}

}  // namespace

bool build_wave(const std::vector<GridRow> &rows, const std::vector<uint8_t> &zent, const std::vector<uint8_t> &went,
                size_t ent_bytes, const std::vector<int32_t> &lev_ptr, int cplx, int kv, int sms, WaveForm &out)
{
    const int n = (int)rows.size() - 1;
    if (lev_ptr.size() != 3 || n < 16 || kv < 1) return false;
    const int h = lev_ptr[1];
    if (lev_ptr[0] != 0 || lev_ptr[2] != n || 2 * h != n) return false;
    auto col = [&](const std::vector<uint8_t> &v, int e) { return *(const int *)(v.data() + (size_t)e * ent_bytes); };
    int dmax = 0;
    for (int p = 0; p < n; ++p) {
        if (rows[p].row != p || (rows[p].info & 3)) return false;  // position = row; no row cut into pieces
        const int d = rows[p + 1].zb - rows[p].zb;
        if (d > SPLIT_ENTRIES || rows[p + 1].wb - rows[p].wb != d) return false;
        dmax = std::max(dmax, d);
        for (int u = 0; u < d; ++u) {
            const int j = col(zent, rows[p].zb + u);
            if (j < 0 || j >= n || (j < h) == (p < h) || col(went, rows[p].wb + u) != j) return false;
        }
    }
    // records of 4 entries when every row has 4, else of 8 (exact when every row has 8)
    bool same = true;
    for (int p = 1; p < n && same; ++p) same = rows[p + 1].zb - rows[p].zb == rows[1].zb - rows[0].zb;
    const int D = same && dmax == 4 ? 4 : 8;
    const bool exact = same && dmax == D;
    // the ring distance between row p's chunk and neighbour j's chunk (each level's
    // chunks counted from its first position)
    auto dist = [&](int p, int j, int S) {
        const int m = h / S;
        int dd = ((j < h ? j : j - h) / S - (p < h ? p : p - h) / S) % m;
        if (dd < 0) dd += m;
        if (dd > m / 2) dd -= m;
        return dd;
    };
    auto band = [&](int S) {
        int B = 1;
        for (int p = 0; p < n; ++p)
            for (int e = rows[p].zb; e < rows[p + 1].zb; ++e) B = std::max(B, std::abs(dist(p, col(zent, e), S)));
        return B;
    };
    int S = 0, B = 0, sv = 0;
    for (int c : {16, 8, 4}) {
        // the widest slice that still gives most SMs a CTA (the narrowest as a last resort)
        if (c != 4 && (kv + c - 1) / c < sms * 5 / 8) continue;
        for (int s : {32, 64, 16, 128}) {
            // whole chunks, each a whole number of a warp's rows (64 / sv: sv / 2 lanes a row)
            if (h % s || s % (64 / c)) continue;
            const int b = band(s);
            if (h / s < 4 * b + 2 || b > 15) continue;
            if (smem_for(s, b, c, cplx, D) > WAVE_SMEM_MAX) continue;
            S = s;
            B = b;
            break;
        }
        if (S) {
            sv = c;
            break;
        }
    }
    if (!S) return false;
    out.S = S;
    out.B = B;
    out.m = h / S;
    out.h = h;
    out.sv = sv;
    out.D = D;
    out.exact = exact;
    const size_t rb = row_bytes(cplx, D);
    out.trow.assign((size_t)n * rb, 0);
    for (int p = 0; p < n; ++p) {
        const int d = rows[p + 1].zb - rows[p].zb;
        uint16_t code[SPLIT_ENTRIES] = {};
        for (int u = 0; u < d; ++u) {
            const int j = col(zent, rows[p].zb + u);
            code[u] = (uint16_t)(((dist(p, j, S) + B) << 10) | ((j < h ? j : j - h) % S));
        }
        uint8_t *r = out.trow.data() + (size_t)p * rb;
        if (cplx) {
            if (D == 4) put_row<true, 4>(r, d, code, zent, went, ent_bytes, rows[p].zb, rows[p].wb);
            else put_row<true, 8>(r, d, code, zent, went, ent_bytes, rows[p].zb, rows[p].wb);
        } else {
            if (D == 4) put_row<false, 4>(r, d, code, zent, went, ent_bytes, rows[p].zb, rows[p].wb);
            else put_row<false, 8>(r, d, code, zent, went, ent_bytes, rows[p].zb, rows[p].wb);
        }
    }
    return true;
}

namespace {

using namespace ring;

static_assert(SPLIT_ENTRIES == 8, "a row record holds the entries of an unsplit row");

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts_vec(uint32_t addr, const float4 &v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// EXACT: every row has D entries (no per-entry guard); SV: the slice width (g.sv)
template <bool CPLX, int V, int D, bool EXACT, int SV>
__global__ void __launch_bounds__(WAVE_THREADS, 1) cc_sweep_wave_kernel(const SweepArgs a, const WaveArgs g)
{
    using P = Prec<CPLX>;
    using L = Lane<CPLX, V>;
    using T = typename L::T;
    using S = typename L::S;
    using Ent = typename P::Ent;
    using Cst = typename P::Cst;
    using Row = WaveRow<CPLX, D>;
    static_assert(sizeof(T) == 16, "a lane holds 16-byte vectors");
    extern __shared__ __align__(128) uint8_t wsm[];
    __shared__ int abort_s;
    volatile int *abort_flag = &abort_s;
    constexpr uint32_t RB = sizeof(Row), CB = sizeof(Cst);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = warp >> 3, wg = warp & 7;  // group 0 updates red chunks, group 1 black ones
    const int SC = g.S, B = g.B, MC = g.m, NB = g.nb, NR = g.nr;
    constexpr int hl = SV / 2;                 // lanes a row: lane j holds vectors j and j + hl
    constexpr int rpw = 32 / hl;               // rows a warp updates side by side
    const int rsub = lane / hl, j = lane % hl;
    constexpr uint32_t rowb = (uint32_t)SV * 32u;  // one position of a slice: SV z vectors, then SV w vectors
    const uint32_t chb = (uint32_t)SC * rowb;
    const bool diag = a.diag_part != nullptr, noisy = a.noise != nullptr;
    const int sl = blockIdx.x;  // the chain slice
    // the slice's noise words and diagonal-partial units (those that exist)
    const int nws = max(1, (SV * V) >> 5);
    const int w0 = (sl * SV * V) >> 5;
    const int nws_here = min(nws, a.nw - w0);
    const uint32_t off_noise = (uint32_t)SC * (RB + CB);
    const uint32_t rcb = off_noise + (uint32_t)(nws * SC) * 4u;  // one record chunk
    const uint32_t black0 = smem_addr(wsm);
    const uint32_t red0 = black0 + (uint32_t)NB * chb;
    const uint32_t stage0 = red0 + (uint32_t)NR * chb;
    const uint32_t bar0 = stage0 + 4u * rcb;

    Lanes<CPLX, V, 2> w;
    w.lane = lane;
    w.seg = a.seg;
    w.diag = diag;
    int wsel[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int vs = j + q * hl;  // the vector within the slice
        const int vg = sl * SV + vs;
        w.cv[q] = (uint32_t)vg;
        w.c0[q] = vg * V;
        w.ok[q] = w.c0[q] < a.K;
        w.dpart[q] = (S *)a.diag_part + (size_t)(diag ? w.c0[q] / (a.seg * V) : 0) * (size_t)a.n;
        w.dlead[q] = diag && w.ok[q] && (vs % a.seg) == 0;
        w.noise_col[q] = nullptr;
        w.cshift[q] = (uint32_t)(w.c0[q] & 31);
        w.zo[q] = (uint32_t)vs;
        w.wo[q] = (uint32_t)(SV + vs);
        wsel[q] = (w.c0[q] >> 5) - w0;     // the noise word among the slice's
    }
    const bool whole = diag && a.seg == SV;  // one unit a row: the two halves add at the last level
    // with units of two or more vectors, vector j + hl's unit sum ends in lane j + 1 (odd),
    // which stores it when the unit's first vector (j + hl - 1) has chains
    const bool lead1 = diag && a.seg >= 2 && (j % a.seg) == 1 && w.c0[1] - V < a.K;
    if (threadIdx.x == 0) {
        abort_s = 0;
        mbar_init1(bar0);
        mbar_init1(bar0 + 8u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    Mat<CPLX> m;
    m.rows = nullptr;
    m.zent = m.went = nullptr;
    m.cst = (const Cst *)g.cst;
    m.z0 = a.z[0];
    m.w0 = a.z[0];  // w beside z in every row of a slice
    m.has_noise = noisy;
    m.rpos = a.rpos;
    m.spos = a.spos;
    m.zsh = a.zsh;
    m.wsh = a.wsh;
    m.ldsh = a.ldsh;
    m.kp = a.kp;
    m.tq = a.tq;
    const float4 *x0 = (const float4 *)a.z[0];
    const uint32_t sliceo = (uint32_t)sl * (uint32_t)a.n * 2u * (uint32_t)SV;  // the slice's first vector
    bool diverged = false;
    bool quit = false;
    uint32_t gst = 0;             // stages waited for so far: stage buffer gst & 1, its phase (gst >> 1) & 1
    const int nfin = 2 * B + 1;   // black chunks updated after the last red one
    const int nst = MC + B + 1;   // m steps, then B + 1 steps of two of those (the last has one)
    // black chunk k of those: the last regular one (m - 1 - B), the B at the end, the B at the start
    auto fin = [&](int k) { return k <= B ? MC - 1 - B + k : k - B - 1; };
    int bslot_next = 0;  // (t + B + 1) mod NB at step t

    for (int cyc = 0; cyc < a.ncyc && !quit; ++cyc) {
        const int cur = a.cur ^ (cyc & 1);           // the buffer holding last cycle's state
        m.zn_off = cur ? 0u : g.nkv;                 // this cycle's
        const uint32_t old_off = cur ? g.nkv : 0u;
        m.noise_cyc = (size_t)cyc * a.nw * (size_t)a.n;
        m.shcol = a.cyc0_in_batch + cyc;
        m.check_div = cyc == a.ncyc - 1;
        // the epilogue's view: with the diagonal on, the caller adds the trace terms (the
        // epilogue forms z conj(w) for the diagonal anyway); without it, the epilogue does
        Mat<CPLX> mt = m;
        if (diag) mt.tq = nullptr;
        float tsum = 0.f;

        // Stage t (< m): black chunk t + B (chunks -B .. B at t = 0) from last cycle's
        // buffer into the black ring, and the records of red chunk t and black chunk
        // t - B - 1.  Stage m: red chunks 0 .. 2B-1 from this cycle's buffer into the
        // black ring, and the records of the first two late black chunks; later stages:
        // two more.  Warp 0 issues the copies, one a lane, all completing on the buffer's
        // mbarrier (no division on this path: the other warps wait for it at the step's end).
        auto issue = [&](int t, uint32_t b) {
            if (warp != 0) return;
            // this CTA's stores to the state and the partials (last cycle's, or this cycle's
            // red rows) before the async-proxy reads of them: stages 0 and m; the slots'
            // earlier generic-proxy reads before their async-proxy writes: every stage
            if (t == 0 || t == MC) asm volatile("fence.proxy.async.global;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            int cfirst, ccnt, nrec = 1;
            bool cred;
            int pr0, pr1 = 0;
            if (t < MC) {
                cred = false;
                cfirst = t == 0 ? -B : t + B;
                ccnt = t == 0 ? 2 * B + 1 : 1;
                pr0 = t * SC;
                if (t >= 2 * B + 1) {
                    pr1 = g.h + (t - B - 1) * SC;
                    nrec = 2;
                }
            } else {
                const int f = t - MC;
                cred = true;
                cfirst = 0;
                ccnt = f == 0 ? 2 * B : 0;
                pr0 = g.h + fin(2 * f) * SC;
                if (2 * f + 1 < nfin) {
                    pr1 = g.h + fin(2 * f + 1) * SC;
                    nrec = 2;
                }
            }
            const int nnw = noisy ? nws_here : 0;
            const int per = 2 + nnw;
            const uint32_t recb = (uint32_t)SC * (RB + CB) + (uint32_t)(nnw * SC) * 4u;
            const uint32_t bar = bar0 + 8u * b;
            if (lane == 0) mbar_expect(bar, (uint32_t)ccnt * chb + (uint32_t)nrec * recb);
            __syncwarp();
            if (t == 0 && a.test_expire) return;  // announced, never copied: the waits for it expire
            const int ncp = ccnt + nrec * per;
            for (int k = lane; k < ncp; k += 32) {
                if (k < ccnt) {
                    // black chunk v (-B <= v < m + B) of last cycle into ring slot v mod NB (NB > B),
                    // or red chunk k of this cycle into slot k
                    const int v = cfirst + k;
                    if (!cred) {
                        const int c = v < 0 ? v + MC : v >= MC ? v - MC : v;
                        int slot = v < 0 ? v + NB : v;
                        while (slot >= NB) slot -= NB;  // (t = 0: at most once; later: v mod NB kept by the caller)
                        if (t > 0) slot = bslot_next;
                        bulk_g2s(black0 + (uint32_t)slot * chb,
                                 x0 + old_off + sliceo + (uint32_t)(g.h + c * SC) * 2u * (uint32_t)SV, chb, bar);
                    } else {
                        bulk_g2s(black0 + (uint32_t)v * chb, x0 + m.zn_off + sliceo + (uint32_t)(v * SC) * 2u * (uint32_t)SV,
                                 chb, bar);
                    }
                } else {
                    const int q = k - ccnt, rc = q >= per ? 1 : 0, jj = q - rc * per;
                    const int p0 = rc ? pr1 : pr0;
                    const uint32_t dst = stage0 + (b * 2u + (uint32_t)rc) * rcb;
                    if (jj == 0) {
                        bulk_g2s(dst, (const uint8_t *)g.trow + (size_t)p0 * RB, (uint32_t)SC * RB, bar);
                    } else if (jj == 1) {
                        bulk_g2s(dst + (uint32_t)SC * RB, (const uint8_t *)g.cst + (size_t)p0 * CB, (uint32_t)SC * CB, bar);
                    } else {
                        const int wq = jj - 2;
                        bulk_g2s(dst + off_noise + (uint32_t)(wq * SC) * 4u,
                                 a.noise + m.noise_cyc + (size_t)(w0 + wq) * (size_t)a.n + (size_t)p0, (uint32_t)SC * 4u, bar);
                    }
                }
            }
        };

        // Update the S rows from p0 whose records are at rc (this group's 8 warps); the
        // lanes 0 .. 2B of tb hold the shared-memory chunk each ring distance -B .. B
        // reads; wslot: where the new values are kept for the other colour (0: not kept).
        auto phase = [&](uint32_t rc, int p0, uint32_t tb, uint32_t wslot) {
            for (int r = wg * rpw + rsub; r < SC; r += 8 * rpw) {
                const int p = p0 + r;
                Row rec;
#pragma unroll
                for (int q = 0; q < (int)(RB / 16); ++q)
                    ((float4 *)&rec)[q] = lds_vec<float4>(rc + (uint32_t)r * RB + 16u * q);
                // the sums in entry order
                T sz0 = L::zero(), sw0 = L::zero(), sz1 = L::zero(), sw1 = L::zero();
                const int dmax = EXACT ? D : __reduce_max_sync(0xffffffffu, rec.d);
                // the running diagonal partials this lane adds to and the row's trace weight,
                // loaded now for the epilogue
                S d0 = P::zero(), d1 = P::zero();
                if (diag) {
                    if (w.dlead[0]) d0 = w.dpart[0][p];
                    if (!whole && (a.seg == 1 ? w.dlead[1] : lead1)) d1 = w.dpart[1][p];
                }
                const float qp = diag && a.tq ? __ldg(&a.tq[p]) : 0.f;
#pragma unroll
                for (int u = 0; u < D; ++u) {
                    if (EXACT || u < dmax) {
                        const uint32_t code = rec.code[u];
                        const uint32_t base = __shfl_sync(0xffffffffu, tb, (int)(code >> 10));
                        if (EXACT || u < rec.d) {
                            Ent ez, ew;
                            ez.col = ew.col = 0;
                            if constexpr (CPLX) {
                                ez.re = rec.zc[u].x; ez.im = rec.zc[u].y; ez.pad = 0;
                                ew.re = rec.wc[u].x; ew.im = rec.wc[u].y; ew.pad = 0;
                            } else {
                                ez.val = rec.zc[u];
                                ew.val = rec.wc[u];
                            }
                            const uint32_t ad = base + (code & 1023u) * rowb + (uint32_t)j * 16u;
                            const T xz0 = lds_vec<T>(ad), xz1 = lds_vec<T>(ad + (uint32_t)hl * 16u);
                            const T xw0 = lds_vec<T>(ad + (uint32_t)SV * 16u);
                            const T xw1 = lds_vec<T>(ad + (uint32_t)(SV + hl) * 16u);
                            L::fma(sz0, ez, xz0);
                            L::fma(sz1, ez, xz1);
                            L::fma(sw0, ew, xw0);
                            L::fma(sw1, ew, xw1);
                        }
                    }
                }
                // the epilogue's operands: constants, noise words, diagonal partials, shadows
                Cst k;
#pragma unroll
                for (int q = 0; q < (int)(CB / 16); ++q)
                    ((float4 *)&k)[q] = lds_vec<float4>(rc + (uint32_t)SC * RB + (uint32_t)r * CB + 16u * q);
                uint32_t bits0 = 0u, bits1 = 0u;
                if (noisy) {
                    const uint32_t wd0 = lds_u32(rc + off_noise + (uint32_t)(wsel[0] * SC + r) * 4u);
                    const uint32_t wd1 =
                        wsel[1] == wsel[0] ? wd0 : lds_u32(rc + off_noise + (uint32_t)(wsel[1] * SC + r) * 4u);
                    bits0 = wd0 >> w.cshift[0];
                    bits1 = wd1 >> w.cshift[1];
                }
                int rp = -1, sp = -1;
                if (m.rpos) {
                    rp = __ldg(&m.rpos[p]);
                    sp = __ldg(&m.spos[p]);
                }
                T zv0 = L::zero(), wv0 = L::zero(), zv1 = L::zero(), wv1 = L::zero();
                const uint32_t iv = sliceo + (uint32_t)p * 2u * (uint32_t)SV;
                const S zero = P::zero();
                // (the trace terms in the epilogue's order, vector 0 then 1)
                S pr0 = finish_keep<CPLX, V, 2>(w, mt, 0, p, iv, sz0, sw0, k, bits0, zero, rp, sp, tsum, diverged, zv0, wv0);
                S pr1 = finish_keep<CPLX, V, 2>(w, mt, 1, p, iv, sz1, sw1, k, bits1, zero, rp, sp, tsum, diverged, zv1, wv1);
                if (diag && a.tq) {
                    if constexpr (CPLX) {
                        if (w.ok[0]) tsum = __fmaf_rn(qp, pr0.x, tsum);
                        if (w.ok[1]) tsum = __fmaf_rn(qp, pr1.x, tsum);
                    } else {
                        if (w.ok[0]) tsum = __fmaf_rn(qp, pr0, tsum);
                        if (w.ok[1]) tsum = __fmaf_rn(qp, pr1, tsum);
                    }
                }
                if (wslot) {
                    const uint32_t o = wslot + (uint32_t)r * rowb + (uint32_t)j * 16u;
                    sts_vec(o, *(const float4 *)&zv0);
                    sts_vec(o + (uint32_t)hl * 16u, *(const float4 *)&zv1);
                    sts_vec(o + (uint32_t)SV * 16u, *(const float4 *)&wv0);
                    sts_vec(o + (uint32_t)(SV + hl) * 16u, *(const float4 *)&wv1);
                }
                if (diag) {
                    if (a.seg == 1) {
                        if (w.dlead[0]) w.dpart[0][p] = P::add(d0, pr0);
                        if (w.dlead[1]) w.dpart[1][p] = P::add(d1, pr1);
                    } else {
                        // the butterfly of the other kernels over a unit's vectors: at its first
                        // level even lanes keep vector j's pair sum and odd lanes vector j + hl's
                        // (each sends the other), then its levels below hl run once for both
                        // halves; a unit of SV vectors adds the halves at its last level
                        const bool odd = (lane & 1) != 0;
                        S keep = odd ? pr1 : pr0;
                        keep = P::add(keep, P::shfl_xor(odd ? pr0 : pr1, 1));
#pragma unroll
                        for (int o = 2; o < hl; o <<= 1)
                            if (o < a.seg) keep = P::add(keep, P::shfl_xor(keep, o));
                        if (whole) {
                            const S other = P::shfl_xor(keep, 1);
                            if (w.dlead[0]) w.dpart[0][p] = P::add(d0, P::add(keep, other));
                        } else {
                            // lane j (j mod seg = 0): vector j's unit; lane j + 1: vector j + hl's
                            if (w.dlead[0]) w.dpart[0][p] = P::add(d0, keep);
                            if (lead1) w.dpart[1][p] = P::add(d1, keep);
                        }
                    }
                }
            }
        };

        // ring slots kept step by step: black chunk t + B + 1 (the next stage's copy), black
        // chunk t - B (the red rows' first), red chunk t (written) and red chunk t - 2B - 1
        // (the black rows' first)
        bslot_next = B + 1;  // (NB = 2B + 2)
        int kb = NB - B, kw = 0, kr = NR - 2 * B - 1;
        issue(0, gst & 1u);
        for (int t = 0; t < nst; ++t) {
            const uint32_t b = gst & 1u;
            // the other buffer, and the black slot of chunk t + 1 + B, were released at the
            // last CTA barrier (stage m waits for the whole black ring: issued below)
            if (t + 1 < nst && t + 1 != MC) issue(t + 1, b ^ 1u);
            if (++bslot_next == NB) bslot_next = 0;
            // a stage that did not land (an expired wait) leaves its rows alone: its records,
            // and so their ring offsets, may never have been written
            const bool landed = __all_sync(0xffffffffu, ring_wait(bar0 + 8u * b, (gst >> 1) & 1u));
            if (!landed) *abort_flag = 1;
            ++gst;
            const uint32_t rc0 = stage0 + b * 2u * rcb, rc1 = rc0 + rcb;
            if (!landed) {
            } else if (t < MC) {
                if (grp == 0) {
                    // red chunk t from black chunks t-B .. t+B (last cycle's values)
                    uint32_t tb = 0u;
                    if (lane <= 2 * B) tb = black0 + (uint32_t)(kb + lane < NB ? kb + lane : kb + lane - NB) * chb;
                    phase(rc0, t * SC, tb, red0 + (uint32_t)kw * chb);
                } else if (t >= 2 * B + 1) {
                    // black chunk t-B-1 from red chunks t-2B-1 .. t-1 (new)
                    const int bc = t - B - 1;
                    uint32_t tb = 0u;
                    if (lane <= 2 * B) tb = red0 + (uint32_t)(kr + lane < NR ? kr + lane : kr + lane - NR) * chb;
                    phase(rc1, g.h + bc * SC, tb, 0u);
                }
            } else {
                // the late black chunks: red chunks 0 .. 2B-1 are in the black ring, the last
                // 2B + 2 in the red ring
                const int k = 2 * (t - MC) + grp;
                if (k < nfin) {
                    const int bc = fin(k);
                    uint32_t tb = 0u;
                    if (lane <= 2 * B) {
                        const int r = (bc + lane - B + MC) % MC;
                        tb = r < 2 * B ? black0 + (uint32_t)r * chb : red0 + (uint32_t)(r % NR) * chb;
                    }
                    phase(grp ? rc1 : rc0, g.h + bc * SC, tb, 0u);
                }
            }
            if (++kb == NB) kb = 0;
            if (++kw == NR) kw = 0;
            if (++kr == NR) kr = 0;
            // an expired wait ends the launch for the whole CTA at once
            if (__syncthreads_or(*abort_flag)) {
                quit = true;
                break;
            }
            if (t == MC - 1) issue(MC, gst & 1u);
        }
        if (quit) break;
        if (a.tpart) {
            // this warp's partial of the cycle's trace series, reduced in a fixed order
            float v = tsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) a.tpart[((size_t)cyc * gridDim.x + blockIdx.x) * WNW + warp] = v;
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

template <bool CPLX, int V, int D, bool EXACT, int SV>
cudaError_t launch_sv(const SweepArgs &a, const WaveArgs &g, int ctas, size_t smem, cudaStream_t s)
{
    auto kern = cc_sweep_wave_kernel<CPLX, V, D, EXACT, SV>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)ctas, WAVE_THREADS, smem, s>>>(a, g);
    return cudaGetLastError();
}

template <bool CPLX, int V, int D, bool EXACT>
cudaError_t launch_one(const SweepArgs &a, const WaveArgs &g, int ctas, size_t smem, cudaStream_t s)
{
    if (g.sv == 16) return launch_sv<CPLX, V, D, EXACT, 16>(a, g, ctas, smem, s);
    if (g.sv == 8) return launch_sv<CPLX, V, D, EXACT, 8>(a, g, ctas, smem, s);
    return launch_sv<CPLX, V, D, EXACT, 4>(a, g, ctas, smem, s);
}

}  // namespace

int wave_ctas(int kv, int sv) { return sv > 0 ? (kv + sv - 1) / sv : 0; }

size_t wave_smem(const WaveArgs &g, int cplx, int seg)
{
    (void)seg;
    return smem_for(g.S, g.B, g.sv, cplx, g.D);
}

cudaError_t launch_sweep_wave(const SweepArgs &a, const WaveArgs &g, int cplx, cudaStream_t s)
{
    const int V = cplx ? 2 : 4;
    if (a.K % V || g.sv < 4 || g.sv > 16 || (g.sv & (g.sv - 1)) || g.B < 1 || g.B > 15 || g.m < 4 * g.B + 2 ||
        g.S % (64 / g.sv) || g.S > 1024 || (g.D != 4 && g.D != 8) || (g.D == 4 && !g.exact) || g.nb != 2 * g.B + 2 ||
        g.nr != 2 * g.B + 2 ||
        (long long)g.m * g.S != g.h || 2LL * g.h != a.n)
        return cudaErrorInvalidValue;
    if (a.diag_part && (a.seg < 1 || a.seg > g.sv || g.sv % a.seg)) return cudaErrorInvalidValue;
    const int kv = a.K / V;
    const int ctas = wave_ctas(kv, g.sv);
    if (2ull * g.nkv >= (1ull << 32) || (unsigned long long)ctas * g.sv * 2ull * a.n > g.nkv) return cudaErrorInvalidValue;
    const size_t smem = wave_smem(g, cplx, a.diag_part ? a.seg : 0);
    if (smem > WAVE_SMEM_MAX) return cudaErrorInvalidValue;
    // records of 4 entries: every row has 4; of 8: every row has 8 (exact) or at most 8
    if (cplx) {
        if (g.D == 4) return launch_one<true, 2, 4, true>(a, g, ctas, smem, s);
        return g.exact ? launch_one<true, 2, 8, true>(a, g, ctas, smem, s) : launch_one<true, 2, 8, false>(a, g, ctas, smem, s);
    }
    if (g.D == 4) return launch_one<false, 4, 4, true>(a, g, ctas, smem, s);
    return g.exact ? launch_one<false, 4, 8, true>(a, g, ctas, smem, s) : launch_one<false, 4, 8, false>(a, g, ctas, smem, s);
}

}  // namespace mcinv
