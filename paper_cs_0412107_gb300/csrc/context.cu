// context.cu -- the C ABI of include/mcinv.h: host-side set-up (CSR
// validation, C^dagger, Gauss-Seidel dependency levels), device memory, and
// the orchestration of the sweep / accumulation / estimate kernels.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/mcinv.h"
#include "internal.h"
#include "partition.h"
#include "prepare.h"
#include "sweep_tiled.h"
#include "sweep_wave.h"
#include "tc_gemm.h"

using namespace mcinv;

struct mcinv_ctx {
    // problem and options
    int64_t n = 0, nnz = 0, K = 0;
    int cplx = 0;
    int W = 0, V = 1, LPR = 1, Q = 1, threads = 0, slices = 0, G = 0, B = 0, acc = 0, flags = 0;
    bool staged = false;  // the staged sweep kernel (sweep_staged.cu) instead of the register one
    bool grid = false;    // the grid-wide sweep kernel (sweep_grid.cu)
    bool gbulk = false;   // its variant that stages the gathers with bulk copies
    bool gpair = false;   // ... on the pair layout of the state (z and w of a chain block side by side)
    bool pair_able = false;  // structurally symmetric, the pair form built
    bool canon_ok = true, pair_ok = false;  // which layout holds the current state
    int gctas = 0;        // its CTAs (all resident at once)
    uint64_t seed = 0;
    int64_t chain_base = 0;
    uint32_t matrix_id = 0;
    cudaStream_t stream = nullptr;
    int nlev = 0, nw = 0;
    // device arrays
    int *d_perm = nullptr, *d_pos = nullptr;
    uint8_t *d_stream = nullptr;
    ChunkDesc *d_chunks = nullptr;
    // the flat form of the matrix for the grid-wide sweep
    GridRow *d_grow = nullptr;
    uint8_t *d_gzent[2] = {nullptr, nullptr}, *d_gwent[2] = {nullptr, nullptr}, *d_gcst = nullptr;
    uint32_t gnkv = 0;
    // the pair form: records (.row = i x 2 kvp), entries with pair-layout offsets, the
    // two pair-layout state buffers (n x 2 kvp vectors each, one allocation)
    GridRow *d_grow_p = nullptr;
    uint8_t *d_gpzent[2] = {nullptr, nullptr}, *d_gpwent[2] = {nullptr, nullptr};
    void *d_x = nullptr;
    uint32_t gpnkv = 0;
    // the tiled form (sweep_tiled.cu): tiles of positions and their staged neighbours
    bool tile_able = false, gtile = false;
    uint8_t *d_trow = nullptr;  // TileRow records by position
    int *d_tptr = nullptr, *d_tslots = nullptr, *d_levtile = nullptr, *d_rptr = nullptr, *d_rrow = nullptr,
        *d_rlen = nullptr;
    int tile_size = 0;
    // the wavefront form (sweep_wave.cu): chunk size, band, chunks a level, positions a
    // level, slice width; records by position
    bool wave_able = false, gwave = false;
    uint8_t *d_wrow = nullptr;
    int wave_S = 0, wave_B = 0, wave_m = 0, wave_h = 0, wave_sv = 0, wave_D = 0, wave_exact = 0;
    int x_layout = 0;  // the layout of d_x when pair_ok: 0 the pair layout, 1 block-major (tiled
                       // sweep), 2 sliced (block-major with blocks of wave_sv vectors: wavefront sweep)
    int *d_levptr = nullptr;
    unsigned *d_gbar = nullptr;
    int nchunks = 0, blob_max = 0, seg = 1, units = 0;
    uint32_t *d_noise = nullptr;
    void *d_z[2] = {nullptr, nullptr}, *d_w[2] = {nullptr, nullptr};
    int cur = 0;
    void *d_diag_part = nullptr;
    double *d_diag_acc = nullptr, *d_counts = nullptr;
    std::vector<double> counts;
    // block estimate
    int64_t nR = 0, nS = 0;
    int *d_R = nullptr, *d_S = nullptr, *d_rpos = nullptr, *d_spos = nullptr;
    float *d_blk = nullptr;
    double *d_bsum = nullptr, *d_bsq = nullptr;
    uint16_t *d_zsh = nullptr, *d_wsh = nullptr;
    long long ldsh = 0, kp = 0;
    TcGemmPlan *gemm = nullptr;
    // estimate scratch
    double *d_mean = nullptr, *d_se = nullptr, *d_q = nullptr;
    // per-cycle trace series (Geyer's Monte Carlo error, Sec. 2.3)
    float *d_tq = nullptr, *d_tpart = nullptr;
    double *d_series = nullptr;
    int64_t nseries = 0, cap_series = 0;
    int *d_status = nullptr;
    // MCINV_F_COLOR_ORDER: the handle samples C' = P C P^T; ord[k] is the row of C
    // that is row k of C' (empty: the rows of C in their given order)
    std::vector<int32_t> ord, inv;
    // mcinv_create_partitioned with blocks of two or more rows: the handle samples
    // C~ = S^-1 C S^-1; per such block the products z~_r conj(w~_s) of its rows are
    // summed per chain group (entries pent_off[m] .. of block pblk[m], row-major)
    Partition part;
    std::vector<int64_t> pblk, pent_off;
    int nent = 0;
    int *d_pent_r = nullptr, *d_pent_s = nullptr, *d_gch = nullptr;
    double *d_pacc = nullptr, *d_acc_est = nullptr;
    // counters
    int64_t cycle = 0, samples = 0, block_batches = 0, block_cycles = 0, launches = 0;
    int64_t bytes = 0;
    // per-kernel timing (mcinv_profile)
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    int64_t prof_launches[MCINV_KERNEL_CLASSES] = {};
    double prof_ms[MCINV_KERNEL_CLASSES] = {};
    std::vector<void *> allocs;
    std::string err;
};

static thread_local std::string g_create_error;

static mcinv_status fail(mcinv_ctx *h, mcinv_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return st;
}

#define CUDA_TRY(h, call)                                                                    \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((h), e_ == cudaErrorMemoryAllocation ? MCINV_E_NOMEM : MCINV_E_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

static cudaError_t prof_begin(mcinv_ctx *h, int kind, cudaEvent_t *stop)
{
    *stop = nullptr;
    if (!h->profiling) return cudaSuccess;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t a, b;
        cudaError_t e = cudaEventCreate(&a);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
        h->ev_pool.emplace_back(a, b);
        h->ev_kind.push_back(0);
    }
    h->ev_kind[h->ev_used] = kind;
    *stop = h->ev_pool[h->ev_used].second;
    return cudaEventRecord(h->ev_pool[h->ev_used++].first, h->stream);
}

// Launch one kernel through `call`, counting it and (when profiling) timing it.
#define LAUNCH_K(h, kind, call)                                     \
    do {                                                            \
        cudaEvent_t stop_;                                          \
        CUDA_TRY(h, prof_begin((h), (kind), &stop_));               \
        CUDA_TRY(h, call);                                          \
        (h)->launches++;                                            \
        if (stop_) CUDA_TRY(h, cudaEventRecord(stop_, (h)->stream)); \
    } while (0)

template <typename T>
static cudaError_t dalloc(mcinv_ctx *h, T **p, size_t count)
{
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) { *p = nullptr; return e; }
    h->allocs.push_back((void *)*p);
    h->bytes += (int64_t)bytes;
    return cudaSuccess;
}

template <typename T>
static cudaError_t upload(mcinv_ctx *h, T **p, const std::vector<T> &v)
{
    cudaError_t e = dalloc(h, p, v.size());
    if (e != cudaSuccess) return e;
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream);
}

extern "C" void mcinv_default_options(mcinv_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->K = 1024;
    opt->acc = MCINV_ACC_BF16_TC;
}

static int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    return sms;
}

// Default slice shape, from measurements on the workloads of this library:
// real sweeps run best with 32-chain slices (8 lanes x 4 chains, one 128-byte
// line per gathered row) spread over a cluster when there are few slices,
// about 128 CTAs of 512 threads; complex sweeps with about 256 CTAs of 256
// threads (two per SM) and 16- to 64-chain slices.  The autotuner
// (MCINV_F_AUTOTUNE) times the alternatives on the actual matrix instead.
static void choose_shape(int64_t K, int cplx, int sms, int *W, int *Q, int *T)
{
    const int vmax = (K % (cplx ? 2 : 4) == 0) ? (cplx ? 2 : 4) : 1;
    int w, q, t;
    if (!cplx) {
        w = 8 * vmax;
        t = 512;
        const int64_t slices = (K + w - 1) / w;
        q = (int)std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)std::llround(0.85 * sms / (double)std::max<int64_t>(slices, 1))));
    } else {
        w = 8 * vmax;
        t = 256;
        while (w < 32 * vmax && (K + w - 1) / w > 2 * sms) w *= 2;
        const int64_t slices = (K + w - 1) / w;
        q = (int)std::max<int64_t>(1, std::min<int64_t>(16, (2 * sms) / std::max<int64_t>(slices, 1)));
    }
    while (w > 1 && w / 2 >= K) w /= 2;
    *W = w;
    *Q = q;
    *T = t;
}

static SweepArgs sweep_args(mcinv_ctx *h, int ncyc, int noise_cyc, bool accumulate, int cyc0_in_batch);

// one sweep launch of the handle's kernel and shape
static GridArgs grid_args(mcinv_ctx *h)
{
    GridArgs g{};
    const bool pair = h->gbulk && h->gpair;
    g.pair = pair ? 1 : 0;
    g.rows = pair ? h->d_grow_p : h->d_grow;
    g.zent[0] = pair ? h->d_gpzent[0] : h->d_gzent[0]; g.zent[1] = pair ? h->d_gpzent[1] : h->d_gzent[1];
    g.went[0] = pair ? h->d_gpwent[0] : h->d_gwent[0]; g.went[1] = pair ? h->d_gpwent[1] : h->d_gwent[1];
    g.nkv = pair ? h->gpnkv : h->gnkv;
    g.kv = (int)(h->K * (h->cplx ? 8 : 4) / 16);
    g.cst = h->d_gcst;
    g.lev_ptr = h->d_levptr;
    g.nlev = h->nlev;
    g.nblk = (int)((h->K + 32 * h->V - 1) / (32 * h->V));
    g.bar = h->d_gbar;
    return g;
}

static WaveArgs wave_args(const mcinv_ctx *h)
{
    WaveArgs g{};
    g.trow = h->d_wrow;
    g.cst = h->d_gcst;
    g.h = h->wave_h;
    g.S = h->wave_S;
    g.B = h->wave_B;
    g.m = h->wave_m;
    g.sv = h->wave_sv;
    g.D = h->wave_D;
    g.exact = h->wave_exact;
    g.nb = 2 * h->wave_B + 2;
    g.nr = 2 * h->wave_B + 2;
    g.nkv = h->gpnkv;
    return g;
}
static int wave_grid(const mcinv_ctx *h) { return wave_ctas((int)(h->K * (h->cplx ? 8 : 4) / 16), h->wave_sv); }

// CTAs and warps per CTA of the sweep launch (the trace-series partials hold one
// slot per cycle, CTA and warp)
static int sweep_ctas(const mcinv_ctx *h) { return h->grid ? h->gctas : h->slices * h->Q; }
static int sweep_warps(const mcinv_ctx *h) { return h->threads / 32; }

// The state of buffer `buf` between the canonical layout and d_x in layout `layout`
// (unpack = 1: d_x -> canonical).
static cudaError_t pack_x(mcinv_ctx *h, int layout, int buf, int unpack)
{
    const size_t nx = (size_t)h->gpnkv * 16;  // bytes of one pair-layout buffer
    const int kv = (int)(h->K * (h->cplx ? 8 : 4) / 16);
    void *x = (char *)h->d_x + buf * nx;
    if (layout == 0) return launch_pair_pack(h->d_z[buf], h->d_w[buf], x, h->n, kv, unpack, h->stream);
    return launch_tile_pack(h->d_z[buf], h->d_w[buf], x, h->n, kv, unpack, h->stream, layout == 2 ? h->wave_sv : 32);
}

// The state in the canonical layout (z[n][K], w[n][K]) again, after sweeps on the
// pair layout; every reader of the state calls this first.
static cudaError_t ensure_canonical(mcinv_ctx *h)
{
    if (h->canon_ok) return cudaSuccess;
    cudaError_t e = pack_x(h, h->x_layout, h->cur, 1);
    if (e == cudaSuccess) h->canon_ok = true;
    return e;
}

static cudaError_t sweep_launch(mcinv_ctx *h, const SweepArgs &a)
{
    if (h->grid && h->gbulk && h->gpair) {
        // the pair layout (block-major for the tiled sweep, sliced for the wavefront
        // sweep): packed from the canonical state when that is the newer, after
        // unpacking another of these layouts if it held it
        const size_t nx = (size_t)h->gpnkv * 16;
        const int layout = h->gwave ? 2 : h->gtile ? 1 : 0;
        if (h->pair_ok && h->x_layout != layout) {
            cudaError_t e = ensure_canonical(h);
            if (e != cudaSuccess) return e;
            h->pair_ok = false;
        }
        if (!h->pair_ok) {
            cudaError_t e = pack_x(h, layout, a.cur, 0);
            if (e != cudaSuccess) return e;
            h->pair_ok = true;
            h->x_layout = layout;
        }
        SweepArgs b = a;
        b.z[0] = h->d_x;
        b.z[1] = (char *)h->d_x + nx;
        b.w[0] = b.z[0];
        b.w[1] = b.z[1];
        h->canon_ok = false;
        if (h->gwave) return launch_sweep_wave(b, wave_args(h), h->cplx, h->stream);
        if (h->gtile) {
            TileArgs t{h->d_trow, h->d_tptr, h->d_tslots, h->d_levtile, h->d_rptr, h->d_rrow, h->d_rlen};
            return launch_sweep_tiled(b, grid_args(h), t, h->cplx, h->gctas, h->stream);
        }
        return launch_sweep_grid(b, grid_args(h), h->cplx, h->gctas, h->threads, h->gbulk, h->stream);
    }
    if (h->grid) return launch_sweep_grid(a, grid_args(h), h->cplx, h->gctas, h->threads, h->gbulk, h->stream);
    if (h->staged) return launch_sweep_staged(a, h->LPR, h->slices, h->stream);
    return launch_sweep(a, h->cplx, h->LPR, h->V, h->slices, h->threads, h->stream);
}

// Autotuner: time every reasonable slice shape (chains per CTA, CTAs per
// cluster, threads per CTA) for two burn-in cycles on the handle's own matrix
// from the zero state, keep the fastest, and put the state back to zero.  The
// choice is cached per (n, nnz, K, real/complex) for the process.
struct TunedShape {
    int W, V, LPR, Q, T;
    bool staged;
    bool grid = false;
    bool gbulk = false;
    bool gpair = false;
    bool gtile = false;
    bool gwave = false;
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int64_t, int64_t, int64_t, int>, TunedShape> g_tune_cache;

static mcinv_status autotune(mcinv_ctx *h)
{
    const auto key = std::make_tuple(h->n, h->nnz, h->K, h->cplx | (h->ord.empty() ? 0 : 2));
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        // (a shape on the pair layout is for handles that hold the pair buffers)
        if (it != g_tune_cache.end() && (!it->second.gpair || h->d_x) && (!it->second.gtile || h->tile_able) &&
            (!it->second.gwave || h->wave_able)) {
            h->W = it->second.W; h->V = it->second.V; h->LPR = it->second.LPR;
            h->Q = it->second.Q; h->threads = it->second.T; h->staged = it->second.staged;
            h->grid = it->second.grid;
            h->gbulk = it->second.gbulk;
            h->gpair = it->second.gpair;
            h->gtile = it->second.gtile;
            h->gwave = it->second.gwave;
            if (h->grid) h->gctas = h->gwave ? wave_grid(h) : h->gtile ? tiled_ctas(h->cplx)
                                                                     : grid_ctas(h->cplx, h->threads, h->gbulk, h->gpair);
            h->slices = (int)((h->K + h->W - 1) / h->W);
            return MCINV_OK;
        }
    }
    const int sms = sm_count();
    const int vmax = (h->K % (h->cplx ? 2 : 4) == 0) ? (h->cplx ? 2 : 4) : 1;
    const int ncyc = (int)std::min<int64_t>(2, h->B);
    LAUNCH_K(h, MCINV_KERNEL_NOISE, launch_noise(h->seed, h->matrix_id, (uint64_t)h->chain_base, (int)h->K, (int)h->n,
                                                 0, ncyc, h->d_pos, h->d_noise, h->stream));
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    TunedShape best{h->W, h->V, h->LPR, h->Q, h->threads, h->staged, h->grid, h->gbulk, h->gpair, h->gtile, h->gwave};
    float best_ms = 1e30f;
    for (int lpr = 1; lpr <= 32; lpr *= 2) {
        const int W = lpr * vmax;
        if (W > h->K && lpr > 1) break;
        const int slices = (int)((h->K + W - 1) / W);
        for (int Q = 1; Q <= 16; Q *= 2) {
            if (Q > 1 && (int64_t)slices * Q > 2 * sms) break;
            if ((int64_t)slices * Q < std::min<int64_t>(64, slices) || (int64_t)slices * Q > 8 * sms) continue;
            for (int T = 256; T <= 512; T *= 2) {
                if (Q > 1 && max_active_clusters(h->cplx, lpr, vmax, T, Q, h->blob_max) < 1) continue;
                const int sW = h->W, sV = h->V, sL = h->LPR, sQ = h->Q, sT = h->threads, sS = h->slices;
                h->W = W; h->V = vmax; h->LPR = lpr; h->Q = Q; h->threads = T; h->slices = slices;
                SweepArgs a = sweep_args(h, ncyc, 0, false, 0);
                float ms = 1e30f;
                cudaError_t e = launch_sweep(a, h->cplx, lpr, vmax, slices, T, h->stream);  // warm-up
                if (e == cudaSuccess) {
                    cudaEventRecord(e0, h->stream);
                    e = launch_sweep(a, h->cplx, lpr, vmax, slices, T, h->stream);
                    cudaEventRecord(e1, h->stream);
                    if (e == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                }
                if (e != cudaSuccess) cudaGetLastError();  // launch refused: skip this shape
                h->launches += 2;
                if (ms < best_ms) { best_ms = ms; best = TunedShape{W, vmax, lpr, Q, T, false, false}; }
                h->W = sW; h->V = sV; h->LPR = sL; h->Q = sQ; h->threads = sT; h->slices = sS;
            }
        }
    }
    // the staged kernel: real matrices, 4 chains per lane
    for (int lpr = 4; lpr <= 8; lpr *= 2) {
        if (!staged_supported(h->cplx, lpr, vmax, h->K, h->blob_max)) continue;
        const int W = lpr * vmax;
        const int slices = (int)((h->K + W - 1) / W);
        for (int Q = 1; Q <= 16; Q *= 2) {
            if ((int64_t)slices * Q > 2 * sms) break;
            if ((int64_t)slices * Q < std::min<int64_t>(64, slices)) continue;
            const int sW = h->W, sV = h->V, sL = h->LPR, sQ = h->Q, sT = h->threads, sS = h->slices;
            h->W = W; h->V = vmax; h->LPR = lpr; h->Q = Q; h->threads = staged_threads(); h->slices = slices;
            SweepArgs a = sweep_args(h, ncyc, 0, false, 0);
            float ms = 1e30f;
            cudaError_t e = launch_sweep_staged(a, lpr, slices, h->stream);  // warm-up
            if (e == cudaSuccess) {
                cudaEventRecord(e0, h->stream);
                e = launch_sweep_staged(a, lpr, slices, h->stream);
                cudaEventRecord(e1, h->stream);
                if (e == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            }
            if (e != cudaSuccess) cudaGetLastError();
            h->launches += 2;
            if (ms < best_ms) { best_ms = ms; best = TunedShape{W, vmax, lpr, Q, staged_threads(), true, false}; }
            h->W = sW; h->V = sV; h->LPR = sL; h->Q = sQ; h->threads = sT; h->slices = sS;
        }
    }
    // the grid-wide kernel: one warp per (row, 32 x V chains), all SMs per level
    for (int variant = 0; variant < 11; ++variant) {
        // register gathers with 384 or 512 threads; bulk-staged with 1, 2 or 4 vectors per
        // lane (12 warps of 32 slots) or 1 (16 warps of 24 slots); bulk-staged on the pair
        // layout (structurally symmetric matrices) with one vector a lane (16 warps) or two
        // (12 or 8 warps); the tile-staged sweep (pair layout, 16 warps) where C has a tiled
        // form; the wavefront sweep (sliced layout, 16 warps) where C has a wavefront form
        static const int kT[11] = {384, 512, 384, 192, 96, 512, 512, 384, 256, 512, 512};
        const int T = kT[variant];
        const bool bulk = variant >= 2;
        const bool pair = variant == 5 || variant >= 7;
        const bool tile = variant == 9;
        const bool wave = variant == 10;
        if (pair && !h->d_x) continue;
        if (tile && !h->tile_able) continue;
        if (wave && !h->wave_able) continue;
        const int ctas = wave ? wave_grid(h) : tile ? tiled_ctas(h->cplx) : grid_ctas(h->cplx, T, bulk, pair);
        if (!grid_supported(h->cplx, vmax, h->K, pair ? 512 : T, bulk) || ctas < 1 || h->gnkv == 0) continue;
        const int sW = h->W, sV = h->V, sL = h->LPR, sQ = h->Q, sT = h->threads, sS = h->slices, sC = h->gctas;
        const bool sG = h->grid, sB = h->gbulk, sP = h->gpair, sI = h->gtile, sX = h->gwave;
        h->V = vmax; h->W = 32 * vmax; h->LPR = 32; h->Q = 1; h->threads = T; h->gctas = ctas; h->grid = true;
        h->gbulk = bulk;
        h->gpair = pair;
        h->gtile = tile;
        h->gwave = wave;
        h->slices = (int)((h->K + h->W - 1) / h->W);
        SweepArgs a = sweep_args(h, ncyc, 0, false, 0);
        float ms = 1e30f;
        cudaError_t e = sweep_launch(h, a);  // warm-up
        if (e == cudaSuccess) {
            cudaEventRecord(e0, h->stream);
            e = sweep_launch(h, a);
            cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        }
        if (e != cudaSuccess) cudaGetLastError();
        h->launches += 2;
        if (ms < best_ms) {
            best_ms = ms;
            best = TunedShape{32 * vmax, vmax, 32, 1, T, false, true, bulk, pair, tile, wave};
        }
        h->W = sW; h->V = sV; h->LPR = sL; h->Q = sQ; h->threads = sT; h->slices = sS; h->gctas = sC; h->grid = sG;
        h->gbulk = sB;
        h->gpair = sP;
        h->gtile = sI;
        h->gwave = sX;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->W = best.W; h->V = best.V; h->LPR = best.LPR; h->Q = best.Q; h->threads = best.T; h->staged = best.staged;
    h->grid = best.grid;
    h->gbulk = best.gbulk;
    h->gpair = best.gpair;
    h->gtile = best.gtile;
    h->gwave = best.gwave;
    h->gctas = h->grid ? (h->gwave ? wave_grid(h) : h->gtile ? tiled_ctas(h->cplx)
                                                             : grid_ctas(h->cplx, h->threads, h->gbulk, h->gpair))
                       : 0;
    h->slices = (int)((h->K + h->W - 1) / h->W);
    // back to Algorithm 1 step 1: z = w = 0, nothing run yet
    const size_t bytes = (size_t)h->n * (size_t)h->K * (h->cplx ? 8 : 4);
    for (int b = 0; b < 2; ++b) {
        CUDA_TRY(h, cudaMemsetAsync(h->d_z[b], 0, bytes, h->stream));
        CUDA_TRY(h, cudaMemsetAsync(h->d_w[b], 0, bytes, h->stream));
    }
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->canon_ok = true;
    h->pair_ok = false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    return MCINV_OK;
}

static mcinv_status create_impl(mcinv_t *out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                                const double *val, mcinv_dtype dt, const mcinv_options *opt_in, const Partition *part);

extern "C" mcinv_status mcinv_create(mcinv_t *out, int64_t n, const int64_t *row_ptr,
                                     const int32_t *col, const double *val, mcinv_dtype dt,
                                     const mcinv_options *opt_in)
{
    return create_impl(out, n, row_ptr, col, val, dt, opt_in, nullptr);
}

extern "C" mcinv_status mcinv_create_partitioned(mcinv_t *out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                                                 const double *val, mcinv_dtype dt, const mcinv_options *opt,
                                                 int64_t nblocks, const int64_t *block_ptr)
{
    if (!out) return fail(nullptr, MCINV_E_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || n > (1LL << 30)) return fail(nullptr, MCINV_E_ARG, "n = %lld out of range", (long long)n);
    if (dt != MCINV_REAL64 && dt != MCINV_COMPLEX128) return fail(nullptr, MCINV_E_ARG, "bad dtype");
    // the block sweep of C is the row sweep of C~ = S^-1 C S^-1 (Sec. 4 partition)
    Partition part;
    std::vector<int64_t> rp2;
    std::vector<int32_t> col2;
    std::vector<double> val2;
    std::string why;
    const mcinv_status st = partition_transform(n, row_ptr, col, val, dt == MCINV_COMPLEX128, nblocks, block_ptr, rp2,
                                                col2, val2, part, &why);
    if (st != MCINV_OK) return fail(nullptr, st, "%s", why.c_str());
    return create_impl(out, n, rp2.data(), col2.data(), val2.data(), dt, opt, &part);
}

static mcinv_status create_impl(mcinv_t *out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                                const double *val, mcinv_dtype dt, const mcinv_options *opt_in, const Partition *part)
{
    if (!out) return fail(nullptr, MCINV_E_ARG, "out is NULL");
    *out = nullptr;
    mcinv_options opt;
    if (opt_in) opt = *opt_in;
    else mcinv_default_options(&opt);
    if (n <= 0 || n > (1LL << 30)) return fail(nullptr, MCINV_E_ARG, "n = %lld out of range", (long long)n);
    if (!row_ptr || !col || !val) return fail(nullptr, MCINV_E_ARG, "NULL CSR array");
    if (dt != MCINV_REAL64 && dt != MCINV_COMPLEX128) return fail(nullptr, MCINV_E_ARG, "bad dtype");
    if (opt.K < 1 || opt.K > (1LL << 24)) return fail(nullptr, MCINV_E_ARG, "K = %lld out of range", (long long)opt.K);
    if (row_ptr[0] != 0) return fail(nullptr, MCINV_E_ARG, "row_ptr[0] != 0");
    const int64_t nnz = row_ptr[n];
    if (nnz < n || nnz > (1LL << 31) - 1) return fail(nullptr, MCINV_E_ARG, "nnz = %lld out of range", (long long)nnz);
    if ((double)n * (double)opt.K > 4.0e9) return fail(nullptr, MCINV_E_ARG, "n*K too large");
    const int cplx = dt == MCINV_COMPLEX128;
    const int NV = cplx ? 2 : 1;

    // the colour order (Sec. 4): sample C' = P C P^T, whose Gauss-Seidel sweep has
    // one dependency level per colour; row-indexed inputs and outputs are mapped
    std::vector<int32_t> ord, inv;
    std::vector<int64_t> rp2;
    std::vector<int32_t> col2;
    std::vector<double> val2;
    if (opt.flags & MCINV_F_COLOR_ORDER) {
        std::string why;
        int nc = 0;
        const mcinv_status st = color_order(n, row_ptr, col, val, cplx, ord, &nc, &why);
        if (st != MCINV_OK) return fail(nullptr, st, "%s", why.c_str());
        permute_csr(n, row_ptr, col, val, cplx, ord, rp2, col2, val2);
        inv.resize(n);
        for (int64_t k = 0; k < n; ++k) inv[ord[k]] = (int32_t)k;
        row_ptr = rp2.data();
        col = col2.data();
        val = val2.data();
    }
    Prepared P;
    {
        std::string why;
        const mcinv_status st = prepare_matrix(n, row_ptr, col, val, cplx, 48 * 1024, P, &why);
        if (st != MCINV_OK) return fail(nullptr, st, "%s", why.c_str());
    }
    mcinv_ctx *h = new (std::nothrow) mcinv_ctx;
    if (!h) return fail(nullptr, MCINV_E_NOMEM, "host allocation failed");
    h->n = n; h->nnz = nnz; h->K = opt.K; h->cplx = cplx;
    h->seed = opt.seed; h->chain_base = opt.chain_base; h->matrix_id = opt.matrix_id;
    h->stream = (cudaStream_t)opt.stream;
    h->flags = opt.flags;
    h->ord = std::move(ord);
    h->inv = inv;
    h->acc = opt.acc;
    h->B = opt.batch_cycles > 0 ? opt.batch_cycles : 8;
    int default_threads = 256;
    {
        int w = 0, q = 1;
        choose_shape(opt.K, cplx, sm_count(), &w, &q, &default_threads);
        h->W = opt.chains_per_cta > 0 ? opt.chains_per_cta : w;
        h->Q = opt.ctas_per_slice > 0 ? opt.ctas_per_slice : (opt.chains_per_cta > 0 ? 1 : q);
        if (h->Q > 16) {
            delete h;
            return fail(nullptr, MCINV_E_ARG, "ctas_per_slice must be <= 16");
        }
    }
    {
        // V chains per lane (one vector load per gather) when K allows it
        const int vmax = cplx ? 2 : 4;
        h->V = (opt.K % vmax == 0 && h->W % vmax == 0) ? vmax : 1;
        h->LPR = h->W / h->V;
        if ((h->W & (h->W - 1)) || h->LPR < 1 || h->LPR > 32) {
            delete h;
            return fail(nullptr, MCINV_E_ARG, "chains_per_cta must be a power of two <= %d for K = %lld",
                        32 * h->V, (long long)opt.K);
        }
    }
    h->threads = opt.threads_per_cta > 0 ? opt.threads_per_cta : default_threads;
    if (h->threads % 32 || h->threads > 512) {
        delete h;
        return fail(nullptr, MCINV_E_ARG, "threads_per_cta must be a multiple of 32, <= 512");
    }
    h->slices = (int)((opt.K + h->W - 1) / h->W);
    h->nw = (int)((opt.K + 31) / 32);
    mcinv_t H = h;
    auto bail = [&](mcinv_status st) {
        std::string msg = h->err;
        mcinv_destroy(H);
        g_create_error = msg;
        return st;
    };

    h->nlev = P.nlev;
    h->blob_max = P.blob_max;
    h->nchunks = (int)P.chunks.size();
    const std::vector<int32_t> &perm = P.perm;
    // ---- clusters: fall back to smaller ones if this one cannot be resident
    if (h->Q > 1) {
        int q = h->Q;
        while (q > 1 && max_active_clusters(cplx, h->LPR, h->V, h->threads, q, h->blob_max) < 1) --q;
        if (q != h->Q && opt.ctas_per_slice > 0) {
            fail(h, MCINV_E_UNSUPPORTED, "a cluster of %d CTAs of %d threads cannot be resident", opt.ctas_per_slice, h->threads);
            return bail(MCINV_E_UNSUPPORTED);
        }
        h->Q = q;
    }

    if ((h->flags & MCINV_F_GRID_PAIR) && !((h->flags & MCINV_F_GRID) && (h->flags & MCINV_F_GRID_BULK))) {
        fail(h, MCINV_E_ARG, "MCINV_F_GRID_PAIR needs MCINV_F_GRID and MCINV_F_GRID_BULK");
        return bail(MCINV_E_ARG);
    }
    if (h->flags & MCINV_F_STAGED) {
        if (!staged_supported(cplx, h->LPR, h->V, opt.K, h->blob_max)) {
            fail(h, MCINV_E_UNSUPPORTED,
                 "the staged sweep needs a real matrix, 4 or 8 lanes per row of 4 chains (16- or 32-chain slices) and K a multiple of the slice");
            return bail(MCINV_E_UNSUPPORTED);
        }
        h->staged = true;
        h->threads = staged_threads();
    }
    if (h->flags & MCINV_F_GRID) {
        const int vmax = cplx ? 2 : 4;
        const bool bulk = (h->flags & MCINV_F_GRID_BULK) != 0;
        const int T = opt.threads_per_cta > 0 ? opt.threads_per_cta : 384;
        // (with bulk staging and no explicit shape, or MCINV_F_GRID_PAIR, the pair layout is
        // chosen below when it applies)
        const bool fpair = (h->flags & MCINV_F_GRID_PAIR) != 0;
        if (fpair && ((h->flags & MCINV_F_GRID_NOPAIR) || (T != 512 && T != 384 && T != 256))) {
            fail(h, MCINV_E_ARG, "MCINV_F_GRID_PAIR takes 512, 384 or 256 threads per CTA, not MCINV_F_GRID_NOPAIR");
            return bail(MCINV_E_ARG);
        }
        const int ctas = grid_supported(cplx, vmax, opt.K, fpair ? 512 : T, bulk) ? grid_ctas(cplx, T, bulk, fpair) : 0;
        if (h->staged || ctas < 1) {
            fail(h, MCINV_E_UNSUPPORTED,
                 "the grid-wide sweep needs K a multiple of %d, 384 or 512 threads per CTA (96, 192, 384 or 512 "
                 "with MCINV_F_GRID_BULK), a resident CTA per SM and not MCINV_F_STAGED", vmax);
            return bail(MCINV_E_UNSUPPORTED);
        }
        h->grid = true;
        h->gbulk = bulk;
        h->gctas = ctas;
        h->V = vmax; h->W = 32 * vmax; h->LPR = 32; h->Q = 1; h->threads = T;
        h->slices = (int)((opt.K + h->W - 1) / h->W);
    }
    double *d_diag = nullptr;
    long long *d_cst_at = nullptr;
    std::vector<int32_t> bad_init(1, 0x7fffffff);
    int *d_bad = nullptr;
#define SETUP(call)                                                                               \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            mcinv_status st_ = e_ == cudaErrorMemoryAllocation ? MCINV_E_NOMEM : MCINV_E_CUDA;    \
            fail(h, st_, "%s: %s", #call, cudaGetErrorString(e_));                                \
            return bail(st_);                                                                     \
        }                                                                                         \
    } while (0)
    SETUP(upload(h, &h->d_stream, P.stream));
    SETUP(upload(h, &h->d_chunks, P.chunks));
    SETUP(upload(h, &h->d_perm, P.perm));
    SETUP(upload(h, &h->d_pos, P.pos));
    SETUP(upload(h, &d_diag, P.diag_pos));
    SETUP(upload(h, &d_cst_at, P.cst_at));
    SETUP(upload(h, &d_bad, bad_init));
    SETUP(launch_constants((int)n, d_diag, cplx, h->d_stream, d_cst_at, d_bad, h->stream));
    h->launches++;
    if (opt.K % (cplx ? 2 : 4) == 0 && (double)n * (double)opt.K / (cplx ? 2 : 4) < 2147483648.0) {
        // the flat form for the grid-wide sweep: records (.row = i K / V), entries for
        // each cycle parity (.col = index of the gathered vector from z[0] / w[0]:
        // this cycle's buffer for j < i, last cycle's for j > i), constants by position
        const uint32_t kv = (uint32_t)(opt.K / (cplx ? 2 : 4));
        h->gnkv = (uint32_t)n * kv;
        std::vector<GridRow> grow = P.grow;
        const size_t esz_ent = cplx ? sizeof(EntC) : sizeof(EntR);
        for (int par = 0; par < 2; ++par) {
            // par: the buffer that holds last cycle's state; this cycle writes the other
            const uint32_t off_new = par ? 0u : h->gnkv, off_old = par ? h->gnkv : 0u;
            std::vector<uint8_t> ez = P.gzent, ew = P.gwent;
            for (int64_t p = 0; p < n; ++p) {
                const int i = P.grow[p].row;
                auto fix = [&](std::vector<uint8_t> &v, int b, int e) {
                    for (int q = b; q < e; ++q) {
                        int *c = (int *)(v.data() + (size_t)q * esz_ent);  // .col of EntR / EntC
                        *c = (int)((*c < i ? off_new : off_old) + (uint32_t)*c * kv);
                    }
                };
                fix(ez, P.grow[p].zb, P.grow[p + 1].zb);
                fix(ew, P.grow[p].wb, P.grow[p + 1].wb);
            }
            SETUP(upload(h, &h->d_gzent[par], ez));
            SETUP(upload(h, &h->d_gwent[par], ew));
        }
        for (int64_t p = 0; p < n; ++p) grow[p].row = (int)((uint32_t)P.grow[p].row * kv);
        SETUP(upload(h, &h->d_grow, grow));
        // the pair form, for structurally symmetric matrices (row i of C and of
        // C^dagger name the same columns in the same order): offsets into the pair
        // layout, rows of 2 kvp vectors (kvp: kv rounded up to a whole chain block)
        const uint32_t kvp = (kv + 31) / 32 * 32;
        bool sym = P.gzent.size() == P.gwent.size() && 2.0 * 2.0 * (double)n * kvp < 4294967296.0;
        for (int64_t p = 0; p < n && sym; ++p) {
            const int zb = P.grow[p].zb, ze = P.grow[p + 1].zb, wb = P.grow[p].wb, we = P.grow[p + 1].wb;
            if (ze - zb != we - wb) { sym = false; break; }
            for (int q = 0; q < ze - zb; ++q)
                if (*(const int *)(P.gzent.data() + (size_t)(zb + q) * esz_ent) !=
                    *(const int *)(P.gwent.data() + (size_t)(wb + q) * esz_ent)) { sym = false; break; }
        }
        if (sym) {
            h->gpnkv = (uint32_t)n * 2u * kvp;
            for (int par = 0; par < 2; ++par) {
                const uint32_t off_new = par ? 0u : h->gpnkv, off_old = par ? h->gpnkv : 0u;
                std::vector<uint8_t> ez = P.gzent, ew = P.gwent;
                for (int64_t p = 0; p < n; ++p) {
                    const int i = P.grow[p].row;
                    auto fix = [&](std::vector<uint8_t> &v, int b, int e) {
                        for (int q = b; q < e; ++q) {
                            int *c = (int *)(v.data() + (size_t)q * esz_ent);
                            *c = (int)((*c < i ? off_new : off_old) + (uint32_t)*c * 2u * kvp);
                        }
                    };
                    fix(ez, P.grow[p].zb, P.grow[p + 1].zb);
                    fix(ew, P.grow[p].wb, P.grow[p + 1].wb);
                }
                SETUP(upload(h, &h->d_gpzent[par], ez));
                SETUP(upload(h, &h->d_gpwent[par], ew));
            }
            std::vector<GridRow> growp = P.grow;
            for (int64_t p = 0; p < n; ++p) growp[p].row = (int)((uint32_t)P.grow[p].row * 2u * kvp);
            SETUP(upload(h, &h->d_grow_p, growp));
            h->pair_able = true;
            // the tiled form: the largest tiles whose staged neighbours fit the stage
            // buffers (lattices in the colour order; a random pattern has none)
            {
                std::vector<int> tptr, tslots, levtile, rptr, rrow, rlen;
                std::vector<uint16_t> slot;
                for (int ts : {64, 32, 16, 8}) {
                    if (!build_tiles(P.grow, P.gzent, esz_ent, P.lev_ptr, ts, tptr, tslots, levtile, rptr, rrow, rlen,
                                     slot))
                        continue;
                    SETUP(upload(h, &h->d_trow, build_tile_rows(P.grow, P.gzent, P.gwent, slot, cplx)));
                    SETUP(upload(h, &h->d_tptr, tptr));
                    SETUP(upload(h, &h->d_tslots, tslots.empty() ? std::vector<int>(1, 0) : tslots));
                    SETUP(upload(h, &h->d_levtile, levtile));
                    SETUP(upload(h, &h->d_rptr, rptr));
                    SETUP(upload(h, &h->d_rrow, rrow.empty() ? std::vector<int>(1, 0) : rrow));
                    SETUP(upload(h, &h->d_rlen, rlen.empty() ? std::vector<int>(1, 0) : rlen));
                    h->tile_able = true;
                    h->tile_size = ts;
                    break;
                }
            }
            // the wavefront form: two colours whose chunks touch only nearby chunks (lattices
            // in the colour order)
            {
                WaveForm wf;
                if (build_wave(P.grow, P.gzent, P.gwent, esz_ent, P.lev_ptr, cplx, (int)kv, sm_count(), wf)) {
                    SETUP(upload(h, &h->d_wrow, wf.trow));
                    h->wave_able = true;
                    h->wave_S = wf.S;
                    h->wave_B = wf.B;
                    h->wave_m = wf.m;
                    h->wave_h = wf.h;
                    h->wave_sv = wf.sv;
                    h->wave_D = wf.D;
                    h->wave_exact = wf.exact ? 1 : 0;
                }
            }
        }
        SETUP(upload(h, &h->d_levptr, P.lev_ptr));
        SETUP(dalloc(h, &h->d_gbar, 1));
        const size_t csz = cplx ? sizeof(CstC) : sizeof(CstR);
        std::vector<long long> at((size_t)n);
        for (int64_t p = 0; p < n; ++p) at[p] = (long long)(p * csz);
        long long *d_at = nullptr;
        SETUP(upload(h, &d_at, at));
        SETUP(dalloc(h, &h->d_gcst, (size_t)n * csz));
        SETUP(launch_constants((int)n, d_diag, cplx, h->d_gcst, d_at, d_bad, h->stream));
        h->launches++;
    } else if (h->grid) {
        fail(h, MCINV_E_UNSUPPORTED, "the grid-wide sweep needs n K / V < 2^31");
        return bail(MCINV_E_UNSUPPORTED);
    }
    // ---- chain state (Algorithm 1 step 1: z = w = 0), noise plane, accumulators
    const size_t esz = cplx ? 8 : 4;
    const size_t state = (size_t)n * (size_t)opt.K;
    // the two buffers of z (and of w) are one allocation: the grid-wide sweep
    // addresses both from z[0]
    SETUP(dalloc(h, (char **)&h->d_z[0], 2 * state * esz));
    SETUP(dalloc(h, (char **)&h->d_w[0], 2 * state * esz));
    h->d_z[1] = (char *)h->d_z[0] + state * esz;
    h->d_w[1] = (char *)h->d_w[0] + state * esz;
    SETUP(cudaMemsetAsync(h->d_z[0], 0, 2 * state * esz, h->stream));
    SETUP(cudaMemsetAsync(h->d_w[0], 0, 2 * state * esz, h->stream));
    // the pair-layout buffers, when the bulk sweep may run on them
    const bool fpair = (h->flags & MCINV_F_GRID_PAIR) != 0;
    if (fpair && !h->pair_able) {
        fail(h, MCINV_E_UNSUPPORTED, "MCINV_F_GRID_PAIR needs a structurally symmetric C (row i of C and of "
                                     "C^dagger naming the same columns)");
        return bail(MCINV_E_UNSUPPORTED);
    }
    const bool want_pair = h->pair_able && !(h->flags & MCINV_F_GRID_NOPAIR) &&
                           (((h->flags & MCINV_F_GRID) && h->gbulk && (opt.threads_per_cta <= 0 || fpair)) ||
                            ((h->flags & MCINV_F_AUTOTUNE) && !(h->flags & MCINV_F_GRID)));
    if (want_pair) {
        // the pair layout: 12 warps a CTA, two 32-vector blocks a warp, by default
        const int pt = fpair && opt.threads_per_cta > 0 ? opt.threads_per_cta : 384;
        const int pc = grid_ctas(cplx, pt, true, true);
        if (pc > 0) {
            SETUP(dalloc(h, (char **)&h->d_x, 2 * (size_t)h->gpnkv * 16));
            if (h->grid) {
                h->gpair = true;
                h->threads = pt;
                h->gctas = pc;
            }
        } else if (fpair) {
            fail(h, MCINV_E_UNSUPPORTED, "the pair-layout sweep with %d threads per CTA has no resident CTA", pt);
            return bail(MCINV_E_UNSUPPORTED);
        }
    }
    if (h->flags & MCINV_F_GRID_TILE) {
        if (!(h->flags & MCINV_F_GRID) || !(h->flags & MCINV_F_GRID_BULK) || (h->flags & MCINV_F_GRID_NOPAIR)) {
            fail(h, MCINV_E_ARG, "MCINV_F_GRID_TILE needs MCINV_F_GRID and MCINV_F_GRID_BULK, not MCINV_F_GRID_NOPAIR");
            return bail(MCINV_E_ARG);
        }
        const int tc = tiled_ctas(cplx);
        if (!h->tile_able || !h->d_x || tc < 1) {
            fail(h, MCINV_E_UNSUPPORTED, "C has no tiled form (it needs a structurally symmetric C, no row cut into "
                                         "pieces, and tiles of consecutive positions naming at most %d neighbours)",
                 TILE_CAP);
            return bail(MCINV_E_UNSUPPORTED);
        }
        h->gpair = true;
        h->gtile = true;
        h->threads = 512;
        h->gctas = tc;
    }
    if ((h->flags & MCINV_F_TEST_EXPIRE_WAIT) && !(h->flags & MCINV_F_GRID_WAVE)) {
        fail(h, MCINV_E_ARG, "MCINV_F_TEST_EXPIRE_WAIT needs MCINV_F_GRID_WAVE");
        return bail(MCINV_E_ARG);
    }
    if (h->flags & MCINV_F_GRID_WAVE) {
        if (!(h->flags & MCINV_F_GRID) || !(h->flags & MCINV_F_GRID_BULK) || (h->flags & MCINV_F_GRID_NOPAIR) ||
            (h->flags & MCINV_F_GRID_TILE)) {
            fail(h, MCINV_E_ARG, "MCINV_F_GRID_WAVE needs MCINV_F_GRID and MCINV_F_GRID_BULK, not MCINV_F_GRID_NOPAIR "
                                 "or MCINV_F_GRID_TILE");
            return bail(MCINV_E_ARG);
        }
        if (!h->wave_able || !h->d_x) {
            fail(h, MCINV_E_UNSUPPORTED, "C has no wavefront form (it needs a structurally symmetric C in an order "
                                         "with two dependency levels of equal size, no row cut into pieces, and each "
                                         "level cut into chunks whose rows touch only nearby chunks of the other)");
            return bail(MCINV_E_UNSUPPORTED);
        }
        h->gpair = true;
        h->gwave = true;
        h->threads = 512;
        h->gctas = wave_grid(h);
    }
    SETUP(dalloc(h, &h->d_noise, (size_t)h->B * h->nw * (size_t)n));
    SETUP(dalloc(h, &h->d_status, 1));
    SETUP(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    if ((h->flags & MCINV_F_AUTOTUNE) && !(h->flags & MCINV_F_GRID) && opt.chains_per_cta == 0 && opt.threads_per_cta == 0 &&
        opt.ctas_per_slice == 0) {
        const mcinv_status st = autotune(h);
        if (st != MCINV_OK) return bail(st);
    }
    // ---- SE groups: the diagonal partials are kept per unit of seg lanes (seg x V
    //      chains, a power of two dividing the slice); G groups of whole units
    {
        const int Greq = opt.groups > 0 ? opt.groups : 32;
        // (at most a wavefront slice: the wavefront sweep sums a row's units in its slice)
        const int segmax = h->wave_able ? std::min(h->LPR, h->wave_sv) : h->LPR;
        int seg = 1;
        while (seg * 2 <= segmax && (int64_t)seg * 2 * h->V * Greq <= opt.K) seg *= 2;
        h->seg = seg;
        const int64_t u = (int64_t)seg * h->V;
        h->units = (int)((opt.K + u - 1) / u);
        h->G = 1;
        for (int g = std::min(Greq, h->units); g >= 1; --g)
            if (h->units % g == 0) { h->G = g; break; }
        h->counts.assign(h->G, 0.0);
        for (int k = 0; k < h->units; ++k)
            h->counts[k / (h->units / h->G)] += (double)std::min<int64_t>(u, opt.K - (int64_t)k * u);
    }

    if (!(h->flags & MCINV_F_NO_DIAG)) {
        SETUP(dalloc(h, (char **)&h->d_diag_part, (size_t)h->units * n * esz));
        SETUP(cudaMemsetAsync(h->d_diag_part, 0, (size_t)h->units * n * esz, h->stream));
        SETUP(dalloc(h, &h->d_diag_acc, (size_t)h->G * n * NV));
        SETUP(cudaMemsetAsync(h->d_diag_acc, 0, (size_t)h->G * n * NV * sizeof(double), h->stream));
        SETUP(upload(h, &h->d_counts, h->counts));
        SETUP(dalloc(h, &h->d_q, (size_t)n));
    }
    size_t est_elems = std::max<size_t>((size_t)n, 2);  // the trace writes mean and SE

    // ---- block estimate
    if (opt.n_block_rows > 0 && opt.n_block_cols > 0) {
        if (!opt.block_rows || !opt.block_cols) { fail(h, MCINV_E_ARG, "block index arrays are NULL"); return bail(MCINV_E_ARG); }
        if (part && part->multi > 0) {
            // rows of a block of two or more rows would need S^-1 on both sides of C~^-1
            std::vector<char> multi(n, 0);
            for (size_t b = 0; b + 1 < part->block_ptr.size(); ++b)
                if (part->block_ptr[b + 1] - part->block_ptr[b] > 1)
                    for (int64_t i = part->block_ptr[b]; i < part->block_ptr[b + 1]; ++i) multi[i] = 1;
            for (int64_t a = 0; a < opt.n_block_rows; ++a)
                if (opt.block_rows[a] >= 0 && opt.block_rows[a] < n && multi[opt.block_rows[a]]) {
                    fail(h, MCINV_E_UNSUPPORTED, "block row %lld lies in a partition block of two or more rows", (long long)opt.block_rows[a]);
                    return bail(MCINV_E_UNSUPPORTED);
                }
            for (int64_t b = 0; b < opt.n_block_cols; ++b)
                if (opt.block_cols[b] >= 0 && opt.block_cols[b] < n && multi[opt.block_cols[b]]) {
                    fail(h, MCINV_E_UNSUPPORTED, "block column %lld lies in a partition block of two or more rows", (long long)opt.block_cols[b]);
                    return bail(MCINV_E_UNSUPPORTED);
                }
        }
        h->nR = opt.n_block_rows; h->nS = opt.n_block_cols;
        std::vector<int32_t> R(h->nR), S(h->nS), rpos(n, -1), spos(n, -1);
        for (int64_t a = 0; a < h->nR; ++a) {
            if (opt.block_rows[a] < 0 || opt.block_rows[a] >= n) { fail(h, MCINV_E_ARG, "block row out of range"); return bail(MCINV_E_ARG); }
            R[a] = inv.empty() ? (int32_t)opt.block_rows[a] : inv[opt.block_rows[a]];
            if (rpos[R[a]] >= 0) { fail(h, MCINV_E_ARG, "repeated block row %lld", (long long)opt.block_rows[a]); return bail(MCINV_E_ARG); }
            rpos[R[a]] = (int32_t)a;
        }
        for (int64_t b = 0; b < h->nS; ++b) {
            if (opt.block_cols[b] < 0 || opt.block_cols[b] >= n) { fail(h, MCINV_E_ARG, "block column out of range"); return bail(MCINV_E_ARG); }
            S[b] = inv.empty() ? (int32_t)opt.block_cols[b] : inv[opt.block_cols[b]];
            if (spos[S[b]] >= 0) { fail(h, MCINV_E_ARG, "repeated block column %lld", (long long)opt.block_cols[b]); return bail(MCINV_E_ARG); }
            spos[S[b]] = (int32_t)b;
        }
        const size_t elems = (size_t)h->nR * h->nS;
        est_elems = std::max(est_elems, elems);
        SETUP(upload(h, &h->d_R, R));
        SETUP(upload(h, &h->d_S, S));
        SETUP(dalloc(h, &h->d_blk, elems * NV));
        SETUP(cudaMemsetAsync(h->d_blk, 0, elems * NV * sizeof(float), h->stream));
        SETUP(dalloc(h, &h->d_bsum, elems * NV));
        SETUP(dalloc(h, &h->d_bsq, elems * NV));
        SETUP(cudaMemsetAsync(h->d_bsum, 0, elems * NV * sizeof(double), h->stream));
        SETUP(cudaMemsetAsync(h->d_bsq, 0, elems * NV * sizeof(double), h->stream));
        if (h->acc == MCINV_ACC_BF16_TC) {
            std::vector<int32_t> rpos_p(n), spos_p(n);
            for (int64_t p = 0; p < n; ++p) { rpos_p[p] = rpos[perm[p]]; spos_p[p] = spos[perm[p]]; }
            SETUP(upload(h, &h->d_rpos, rpos_p));
            SETUP(upload(h, &h->d_spos, spos_p));
            // shadow rows hold B cycle blocks of K chains (x2 for re,im), each block
            // padded to 64 elements with zeros
            h->kp = (opt.K * NV + 63) / 64 * 64;
            h->ldsh = (long long)h->B * h->kp;
            const size_t zrows = (size_t)((h->nR + 127) / 128 * 128);
            const size_t wrows = (size_t)(((h->nS * NV) + 255) / 256 * 256);
            SETUP(dalloc(h, &h->d_zsh, zrows * (size_t)h->ldsh));
            SETUP(dalloc(h, &h->d_wsh, wrows * (size_t)h->ldsh));
            SETUP(cudaMemsetAsync(h->d_zsh, 0, zrows * (size_t)h->ldsh * 2, h->stream));
            SETUP(cudaMemsetAsync(h->d_wsh, 0, wrows * (size_t)h->ldsh * 2, h->stream));
            std::string why;
            h->gemm = tc_gemm_plan_create(h->d_zsh, zrows, h->d_wsh, wrows, h->ldsh, h->d_blk,
                                          h->nR, h->nS * NV, &why);
            if (!h->gemm) { fail(h, MCINV_E_UNSUPPORTED, "tensor-core block contraction: %s", why.c_str()); return bail(MCINV_E_UNSUPPORTED); }
        } else if (h->acc != MCINV_ACC_FP32_SIMT) {
            fail(h, MCINV_E_ARG, "unknown accumulation mode %d", h->acc);
            return bail(MCINV_E_ARG);
        }
    }
    SETUP(dalloc(h, &h->d_mean, est_elems * NV));
    SETUP(dalloc(h, &h->d_se, est_elems * NV));

    // ---- block partition: the row pairs of every block of two or more rows (rows of
    //      the sampled matrix), the chain range of each SE group, the FP64 sums
    if (part && part->multi > 0) {
        h->part = *part;
        std::vector<int32_t> er, es;
        for (int64_t b = 0; b + 1 < (int64_t)part->block_ptr.size(); ++b) {
            const int64_t b0 = part->block_ptr[b], sz = part->block_ptr[b + 1] - b0;
            if (sz < 2) continue;
            h->pblk.push_back(b);
            h->pent_off.push_back((int64_t)er.size());
            for (int64_t r = 0; r < sz; ++r)
                for (int64_t c = 0; c < sz; ++c) {
                    er.push_back(inv.empty() ? (int32_t)(b0 + r) : inv[b0 + r]);
                    es.push_back(inv.empty() ? (int32_t)(b0 + c) : inv[b0 + c]);
                }
        }
        h->nent = (int)er.size();
        std::vector<int32_t> gch(h->G + 1);
        const int64_t u = (int64_t)h->seg * h->V, upg = h->units / h->G;
        for (int g = 0; g <= h->G; ++g) gch[g] = (int32_t)std::min<int64_t>(opt.K, (int64_t)g * upg * u);
        SETUP(upload(h, &h->d_pent_r, er));
        SETUP(upload(h, &h->d_pent_s, es));
        SETUP(upload(h, &h->d_gch, gch));
        SETUP(dalloc(h, &h->d_pacc, (size_t)h->G * h->nent * NV));
        SETUP(cudaMemsetAsync(h->d_pacc, 0, (size_t)h->G * h->nent * NV * sizeof(double), h->stream));
        if (h->d_diag_acc) SETUP(dalloc(h, &h->d_acc_est, (size_t)h->G * n * NV));
    }
    SETUP(cudaStreamSynchronize(h->stream));
    // the block accumulation on CUDA cores and the partition's block sums read the
    // state after every cycle: keep it in the canonical layout for them
    if (h->gpair && ((h->nR > 0 && h->acc == MCINV_ACC_FP32_SIMT) || h->nent > 0)) {
        h->gpair = false;
        h->threads = 384;
        h->gctas = grid_ctas(h->cplx, 384, true);
    }
    *out = h;
    return MCINV_OK;
#undef SETUP
}

static SweepArgs sweep_args(mcinv_ctx *h, int ncyc, int noise_cyc, bool accumulate, int cyc0_in_batch)
{
    SweepArgs a{};
    a.n = (int)h->n; a.K = (int)h->K; a.nw = h->nw;
    a.nchunks = h->nchunks; a.blob_max = h->blob_max;
    a.stream = h->d_stream; a.chunks = h->d_chunks;
    a.noise = h->d_noise + (size_t)noise_cyc * h->nw * (size_t)h->n;
    a.z[0] = h->d_z[0]; a.z[1] = h->d_z[1]; a.w[0] = h->d_w[0]; a.w[1] = h->d_w[1];
    a.cur = h->cur; a.ncyc = ncyc;
    a.diag_part = accumulate ? h->d_diag_part : nullptr;
    a.seg = h->seg;
    a.test_expire = (h->flags & MCINV_F_TEST_EXPIRE_WAIT) ? 1 : 0;
    if (accumulate && h->gemm) {
        a.rpos = h->d_rpos; a.spos = h->d_spos;
        a.zsh = h->d_zsh; a.wsh = h->d_wsh; a.ldsh = h->ldsh; a.kp = h->kp;
        a.cyc0_in_batch = cyc0_in_batch;
    }
    a.status = h->d_status;
    a.ctas_per_slice = h->Q;
    if (accumulate && h->d_tq) {
        a.tq = h->d_tq;
        a.tpart = h->d_tpart;
    }
    return a;
}

// Append the last sweep launch's `ncyc` trace-series values (device FP64).
static mcinv_status series_append(mcinv_ctx *h, int ncyc)
{
    if (h->nseries + ncyc > h->cap_series) {
        const int64_t cap = std::max<int64_t>(2 * h->cap_series, std::max<int64_t>(h->nseries + ncyc, 4096));
        double *nb = nullptr;
        CUDA_TRY(h, cudaMallocAsync((void **)&nb, (size_t)cap * sizeof(double), h->stream));
        if (h->nseries) CUDA_TRY(h, cudaMemcpyAsync(nb, h->d_series, (size_t)h->nseries * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        if (h->d_series) CUDA_TRY(h, cudaFreeAsync(h->d_series, h->stream));
        h->d_series = nb;
        h->cap_series = cap;
    }
    LAUNCH_K(h, MCINV_KERNEL_FOLD, launch_series_fold(ncyc, sweep_ctas(h), sweep_warps(h), h->d_tpart, (double)h->K,
                                                      h->d_series, h->nseries, h->stream));
    h->nseries += ncyc;
    return MCINV_OK;
}

static mcinv_status run_cycles(mcinv_ctx *h, int64_t cycles, bool accumulate)
{
    const bool block = accumulate && h->nR > 0;
    while (cycles > 0) {
        const int b = (int)std::min<int64_t>(h->B, cycles);
        LAUNCH_K(h, MCINV_KERNEL_NOISE, launch_noise(h->seed, h->matrix_id, (uint64_t)h->chain_base, (int)h->K, (int)h->n,
                               (uint32_t)h->cycle, b, h->d_pos, h->d_noise, h->stream));
        const bool simt_block = block && h->acc == MCINV_ACC_FP32_SIMT;
        const bool pblock = accumulate && h->nent > 0;
        if (simt_block || pblock) {
            // one cycle per launch: the state of every cycle is read before the next overwrites it
            for (int k = 0; k < b; ++k) {
                SweepArgs a = sweep_args(h, 1, k, accumulate, k);
                LAUNCH_K(h, MCINV_KERNEL_SWEEP, sweep_launch(h, a));
                if (accumulate && h->d_tq) {
                    mcinv_status st = series_append(h, 1);
                    if (st != MCINV_OK) return st;
                }
                h->cur ^= 1;
                CUDA_TRY(h, ensure_canonical(h));
                if (simt_block)
                    LAUNCH_K(h, MCINV_KERNEL_BLOCK, launch_block_simt(h->cplx, (int)h->K, h->d_z[h->cur], h->d_w[h->cur], h->d_R,
                                                (int)h->nR, h->d_S, (int)h->nS, h->d_blk, h->stream));
                if (pblock)
                    LAUNCH_K(h, MCINV_KERNEL_FOLD, launch_pblock_acc(h->cplx, h->nent, h->d_pent_r, h->d_pent_s, (int)h->K, h->G,
                                                h->d_gch, h->d_z[h->cur], h->d_w[h->cur], h->d_pacc, h->stream));
            }
            if (block && !simt_block) {
                const long long inner = (long long)b * h->kp;
                LAUNCH_K(h, MCINV_KERNEL_BLOCK, tc_gemm_run(h->gemm, inner, h->d_status, h->stream));
            }
        } else {
            SweepArgs a = sweep_args(h, b, 0, accumulate, 0);
            LAUNCH_K(h, MCINV_KERNEL_SWEEP, sweep_launch(h, a));
            if (accumulate && h->d_tq) {
                mcinv_status st = series_append(h, b);
                if (st != MCINV_OK) return st;
            }
            if (b & 1) h->cur ^= 1;
            if (block) {
                const long long inner = (long long)b * h->kp;
                LAUNCH_K(h, MCINV_KERNEL_BLOCK, tc_gemm_run(h->gemm, inner, h->d_status, h->stream));
            }
        }
        if (block) {
            const double Kd = (double)h->K;
            LAUNCH_K(h, MCINV_KERNEL_FOLD, launch_block_fold(h->cplx, (long long)h->nR * h->nS, 1.0 / (Kd * Kd * b), h->d_blk,
                                        h->d_bsum, h->d_bsq, h->acc == MCINV_ACC_FP32_SIMT, h->stream));
            h->block_batches++;
            h->block_cycles += b;
        }
        if (accumulate && h->d_diag_part) {
            LAUNCH_K(h, MCINV_KERNEL_FOLD, launch_diag_fold(h->cplx, (int)h->n, h->units, h->G, h->d_perm, h->d_diag_part, h->d_diag_acc, h->stream));
        }
        h->cycle += b;
        if (accumulate) h->samples += b;
        cycles -= b;
    }
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_burnin_coupled(mcinv_t h, double tol, int64_t max_cycles, int64_t *cycles_out)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (!(tol > 0.0) || max_cycles < 0) return fail(h, MCINV_E_ARG, "need tol > 0 and max_cycles >= 0");
    // Algorithm 1, steps 1-5, by Eq. 12: the difference of the coupled paths
    // (z* - z, started at (1..n) - 0 and sharing the noise) evolves by
    // noise-free Gauss-Seidel on C (and on C^dagger for w), identically for
    // every chain; it is swept once, one cycle at a time, until
    // max_i |d_i| < tol for both, and every chain then runs that many cycles.
    const size_t esz = h->cplx ? 8 : 4;
    const size_t n = (size_t)h->n;
    char *buf = nullptr;
    CUDA_TRY(h, cudaMallocAsync((void **)&buf, 4 * n * esz + 256, h->stream));
    void *dz[2] = {buf, buf + n * esz}, *dw[2] = {buf + 2 * n * esz, buf + 3 * n * esz};
    unsigned *d_max = (unsigned *)(buf + 4 * n * esz);
    mcinv_status st = MCINV_OK;
    int64_t p = -1;
    auto run = [&]() -> mcinv_status {
        LAUNCH_K(h, MCINV_KERNEL_SWEEP, launch_iota1(h->cplx, (int)n, dz[0], h->stream));
        LAUNCH_K(h, MCINV_KERNEL_SWEEP, launch_iota1(h->cplx, (int)n, dw[0], h->stream));
        SweepArgs a = sweep_args(h, 1, 0, false, 0);
        a.K = 1;
        a.nw = 1;
        a.noise = nullptr;
        a.ctas_per_slice = 1;
        int cur = 0;
        for (int64_t k = 1; k <= max_cycles; ++k) {
            a.z[0] = dz[0]; a.z[1] = dz[1]; a.w[0] = dw[0]; a.w[1] = dw[1];
            a.cur = cur;
            LAUNCH_K(h, MCINV_KERNEL_SWEEP, launch_sweep(a, h->cplx, 1, 1, 1, 256, h->stream));
            cur ^= 1;
            CUDA_TRY(h, cudaMemsetAsync(d_max, 0, 2 * sizeof(unsigned), h->stream));
            LAUNCH_K(h, MCINV_KERNEL_ESTIMATE, launch_maxabs2(h->cplx, (int)n, dz[cur], dw[cur], d_max, h->stream));
            unsigned m[2];
            CUDA_TRY(h, cudaMemcpyAsync(m, d_max, sizeof m, cudaMemcpyDeviceToHost, h->stream));
            CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            float fz, fw;
            std::memcpy(&fz, &m[0], 4);
            std::memcpy(&fw, &m[1], 4);
            if (fz < tol && fw < tol) {
                p = k;
                return MCINV_OK;
            }
        }
        return MCINV_OK;
    };
    st = run();
    cudaFreeAsync(buf, h->stream);
    if (st != MCINV_OK) return st;
    if (p < 0) return fail(h, MCINV_E_DIVERGED, "coupled paths still differ by more than %g after %lld cycles", tol, (long long)max_cycles);
    if (cycles_out) *cycles_out = p;
    return mcinv_burnin(h, p);
}

extern "C" mcinv_status mcinv_burnin(mcinv_t h, int64_t cycles)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (cycles < 0) return fail(h, MCINV_E_ARG, "cycles < 0");
    return run_cycles(h, cycles, false);
}

extern "C" mcinv_status mcinv_sample(mcinv_t h, int64_t cycles)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (cycles < 0) return fail(h, MCINV_E_ARG, "cycles < 0");
    return run_cycles(h, cycles, true);
}

extern "C" mcinv_status mcinv_sync(mcinv_t h)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    int status = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (status & 2) return fail(h, MCINV_E_TIMEOUT, "a bounded wait in the tensor-core contraction expired; its block batch was abandoned");
    if (status & 4) return fail(h, MCINV_E_TIMEOUT, "a bounded wait for matrix data in the sweep expired; the sweep was abandoned");
    if (status & 1) return fail(h, MCINV_E_DIVERGED, "a chain diverged (non-finite or |value| > 1e30): the sweep does not converge for this matrix");
    return MCINV_OK;
}

// The diagonal accumulators with the rows of partition blocks of two or more rows
// replaced, group by group, by the diagonal of S_b^-1 M_g S_b^-1 (M_g the group's sums
// of z~_r conj(w~_s) over the block's rows): linear in the sums, so the group means
// and SE of the estimate kernels stay exact.  Returns the buffer to estimate from.
static const double *partition_acc(mcinv_ctx *h, mcinv_status *st)
{
    *st = MCINV_OK;
    if (h->nent == 0) return h->d_diag_acc;
    const int NV = h->cplx ? 2 : 1;
    const size_t n = (size_t)h->n, G = (size_t)h->G;
    std::vector<double> pacc(G * h->nent * NV);
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess && *st == MCINV_OK) *st = fail(h, MCINV_E_CUDA, "partition estimate: %s", cudaGetErrorString(e));
    };
    chk(cudaMemcpyAsync(h->d_acc_est, h->d_diag_acc, G * n * NV * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    chk(cudaMemcpyAsync(pacc.data(), h->d_pacc, pacc.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    chk(cudaStreamSynchronize(h->stream));
    if (*st != MCINV_OK) return nullptr;
    std::vector<long long> idx;
    std::vector<double> vals;
    using cd = std::complex<double>;
    for (size_t m = 0; m < h->pblk.size(); ++m) {
        const int64_t b = h->pblk[m], b0 = h->part.block_ptr[b], sz = h->part.block_ptr[b + 1] - b0;
        const cd *Z = h->part.sinv.data() + h->part.sinv_off[b];
        for (size_t g = 0; g < G; ++g) {
            const double *M = pacc.data() + (g * h->nent + h->pent_off[m]) * NV;
            for (int64_t i = 0; i < sz; ++i) {
                cd x = 0.0;  // (Z M Z)_ii
                for (int64_t r = 0; r < sz; ++r)
                    for (int64_t c = 0; c < sz; ++c) {
                        const cd mrc = NV == 2 ? cd(M[(r * sz + c) * 2], M[(r * sz + c) * 2 + 1]) : cd(M[r * sz + c], 0.0);
                        x += Z[i * sz + r] * mrc * Z[c * sz + i];
                    }
                const int64_t row = h->inv.empty() ? b0 + i : h->inv[b0 + i];
                idx.push_back((long long)((g * n + (size_t)row) * NV));
                vals.push_back(x.real());
                if (NV == 2) {
                    idx.push_back((long long)((g * n + (size_t)row) * NV + 1));
                    vals.push_back(x.imag());
                }
            }
        }
    }
    long long *d_idx = nullptr;
    double *d_vals = nullptr;
    chk(cudaMallocAsync((void **)&d_idx, idx.size() * sizeof(long long), h->stream));
    chk(cudaMallocAsync((void **)&d_vals, vals.size() * sizeof(double), h->stream));
    if (*st == MCINV_OK) {
        chk(cudaMemcpyAsync(d_idx, idx.data(), idx.size() * sizeof(long long), cudaMemcpyHostToDevice, h->stream));
        chk(cudaMemcpyAsync(d_vals, vals.data(), vals.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        chk(launch_scatter((int)idx.size(), d_idx, d_vals, h->d_acc_est, h->stream));
        h->launches++;
    }
    if (d_idx) chk(cudaFreeAsync(d_idx, h->stream));
    if (d_vals) chk(cudaFreeAsync(d_vals, h->stream));
    chk(cudaStreamSynchronize(h->stream));
    return *st == MCINV_OK ? h->d_acc_est : nullptr;
}

// Chain state of the sampled matrix C~ to that of the block sweep of C and back:
// z = S^-1 z~, w = S^-H w~ (to_c), or z~ = S z, w~ = S^H w; x is [n][width] with rows
// of C, complex values interleaved when the handle is complex.
static void partition_state(mcinv_ctx *h, double *x, size_t width, bool is_w, bool to_c)
{
    using cd = std::complex<double>;
    const int NV = h->cplx ? 2 : 1;
    const size_t nc = width / NV;  // chains
    for (size_t m = 0; m < h->pblk.size(); ++m) {
        const int64_t b = h->pblk[m], b0 = h->part.block_ptr[b], sz = h->part.block_ptr[b + 1] - b0;
        const cd *F = (to_c ? h->part.sinv.data() : h->part.s.data()) + h->part.sinv_off[b];
        std::vector<cd> v(sz), y(sz);
        for (size_t c = 0; c < nc; ++c) {
            for (int64_t r = 0; r < sz; ++r) {
                const double *p = x + (size_t)(b0 + r) * width + c * NV;
                v[r] = NV == 2 ? cd(p[0], p[1]) : cd(p[0], 0.0);
            }
            for (int64_t r = 0; r < sz; ++r) {
                cd acc = 0.0;
                for (int64_t k = 0; k < sz; ++k) acc += (is_w ? std::conj(F[k * sz + r]) : F[r * sz + k]) * v[k];
                y[r] = acc;
            }
            for (int64_t r = 0; r < sz; ++r) {
                double *p = x + (size_t)(b0 + r) * width + c * NV;
                p[0] = y[r].real();
                if (NV == 2) p[1] = y[r].imag();
            }
        }
    }
}

// rows of C' (the colour order) back to rows of C: x[ord[k]] = x'[k], `width` values per row
static void unpermute_rows(mcinv_ctx *h, double *x, size_t width)
{
    std::vector<double> t(x, x + (size_t)h->n * width);
    for (int64_t k = 0; k < h->n; ++k)
        for (size_t v = 0; v < width; ++v) x[(size_t)h->ord[k] * width + v] = t[(size_t)k * width + v];
}

extern "C" mcinv_status mcinv_estimate(mcinv_t h, mcinv_kind kind, const double *q, double *out, double *se_out)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (!out) return fail(h, MCINV_E_ARG, "out is NULL");
    mcinv_status st = mcinv_sync(h);
    if (st != MCINV_OK) return st;
    const int NV = h->cplx ? 2 : 1;
    size_t count = 0;
    if (kind == MCINV_EST_DIAG || kind == MCINV_EST_TRACE) {
        if (!h->d_diag_acc) return fail(h, MCINV_E_STATE, "diagonal accumulation was disabled");
        if (h->samples == 0) return fail(h, MCINV_E_STATE, "no cycles sampled yet");
        mcinv_status pst;
        const double *acc_in = partition_acc(h, &pst);
        if (!acc_in) return pst;
        if (kind == MCINV_EST_DIAG) {
            LAUNCH_K(h, MCINV_KERNEL_ESTIMATE, launch_diag_estimate(h->cplx, (int)h->n, h->G, h->d_counts, (double)h->samples,
                                           acc_in, h->d_mean, h->d_se, h->stream));
            count = (size_t)h->n * NV;
            CUDA_TRY(h, cudaMemcpyAsync(out, h->d_mean, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            if (se_out) CUDA_TRY(h, cudaMemcpyAsync(se_out, h->d_se, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            if (!h->ord.empty()) {
                CUDA_TRY(h, cudaStreamSynchronize(h->stream));
                unpermute_rows(h, out, NV);
                if (se_out) unpermute_rows(h, se_out, NV);
            }
        } else {
            if (!q) return fail(h, MCINV_E_ARG, "q_diag is NULL");
            std::vector<double> qk;
            if (!h->ord.empty()) {
                qk.resize((size_t)h->n);
                for (int64_t k = 0; k < h->n; ++k) qk[k] = q[h->ord[k]];
                q = qk.data();
            }
            CUDA_TRY(h, cudaMemcpyAsync(h->d_q, q, (size_t)h->n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            LAUNCH_K(h, MCINV_KERNEL_ESTIMATE, launch_trace_estimate(h->cplx, (int)h->n, h->G, h->d_counts, (double)h->samples,
                                            acc_in, h->d_q, h->d_mean, h->stream));
            CUDA_TRY(h, cudaMemcpyAsync(out, h->d_mean, NV * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            if (se_out) CUDA_TRY(h, cudaMemcpyAsync(se_out, h->d_mean + NV, NV * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        }
    } else if (kind == MCINV_EST_BLOCK) {
        if (h->nR == 0) return fail(h, MCINV_E_STATE, "no block was configured");
        if (h->block_batches == 0) return fail(h, MCINV_E_STATE, "no cycles sampled yet");
        const long long elems = (long long)h->nR * h->nS;
        LAUNCH_K(h, MCINV_KERNEL_ESTIMATE, launch_block_estimate(h->cplx, elems, (double)h->K, (double)h->block_cycles,
                                        (double)h->block_batches, h->d_bsum, h->d_bsq, h->d_mean, h->d_se, h->stream));
        count = (size_t)elems * NV;
        CUDA_TRY(h, cudaMemcpyAsync(out, h->d_mean, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (se_out) CUDA_TRY(h, cudaMemcpyAsync(se_out, h->d_se, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    } else {
        return fail(h, MCINV_E_ARG, "unknown estimate kind %d", (int)kind);
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_set_trace_weights(mcinv_t h, const double *q)
{
    if (!h || !q) return fail(h, MCINV_E_ARG, "NULL argument");
    if (h->nent) return fail(h, MCINV_E_UNSUPPORTED, "the trace series is not available with partition blocks of two or more rows");
    if (h->samples > 0) return fail(h, MCINV_E_STATE, "trace weights must be set before sampling");
    std::vector<float> qp((size_t)h->n);
    std::vector<int32_t> perm((size_t)h->n);
    CUDA_TRY(h, cudaMemcpy(perm.data(), h->d_perm, (size_t)h->n * 4, cudaMemcpyDeviceToHost));
    for (int64_t p = 0; p < h->n; ++p) qp[p] = (float)q[h->ord.empty() ? perm[p] : h->ord[perm[p]]];
    if (!h->d_tq) {
        CUDA_TRY(h, dalloc(h, &h->d_tq, (size_t)h->n));
        CUDA_TRY(h, dalloc(h, &h->d_tpart, (size_t)h->B * sweep_ctas(h) * sweep_warps(h)));
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->d_tq, qp.data(), (size_t)h->n * 4, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->nseries = 0;
    return MCINV_OK;
}

// Geyer (1992) initial monotone sequence estimate on the per-cycle series:
// gamma(k) the lag-k autocovariance, Gamma_j = gamma(2j) + gamma(2j+1) taken
// while positive, each capped by the one before (the monotone refinement of
// the initial positive sequence), asymptotic variance
// sigma^2 = -gamma(0) + 2 sum_j Gamma_j, effective length M gamma(0) / sigma^2,
// Monte Carlo SE = sqrt(gamma(0) / effective length) (Sec. 2.3, Sec. 3.1).
static void geyer(const std::vector<double> &x, double *mean, double *var, double *ess, double *se)
{
    const size_t M = x.size();
    double m = 0.0;
    for (double v : x) m += v;
    m /= (double)M;
    auto gamma = [&](size_t k) {
        double g = 0.0;
        for (size_t t = 0; t + k < M; ++t) g += (x[t] - m) * (x[t + k] - m);
        return g / (double)M;
    };
    const double g0 = gamma(0);
    double sum = 0.0, prev = 1e300;
    for (size_t j = 0; 2 * j + 1 < M; ++j) {
        double G = gamma(2 * j) + gamma(2 * j + 1);
        if (!(G > 0.0)) break;
        G = std::min(G, prev);
        prev = G;
        sum += G;
    }
    const double sigma2 = std::max(-g0 + 2.0 * sum, 1e-300);
    *mean = m;
    *var = g0;
    *ess = (double)M * g0 / sigma2;
    *se = std::sqrt(sigma2 / (double)M);
}

extern "C" mcinv_status mcinv_trace_mc_error(mcinv_t h, double *mean, double *var, double *ess, double *se)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (h->nent) return fail(h, MCINV_E_UNSUPPORTED, "the trace series is not available with partition blocks of two or more rows");
    if (!h->d_tq) return fail(h, MCINV_E_STATE, "no trace weights were set (mcinv_set_trace_weights)");
    if (h->nseries < 4) return fail(h, MCINV_E_STATE, "need at least 4 sampled cycles");
    mcinv_status st = mcinv_sync(h);
    if (st != MCINV_OK) return st;
    std::vector<double> x((size_t)h->nseries);
    CUDA_TRY(h, cudaMemcpy(x.data(), h->d_series, x.size() * sizeof(double), cudaMemcpyDeviceToHost));
    double m, v, e, s2;
    geyer(x, &m, &v, &e, &s2);
    if (mean) *mean = m;
    if (var) *var = v;
    if (ess) *ess = e;
    if (se) *se = s2;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_trace_series(mcinv_t h, double *out, int64_t capacity, int64_t *length)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (h->nent) return fail(h, MCINV_E_UNSUPPORTED, "the trace series is not available with partition blocks of two or more rows");
    mcinv_status st = mcinv_sync(h);
    if (st != MCINV_OK) return st;
    if (length) *length = h->nseries;
    if (out && capacity > 0 && h->nseries > 0)
        CUDA_TRY(h, cudaMemcpy(out, h->d_series, (size_t)std::min(capacity, h->nseries) * sizeof(double), cudaMemcpyDeviceToHost));
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_sample_until(mcinv_t h, double rel_tol, int64_t check_every, int64_t max_cycles,
                                           int64_t *cycles_out)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (h->nent) return fail(h, MCINV_E_UNSUPPORTED, "the trace series is not available with partition blocks of two or more rows");
    if (!(rel_tol > 0.0) || check_every < 4 || max_cycles < check_every) return fail(h, MCINV_E_ARG, "bad stop-rule arguments");
    if (!h->d_tq) return fail(h, MCINV_E_STATE, "the stop rule needs trace weights (mcinv_set_trace_weights)");
    int64_t done = 0;
    for (;;) {
        mcinv_status st = mcinv_sample(h, check_every);
        if (st != MCINV_OK) return st;
        done += check_every;
        double m, v, e, se;
        st = mcinv_trace_mc_error(h, &m, &v, &e, &se);
        if (st != MCINV_OK) return st;
        if (se < rel_tol * std::fabs(m) || done + check_every > max_cycles) break;
    }
    if (cycles_out) *cycles_out = done;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_get_state(mcinv_t h, int64_t chain0, int64_t nchains, double *z, double *w, int64_t *cycle)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (chain0 < 0 || nchains < 0 || chain0 + nchains > h->K) return fail(h, MCINV_E_ARG, "chain range out of bounds");
    mcinv_status st = mcinv_sync(h);
    if (st != MCINV_OK && st != MCINV_E_DIVERGED) return st;
    const int NV = h->cplx ? 2 : 1;
    const size_t esz = NV * sizeof(float);
    std::vector<float> tmp((size_t)h->n * nchains * NV);
    double *dst[2] = {z, w};
    CUDA_TRY(h, ensure_canonical(h));
    void *src[2] = {h->d_z[h->cur], h->d_w[h->cur]};
    for (int v = 0; v < 2; ++v) {
        if (!dst[v] || nchains == 0) continue;
        CUDA_TRY(h, cudaMemcpy2DAsync(tmp.data(), nchains * esz, (char *)src[v] + chain0 * esz, h->K * esz,
                                      nchains * esz, h->n, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        for (size_t k = 0; k < tmp.size(); ++k) dst[v][k] = (double)tmp[k];
        if (!h->ord.empty()) unpermute_rows(h, dst[v], (size_t)nchains * NV);
        if (h->nent) partition_state(h, dst[v], (size_t)nchains * NV, v == 1, true);
    }
    if (cycle) *cycle = h->cycle;
    return st;
}

extern "C" mcinv_status mcinv_reset_estimates(mcinv_t h)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    const int NV = h->cplx ? 2 : 1;
    const size_t esz = NV * sizeof(float);
    if (h->d_diag_part) {
        CUDA_TRY(h, cudaMemsetAsync(h->d_diag_part, 0, (size_t)h->units * h->n * esz, h->stream));
        CUDA_TRY(h, cudaMemsetAsync(h->d_diag_acc, 0, (size_t)h->G * h->n * NV * sizeof(double), h->stream));
    }
    if (h->nR) {
        const size_t elems = (size_t)h->nR * h->nS * NV;
        CUDA_TRY(h, cudaMemsetAsync(h->d_blk, 0, elems * sizeof(float), h->stream));
        CUDA_TRY(h, cudaMemsetAsync(h->d_bsum, 0, elems * sizeof(double), h->stream));
        CUDA_TRY(h, cudaMemsetAsync(h->d_bsq, 0, elems * sizeof(double), h->stream));
    }
    if (h->d_pacc)
        CUDA_TRY(h, cudaMemsetAsync(h->d_pacc, 0, (size_t)h->G * h->nent * NV * sizeof(double), h->stream));
    h->samples = 0;
    h->block_batches = 0;
    h->block_cycles = 0;
    h->nseries = 0;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_set_state(mcinv_t h, const double *z, const double *w, int64_t cycle)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if (!z || !w || cycle < 0) return fail(h, MCINV_E_ARG, "bad state arguments");
    mcinv_status st = mcinv_sync(h);
    if (st != MCINV_OK && st != MCINV_E_DIVERGED) return st;
    const int NV = h->cplx ? 2 : 1;
    const size_t count = (size_t)h->n * h->K * NV;
    std::vector<float> tmp(count);
    const double *srcs[2] = {z, w};
    void *dsts[2] = {h->d_z[h->cur], h->d_w[h->cur]};
    const size_t row = (size_t)h->K * NV;
    std::vector<double> part_in;
    for (int v = 0; v < 2; ++v) {
        const double *src = srcs[v];
        if (h->nent) {  // the block sweep's z, w to the sampled matrix's z~ = S z, w~ = S^H w
            part_in.assign(src, src + count);
            partition_state(h, part_in.data(), row, v == 1, false);
            src = part_in.data();
        }
        if (h->ord.empty()) {
            for (size_t k = 0; k < count; ++k) tmp[k] = (float)src[k];
        } else {
            for (int64_t r = 0; r < h->n; ++r)
                for (size_t c = 0; c < row; ++c) tmp[(size_t)r * row + c] = (float)src[(size_t)h->ord[r] * row + c];
        }
        CUDA_TRY(h, cudaMemcpyAsync(dsts[v], tmp.data(), count * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    h->canon_ok = true;  // the pair layout (if any) is stale now
    h->pair_ok = false;
    h->cycle = cycle;
    return mcinv_reset_estimates(h);
}

extern "C" mcinv_status mcinv_info(mcinv_t h, mcinv_info_t *info)
{
    if (!h || !info) return fail(h, MCINV_E_ARG, "NULL argument");
    info->n = h->n; info->nnz = h->nnz; info->K = h->K;
    info->is_complex = h->cplx; info->chains_per_cta = h->W; info->threads_per_cta = h->threads;
    info->ctas_per_slice = h->Q; info->chains_per_lane = h->V;
    info->slices = h->slices; info->groups = h->G; info->levels = h->nlev;
    info->batch_cycles = h->B; info->acc = h->acc;
    info->cycle = h->cycle; info->samples = h->samples; info->block_batches = h->block_batches;
    info->kernel_launches = h->launches; info->device_bytes = h->bytes;
    info->sweep_kernel = h->grid ? (h->gwave ? 6 : h->gtile ? 5 : h->gbulk ? (h->gpair ? 4 : 3) : 2) : h->staged ? 1 : 0;
    info->grid_ctas = h->grid ? h->gctas : 0;
    return MCINV_OK;
}

static mcinv_status prof_collect(mcinv_ctx *h)
{
    if (h->ev_used == 0) return MCINV_OK;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k < h->ev_used; ++k) {
        float ms = 0.f;
        CUDA_TRY(h, cudaEventElapsedTime(&ms, h->ev_pool[k].first, h->ev_pool[k].second));
        h->prof_ms[h->ev_kind[k]] += ms;
        h->prof_launches[h->ev_kind[k]]++;
    }
    h->ev_used = 0;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_profile(mcinv_t h, int enable)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    mcinv_status st = prof_collect(h);
    if (st != MCINV_OK) return st;
    if (enable) {
        for (int k = 0; k < MCINV_KERNEL_CLASSES; ++k) { h->prof_ms[k] = 0.0; h->prof_launches[k] = 0; }
    }
    h->profiling = enable != 0;
    return MCINV_OK;
}

extern "C" mcinv_status mcinv_profile_read(mcinv_t h, mcinv_kernel kernel, int64_t *launches, double *ms)
{
    if (!h) return fail(nullptr, MCINV_E_ARG, "NULL handle");
    if ((int)kernel < 0 || (int)kernel >= MCINV_KERNEL_CLASSES) return fail(h, MCINV_E_ARG, "bad kernel class");
    mcinv_status st = prof_collect(h);
    if (st != MCINV_OK) return st;
    if (launches) *launches = h->prof_launches[kernel];
    if (ms) *ms = h->prof_ms[kernel];
    return MCINV_OK;
}

extern "C" void mcinv_destroy(mcinv_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto &e : h->ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    if (h->d_series) cudaFree(h->d_series);
    if (h->gemm) tc_gemm_plan_destroy(h->gemm);
    for (void *p : h->allocs) cudaFree(p);
    delete h;
}

extern "C" const char *mcinv_last_error(mcinv_t h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

extern "C" mcinv_status mcinv_selftest_tc_gemm(int64_t M, int64_t N, int64_t inner, const uint16_t *A,
                                               const uint16_t *B, float *D)
{
    if (M <= 0 || N <= 0 || inner <= 0 || !A || !B || !D) return fail(nullptr, MCINV_E_ARG, "bad self-test arguments");
    const size_t ld = (size_t)((inner + 63) / 64 * 64);
    const size_t ar = (size_t)((M + 127) / 128 * 128), br = (size_t)((N + 255) / 256 * 256);
    uint16_t *dA = nullptr, *dB = nullptr;
    float *dD = nullptr;
    int *dS = nullptr;
    mcinv_status st = MCINV_OK;
    std::string why;
    TcGemmPlan *plan = nullptr;
    int status = 0;
    auto chk = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == MCINV_OK) st = fail(nullptr, MCINV_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
        return e == cudaSuccess;
    };
    if (chk(cudaMalloc(&dA, ar * ld * 2), "malloc A") && chk(cudaMalloc(&dB, br * ld * 2), "malloc B") &&
        chk(cudaMalloc(&dD, (size_t)M * N * 4), "malloc D") && chk(cudaMalloc(&dS, sizeof(int)), "malloc status") &&
        chk(cudaMemset(dA, 0, ar * ld * 2), "memset") && chk(cudaMemset(dB, 0, br * ld * 2), "memset") &&
        chk(cudaMemset(dS, 0, sizeof(int)), "memset") &&
        chk(cudaMemcpy2D(dA, ld * 2, A, inner * 2, inner * 2, M, cudaMemcpyHostToDevice), "copy A") &&
        chk(cudaMemcpy2D(dB, ld * 2, B, inner * 2, inner * 2, N, cudaMemcpyHostToDevice), "copy B")) {
        plan = tc_gemm_plan_create(dA, ar, dB, br, (long long)ld, dD, M, N, &why);
        if (!plan) st = fail(nullptr, MCINV_E_UNSUPPORTED, "%s", why.c_str());
        else if (chk(tc_gemm_run(plan, (long long)ld, dS, nullptr), "launch") && chk(cudaDeviceSynchronize(), "sync") &&
                 chk(cudaMemcpy(D, dD, (size_t)M * N * 4, cudaMemcpyDeviceToHost), "copy D") &&
                 chk(cudaMemcpy(&status, dS, sizeof(int), cudaMemcpyDeviceToHost), "copy status") && status)
            st = fail(nullptr, MCINV_E_TIMEOUT, "tensor-core contraction timed out");
    }
    tc_gemm_plan_destroy(plan);
    cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(dS);
    return st;
}
