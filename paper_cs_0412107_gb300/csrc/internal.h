// internal.h -- declarations shared by the translation units of libmcinv.
// Not part of the public ABI (that is include/mcinv.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mcinv {

// One off-diagonal CSR entry as the sweep reads it: a single aligned load.
struct EntR {
    int col;
    float val;
};
struct __align__(16) EntC {
    int col;
    float re, im;
    int pad;
};

// Per-row constants of Eqs. 4/5 in the sweep precision (formed in FP64).
struct __align__(16) CstR {
    float alpha, beta, inv_d, pad;  // 1/sqrt(c_ii), 1/conj(sqrt(c_ii)), 1/c_ii
};
struct __align__(16) CstC {
    float2 alpha, beta, inv_d, pad;
};

// The sweep reads the matrix as a stream of chunks, in "position" order: the
// rows of Gauss-Seidel dependency level 0, then level 1, ... (rows of one
// level do not read each other through C or C^dagger, so a CTA may update
// them concurrently and get exactly the in-place ascending-row result of
// Eqs. 4/5).  A chunk is a run of positions inside one level whose data fit
// one shared-memory buffer; its blob is
//   RowMeta[items + 1] | Cst[rows] | C entries | C^dagger entries
// (each part 16-byte aligned) and is copied to shared memory in one bulk copy.
//
// A chunk's rows are cut into work items.  A row with more than SPLIT_ENTRIES
// off-diagonal entries in C or in C^dagger becomes P = 2 or 4 items, each a
// contiguous slice of both entry lists (at most P = 4; a slice may be empty);
// the slices' partial sums are added in piece order, ((p0 + p1) + p2) + p3,
// whichever lanes compute them, so every launch shape gives the same bits.
// Items of one row are consecutive and start at a multiple of P inside the
// chunk (rows are ordered by decreasing P within a level).
constexpr int SPLIT_ENTRIES = 8;
struct RowMeta {
    int row;   // row index i of C
    int zoff;  // first C entry of the item within the chunk's C entries (item `items`: end)
    int woff;  // same for C^dagger
    int info;  // bits 0-1: the item's piece k; bits 2-3: log2 P; bits 4-31: the row's index in the chunk
};

// The same rows for the grid-wide sweep (sweep_grid.cu), flat and by position:
// row p's C entries are zent[zb .. next.zb), its C^dagger entries went[wb ..
// next.wb) (the same order as in its chunk), and info packs log2 P (bits 0-1,
// the pieces the chunk stream cuts the row into), the C entry count (bits
// 2-16) and the C^dagger entry count (bits 17-31).  Record n is a sentinel.
struct __align__(16) GridRow {
    int row, zb, wb, info;
};
constexpr int GRID_DEG_MAX = (1 << 15) - 1;

struct ChunkDesc {
    long long off;  // byte offset of the blob in the stream (16-byte aligned)
    int bytes;      // blob size (multiple of 16)
    int rows;       // positions pb .. pb + rows - 1
    int pb;
    int cst_off, zent_off, went_off;  // byte offsets of the parts within the blob
    int flags;      // CHUNK_LEVEL_END: the next chunk starts a new level; CHUNK_SPLIT
    int items;      // work items (rows + the extra pieces of split rows)
};
constexpr int CHUNK_LEVEL_END = 1;
constexpr int CHUNK_SPLIT = 2;  // the chunk holds split rows (some item with P > 1)

// Arguments of the coupled sweep.
struct SweepArgs {
    int n, K, nw;              // nw = ceil(K/32) noise words per position
    int nchunks, blob_max;     // chunks per cycle; bytes of one shared-memory buffer
    const uint8_t *stream;     // chunk blobs
    const ChunkDesc *chunks;
    const uint32_t *noise;     // [ncyc][nw][n] by position: Z2 sign bits (bit c%32 of word c/32), 1 -> phi = -1;
                               // null: phi = 0 (noise-free Gauss-Seidel, Eq. 12)
    void *z[2], *w[2];         // double-buffered chain state [n][K] by row (float / float2)
    int cur;                   // buffer holding the state before the first cycle of this launch
    int ncyc;                  // cycles this launch runs
    // running sums of z_i conj(w_i) over "units" of seg lanes (seg * V chains):
    // [units][n] by position, read-modify-write by the one lane that owns it; null: off
    void *diag_part;
    int seg;
    // BF16 shadows of rows in R (z) and S (w) for the tensor-core block contraction
    const int *rpos, *spos;    // [n] by position -> index in R / S, or -1; null disables shadows
    uint16_t *zsh, *wsh;
    long long ldsh;            // elements per shadow row (batch_cycles * kp)
    long long kp;              // elements per cycle block: K (x2 complex) rounded up to 64
    int cyc0_in_batch;         // shadow column block of this launch's first cycle
    int ctas_per_slice;        // Q: CTAs (one thread-block cluster) per chain slice
    // per-cycle trace series (Geyer's Monte Carlo error): q_i by position, and
    // per-(cycle, CTA, warp) partial sums of q_i Re(z_i conj(w_i)); null: off
    const float *tq;
    float *tpart;
    int *status;               // bit 0: a chain diverged; bit 2: a staging wait expired
    int test_expire;           // the wavefront sweep's first stage is never copied (its waits expire)
};

// Launchers (sweep.cu)
// noise plane by position: pos[row] gives the position of each row
cudaError_t launch_noise(uint64_t seed, uint32_t matrix, uint64_t chain_base, int K, int n,
                         uint32_t cycle0, int ncyc, const int *pos, uint32_t *out, cudaStream_t s);
// per-row constants written into the chunk stream at stream + cst_at[p] (by position)
cudaError_t launch_constants(int n, const double *diag, int cplx, uint8_t *stream,
                             const long long *cst_at, int *bad, cudaStream_t s);
// slices CTAs of lanes_per_row x chains_per_lane chains each; chains_per_lane
// is 1 or the vector width (4 real, 2 complex) and then divides K.
cudaError_t launch_sweep(const SweepArgs &a, int cplx, int lanes_per_row, int chains_per_lane,
                         int slices, int threads, cudaStream_t s);

// Clusters of q CTAs of the sweep that can be resident at once (0: not launchable).
int max_active_clusters(int cplx, int lanes_per_row, int chains_per_lane, int threads, int q,
                        int blob_max);

// accumulate.cu
// acc[g][perm[p]] += sum of the group's units' part[u][p]; part is cleared
cudaError_t launch_diag_fold(int cplx, int n, int units, int G, const int *perm, void *diag_part,
                             double *acc, cudaStream_t s);
cudaError_t launch_block_simt(int cplx, int K, const void *z, const void *w, const int *R, int nR,
                              const int *S, int nS, float *blk, cudaStream_t s);
cudaError_t launch_block_fold(int cplx, long long elems, double scale_sq, float *blk,
                              double *sum, double *sq, int zero_blk, cudaStream_t s);
cudaError_t launch_diag_estimate(int cplx, int n, int G, const double *counts, double samples,
                                 const double *acc, double *mean, double *se, cudaStream_t s);
cudaError_t launch_trace_estimate(int cplx, int n, int G, const double *counts, double samples,
                                  const double *acc, const double *q, double *out, cudaStream_t s);
cudaError_t launch_block_estimate(int cplx, long long elems, double K, double T, double nb,
                                  const double *sum, const double *sq, double *mean, double *se,
                                  cudaStream_t s);

// series[first + c] = (sum over CTAs and warps of tpart[c][cta][warp]) / K, FP64, fixed order
cudaError_t launch_series_fold(int ncyc, int ctas, int warps, const float *tpart, double K, double *series,
                               long long first, cudaStream_t s);

// coupling burn-in helpers (accumulate.cu)
cudaError_t launch_maxabs2(int cplx, int n, const void *a, const void *b, unsigned *out, cudaStream_t s);
cudaError_t launch_iota1(int cplx, int n, void *d, cudaStream_t s);
// The staged sweep (sweep_staged.cu): real matrices, 4 chains per lane, 4 or 8 lanes
// per row, K a multiple of the slice; a producer warp stages the gathers in shared memory.
bool staged_supported(int cplx, int lanes_per_row, int chains_per_lane, int64_t K, int blob_max);
cudaError_t launch_sweep_staged(const SweepArgs &a, int lanes_per_row, int slices, cudaStream_t s);
int staged_threads();
// The grid-wide sweep (sweep_grid.cu): one cooperative launch of grid_ctas()
// CTAs; a warp takes a (row, 32 x V chain) item, all CTAs share every dependency
// level, a grid barrier ends each level.  Real matrices with 4 chains per lane
// or complex with 2, K a multiple of that.  The two state buffers of z (and of
// w) are one allocation: z[1] = z[0] + n K / V vectors.
struct GridArgs {
    const GridRow *rows;       // [n + 1] by position; .row holds i * K / V (the row's first vector)
    const void *zent[2];       // EntR / EntC of C by position, for the cycles that start from state
    const void *went[2];       // buffer 0 / 1; .col holds the gathered vector's index from z[0] / w[0]
    const void *cst;           // CstR / CstC by position
    const int *lev_ptr;        // [nlev + 1]: first position of each level
    int nlev;
    int nblk;                  // chain blocks per row: ceil(K / (32 V))
    int kv;                    // 16-byte vectors per row of z (or of w): K / V
    uint32_t nkv;              // vectors per state buffer: n K / V (pair layout: n x 2 x 32 nblk)
    int pair;                  // bulk staging on the pair layout (a.z[0]: its two buffers)
    unsigned *bar;             // barrier arrivals (zeroed by the launcher before each launch)
};
// threads: 384 or 512 with the gathers in registers; bulk: the warps stage their
// gathers in shared memory with bulk copies, 384 or 512 threads with 512-byte
// segments, 192 with 1 KB or 96 with 2 KB (a warp's chain block is 1, 2 or 4 x 32
// vectors); on the pair layout (GridArgs.pair, pair = true) 512 threads with 1 KB
// segments (z and w of a 32-vector block) or 384 or 256 with 2 KB (two blocks).
// One CTA per SM.
bool grid_supported(int cplx, int chains_per_lane, int64_t K, int threads, bool bulk);
int grid_ctas(int cplx, int threads, bool bulk, bool pair = false);  // CTAs resident at once on the device; 0: not launchable
cudaError_t launch_sweep_grid(const SweepArgs &a, const GridArgs &g, int cplx, int ctas, int threads, bool bulk,
                              cudaStream_t s);
// The pair layout of the chain state for the grid-wide bulk sweep of structurally
// symmetric matrices: row j, chain block k (32 vectors of 16 bytes) holds the
// block's z vectors, then the same chains' w vectors (rows of 64 ceil(kv / 32)
// vectors).  unpack = 0: canonical z, w ([n][kv] vectors each) -> x; 1: back.
cudaError_t launch_pair_pack(const void *z, const void *w, void *x, long long n, int kv, int unpack, cudaStream_t s);
// Block partition (Sec. 4): for every pair (r, s) of rows of one diagonal block
// (entry e: rows ent_r[e], ent_s[e] of the state) and every chain group g (chains
// gch[g] .. gch[g+1]-1): acc[g][e] += sum over the group's chains of z_r conj(w_s), FP64.
cudaError_t launch_pblock_acc(int cplx, int nent, const int *ent_r, const int *ent_s, int K, int G, const int *gch,
                              const void *z, const void *w, double *acc, cudaStream_t s);
// dst[idx[k]] = val[k], k < count
cudaError_t launch_scatter(int count, const long long *idx, const double *val, double *dst, cudaStream_t s);

}  // namespace mcinv
