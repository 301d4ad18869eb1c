// sweep_tiled.h -- the tile-staged coupled sweep (sweep_tiled.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace mcinv {

// Staged rows a tile may name: two buffers of this many 1 KB slabs, with the tiles'
// row records and constants beside them, fit a CTA.
constexpr int TILE_CAP = 100;
// Positions a tile may hold (tiles of 64, 32, 16 or 8).
constexpr int TILE_MAX_ROWS = 64;

// The tiled form of a structurally symmetric matrix (row i of C and of C^dagger
// name the same columns in the same order).  The positions of every dependency
// level are cut into tiles of at most `tile` consecutive positions; a tile's rows
// name at most TILE_CAP distinct neighbours (row j, and whether the row reads
// this cycle's buffer, j < i, or last cycle's, j > i), its staged list, kept as
// runs of consecutive rows read from one buffer.
//
// The tiled sweep keeps the state in the block-major pair layout: chain block b
// (32 vectors of 16 bytes), row j holds the block's z vectors then its w vectors
// at vector b n 64 + j 64, so a run of consecutive rows of one block is one
// contiguous copy.
// One position's row in the tiled form, everything a row reads to sum its entries
// in one record of independent loads: its first vector (i x 64, block-major), its
// entry count d, the entries' slots in the tile's stage, and the coefficients of
// C (z side) and of C^dagger (w side), entry u at index u (u >= d: zero).
template <bool CPLX> struct TileRow;
template <> struct __align__(16) TileRow<false> {
    int iv, d, pad0, pad1;
    uint16_t slot[8];
    float zc[8], wc[8];
};
template <> struct __align__(16) TileRow<true> {
    int iv, d, pad0, pad1;
    uint16_t slot[8];
    float2 zc[8], wc[8];
};
static_assert(sizeof(TileRow<false>) == 96 && sizeof(TileRow<true>) == 160, "whole 16-byte loads");

struct TileArgs {
    const void *trow;         // [n] TileRow by position
    const int *tile_ptr;      // [ntiles + 1]: first position of each tile
    const int *tile_slots;    // [ntiles]: rows the tile stages
    const int *lev_tile;      // [nlev + 1]: first tile of each level
    const int *run_ptr;       // [ntiles + 1]: first run of each tile
    const int *run_row;       // per run: its first row j, bit 31 set when read from this cycle's buffer
    const int *run_len;       // per run: rows (bits 0-15) and first slot in the tile's stage (bits 16-31)
};

// Host: the tiled form from the flat form (rows by position with their row index
// i in .row, entries with the neighbour's row index j in .col), or false when
// some row is cut into pieces or some tile would stage more than TILE_CAP
// neighbours.  Tiles of `tile` positions (the caller tries 64, 32, 16, 8).
bool build_tiles(const std::vector<GridRow> &rows, const std::vector<uint8_t> &zent, size_t ent_bytes,
                 const std::vector<int32_t> &lev_ptr, int tile, std::vector<int> &tile_ptr,
                 std::vector<int> &tile_slots, std::vector<int> &lev_tile, std::vector<int> &run_ptr,
                 std::vector<int> &run_row, std::vector<int> &run_len, std::vector<uint16_t> &slot);

// Host: the TileRow records (bytes, n of them) from the flat form and the slots
// build_tiles gave each entry.
std::vector<uint8_t> build_tile_rows(const std::vector<GridRow> &rows, const std::vector<uint8_t> &zent,
                                     const std::vector<uint8_t> &went, const std::vector<uint16_t> &slot, int cplx);

// The state between the canonical layout (z, w: [n][kv] vectors each) and the
// block-major pair layout x with blocks of bw vectors (a power of two up to 32: block
// b, row j at vector (b n + j) 2 bw: the block's z vectors, then its w vectors; the
// tiled sweep's bw = 32, the wavefront sweep's its slice width); unpack = 1: x -> z, w.
cudaError_t launch_tile_pack(const void *z, const void *w, void *x, long long n, int kv, int unpack, cudaStream_t s,
                             int bw = 32);

// CTAs of the tiled sweep resident at once on the device (one per SM); 0: not launchable.
int tiled_ctas(int cplx);
// One launch of a.ncyc cycles on the block-major pair layout (a.z[0]: its two
// buffers; g: the pair form's entries, cycle count and levels; t: the tiled form).
// Cooperative: a grid barrier ends each level.
cudaError_t launch_sweep_tiled(const SweepArgs &a, const GridArgs &g, const TileArgs &t, int cplx, int ctas,
                               cudaStream_t s);

}  // namespace mcinv
