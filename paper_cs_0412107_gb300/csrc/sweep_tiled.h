// sweep_tiled.h -- the tile-staged coupled sweep (sweep_tiled.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace mcinv {

// Staged positions a tile may name: two buffers of this many 1 KB slabs fit a CTA.
constexpr int TILE_CAP = 104;

// The tiled form of a structurally symmetric matrix (row i of C and of C^dagger
// name the same columns in the same order).  The positions of every dependency
// level are cut into tiles of at most `tile` consecutive positions; a tile's rows
// name at most TILE_CAP distinct neighbours (row j, and whether the row reads
// this cycle's buffer, j < i, or last cycle's, j > i), its staged list.
struct TileArgs {
    const int *tile_ptr;      // [ntiles + 1]: first position of each tile
    const int *lev_tile;      // [nlev + 1]: first tile of each level
    const int *stage_ptr;     // [ntiles + 1]: first staged entry of each tile
    const int *stage_row;     // staged neighbours: row j, bit 31 set when read from this cycle's buffer
    const uint16_t *slot;     // by C entry index (flat form): the entry's neighbour in its tile's staged list
};

// Host: the tiled form from the flat form (rows by position with their row index
// i in .row, entries with the neighbour's row index j in .col), or false when
// some row is cut into pieces or some tile would stage more than TILE_CAP
// neighbours.  Tiles of `tile` positions (the caller tries 64, 32, 16, 8).
bool build_tiles(const std::vector<GridRow> &rows, const std::vector<uint8_t> &zent, size_t ent_bytes,
                 const std::vector<int32_t> &lev_ptr, int tile, std::vector<int> &tile_ptr, std::vector<int> &lev_tile,
                 std::vector<int> &stage_ptr, std::vector<int> &stage_row, std::vector<uint16_t> &slot);

// CTAs of the tiled sweep resident at once on the device (one per SM); 0: not launchable.
int tiled_ctas(int cplx);
// One launch of a.ncyc cycles on the pair layout (a.z[0]: its two buffers; g: the
// pair form of the rows and entries).  Cooperative: a grid barrier ends each level.
cudaError_t launch_sweep_tiled(const SweepArgs &a, const GridArgs &g, const TileArgs &t, int cplx, int ctas,
                               cudaStream_t s);

}  // namespace mcinv
