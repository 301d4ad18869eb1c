// sweep_wave.h -- the chain-sliced wavefront sweep of a two-colour banded matrix
// (sweep_wave.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace mcinv {

// A row of the wavefront form: its entry count d, each entry's code (ring distance of
// the neighbour's chunk + B, shifted left by 10, or'd with the neighbour's index in its
// chunk), the coefficients of C (z side) and of C^dagger (w side), entry u at index u;
// D = 4 when every row has four entries, else 8.
template <bool CPLX, int D> struct WaveRow;
template <> struct __align__(16) WaveRow<true, 4> {
    int d;
    uint16_t code[4];
    int pad;
    float2 zc[4], wc[4];
};
template <> struct __align__(16) WaveRow<true, 8> {
    int d, pad0, pad1, pad2;
    uint16_t code[8];
    float2 zc[8], wc[8];
};
template <> struct __align__(16) WaveRow<false, 4> {
    int d;
    uint16_t code[4];
    int pad;
    float zc[4], wc[4];
};
template <> struct __align__(16) WaveRow<false, 8> {
    int d, pad0, pad1, pad2;
    uint16_t code[8];
    float zc[8], wc[8];
};
static_assert(sizeof(WaveRow<true, 4>) == 80 && sizeof(WaveRow<true, 8>) == 160 && sizeof(WaveRow<false, 4>) == 48 &&
                  sizeof(WaveRow<false, 8>) == 96,
              "whole 16-byte loads");

// The wavefront form of a matrix in the colour order with two dependency levels
// of h positions each (level 0, "red": positions 0 .. h-1; level 1, "black":
// h .. 2h-1; position = row).  Each level is cut into m = h / S chunks of S
// consecutive positions, and every row's neighbours lie in the other level's
// chunks within ring distance B of its own chunk index (mod m): a lattice in the
// colour order, whose red half-rows only touch the black half-rows next to them.
struct WaveForm {
    int S = 0, B = 0, m = 0, h = 0;
    int sv = 0;                  // 16-byte vectors of one chain slice (4, 8 or 16): one CTA a slice
    int D = 0;                   // entries a row record holds (4 or 8)
    bool exact = false;          // every row has D entries
    std::vector<uint8_t> trow;   // WaveRow<cplx, D> records by position
};

struct WaveArgs {
    const void *trow;   // [n] WaveRow by position
    const void *cst;    // [n] Cst by position
    int h, S, B, m;     // positions per level, chunk positions, band in chunks, chunks per level
    int sv;             // vectors per chain slice
    int D;              // entries of a row record
    int exact;          // every row has D entries
    int nb, nr;         // black and red ring slots (2B + 2 each)
    uint32_t nkv;       // vectors of one state buffer (the second starts there)
};

// Host: the wavefront form from the flat form (rows by position, entries with the
// neighbour's row index in .col), or false when C is not a two-level banded matrix
// of this kind whose window fits a CTA's shared memory.  kv: vectors per row of z;
// sms: the device's SMs (the slice width is chosen to give about one CTA an SM).
bool build_wave(const std::vector<GridRow> &rows, const std::vector<uint8_t> &zent, const std::vector<uint8_t> &went,
                size_t ent_bytes, const std::vector<int32_t> &lev_ptr, int cplx, int kv, int sms, WaveForm &out);

// Bytes of dynamic shared memory of one CTA (seg: vectors of one diagonal-partial unit;
// 0: no diagonal partials).
size_t wave_smem(const WaveArgs &g, int cplx, int seg);

// One launch of a.ncyc cycles on the sliced layout (a.z[0]: its two buffers; slice s,
// position p at vector (s n + p) 2 sv: the slice's z vectors, then its w vectors).
// One CTA per slice, independent of one another (no grid barrier).
cudaError_t launch_sweep_wave(const SweepArgs &a, const WaveArgs &g, int cplx, cudaStream_t s);
int wave_ctas(int kv, int sv);

}  // namespace mcinv
