// spectral.cuh -- the spectral matrix-free product (sparse real space over
// cell lists, reciprocal sum on a mesh): plan state and launchers.
#pragma once

#include "bd_internal.cuh"
#include "fft.cuh"

namespace bd {

constexpr int kMeshTile = 8;    // mesh tile edge of the spreading kernel

struct PmeState {
    int K, p;                     // mesh points per edge, B-spline order
    int nc;                       // cells per edge of the real-space cell list
    int span;                     // neighbour cells searched on each side (0: one cell)
    long ncell;                   // nc^3
    long K3, Kh;                  // K^3 and K * K * (K/2 + 1)
    int mcap;                     // columns the grids hold (max_rhs + 3)
    int *d_cell_of;               // [n] cell of each bead
    int *d_cell_count;            // [ncell] beads per cell, then scatter cursors
    int *d_cell_start;            // [ncell + 1] exclusive prefix sums
    int *d_cell_beads;            // [n] bead indices grouped by cell, ascending in a cell
    int *d_cell_tmp;              // [n] the same before the in-cell sort
    // real-space neighbour table: rows are the beads in cell order (row r is
    // bead cell_beads[r]); a row's entries are the rows within r_c (itself
    // included) and the six components of their 3x3 block, stored by
    // component ([6][pair_cap])
    int *d_row_start;             // [n + 1] first entry of each row (counts before the scan)
    void *d_rowpos;               // [n] positions in row order, 32 bytes a row
    int *d_nbr;                   // [pair_cap] neighbour rows
    int *d_prow;                  // [pair_cap] the entry's own row (-1: padding)
    void *d_tens;                 // [6][pair_cap] xx, xy, xz, yy, yz, zz (working precision)
    long pair_cap, npair;         // entries allocated, entries in use
    void *d_xrows;                // operand rows in cell order, by column chunk
    long xrows_len;               // elements allocated for d_xrows
    long long *h_npair;           // pinned host word for the entry count
    void *d_infl;                 // [Kh][6] influence function G(m)|b(m)|^2 (working precision)
    // mesh tiles of kMeshTile^3 points: beads binned by the tile holding their
    // spline base index floor(u) (ascending bead index inside a bin)
    int tpd;                      // tiles per edge, K / kMeshTile
    long ntile;                   // tpd^3
    int *d_tile_of;               // [n]
    int *d_tile_count;            // [ntile]
    int *d_tile_start;            // [ntile + 1]
    int *d_tile_beads;            // [n]
    int *d_bfl;                   // [n][3] floor(u_d) mod K of each bead
    void *d_bw;                   // [n][3][p] spline weights M_p(u_d - floor(u_d) + j)
    void *d_qreal;                // [3 mcap][K3] real mesh (working precision)
    void *d_qhat;                 // [3 mcap][Kh] complex mesh
    FftPlan fft;                  // the mesh transforms (fft.cu)
};

// the spectral product needs pme_grid > 0 in the plan parameters; creates the
// state (allocations, influence function, cell geometry)
bd_status spectral_init(Plan &P);
void spectral_free(Plan &P);
// cell list, neighbour table, mesh-tile bins and spline weights of the
// current positions (after the wrapped positions are built); synchronises the
// stream once to size the neighbour table
bd_status spectral_tables(Plan &P, cudaStream_t s);
// Y = D(R) X: real space over the cell list plus the mesh reciprocal sum
bd_status launch_apply_spectral(Plan &P, const double *X, int m, double *Y, cudaStream_t s);

// real-space part (ewald_build.cu): the neighbour table of the current cell
// list, and Y = (real-space part of D) X over it
bd_status build_real_pairs(Plan &P, cudaStream_t s);
bd_status launch_real_pairs(Plan &P, const double *X, int m, double *Y, cudaStream_t s);
// elements of the operand-row buffer for products of up to mcap columns
long real_pairs_rows_len(int n, int mcap, bool dbl);
// exclusive prefix sum of len counts into start[0 .. len] (count and start
// may be the same array; count is overwritten)
void launch_scan_counts(int *count, long len, int *start, cudaStream_t s);
// column chunk of the real-space product per working precision
constexpr int kPairCols32 = 9;
constexpr int kPairCols64 = 6;

}  // namespace bd
