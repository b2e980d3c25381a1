// spectral.cuh -- the spectral matrix-free product (sparse real space over
// cell lists, reciprocal sum on a mesh): plan state and launchers.
#pragma once
#include <cufft.h>

#include "bd_internal.cuh"

namespace bd {

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
    double *d_rpart;              // [2 span + 1][3N x mcap] real-space partials per neighbour slab
    void *d_infl;                 // [Kh][6] influence function G(m)|b(m)|^2 (working precision)
    unsigned long long *d_qfix;   // [3 mcap][K3] spread in 64-bit fixed point
    void *d_qreal;                // [3 mcap][K3] real mesh (working precision)
    void *d_qhat;                 // [3 mcap][Kh] complex mesh
    unsigned long long *d_xmax;   // [4] max |x| of the operand, fixed-point scale, its inverse
    cufftHandle fwd, inv;         // batched R2C / C2R plans for plan_m columns
    int plan_m;                   // 0: no cuFFT plans yet
};

// the spectral product needs pme_grid > 0 in the plan parameters; creates the
// state (allocations, influence function, cell geometry)
bd_status spectral_init(Plan &P);
void spectral_free(Plan &P);
// cell list of the current positions (after the wrapped positions are built)
void spectral_tables(Plan &P, cudaStream_t s);
// Y = D(R) X: real space over the cell list plus the mesh reciprocal sum
bd_status launch_apply_spectral(Plan &P, const double *X, int m, double *Y, cudaStream_t s);

// real-space part over the cell list (ewald_build.cu)
bd_status launch_real_cells(Plan &P, const double *X, int m, double *Y, cudaStream_t s);

}  // namespace bd
