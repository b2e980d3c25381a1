// rows_gemm.cuh -- launch shape 5 of the mixed products (row-streamed, few
// columns) and the batched Chebyshev loop (rows_gemm.cu).
#pragma once
#include "bd_internal.cuh"

namespace bd {

constexpr int kRowsShape = 5;
constexpr int kRowsMaxCols = 8;   // columns of one row-streamed product
constexpr int kRowsMaxLoopCols = 5;   // columns of the Chebyshev loop (m <= 4 and the Lanczos vector)
// the loop's control words: grid-barrier count and generation, the Lanczos
// item count, a spare word, then one item counter per Chebyshev term
constexpr int kRowsBarWords = 4;
constexpr int kRowsBarAlloc = kRowsBarWords + kMaxCheb;

// one replica of a batched Chebyshev loop (device table entry)
struct RowsRep {
    const uint16_t *D16;         // 16-bit D (half or bfloat16 bits), row-major, ld
    long ld;
    int n3, xs;                  // 3N; stride of the FP32 operand columns
    int m, lan, is_bf16;         // Wiener columns; 1: the Lanczos vector is column m
    int item0, nitems;           // first work item of the replica in the list; its items
    const double *coef, *bounds;
    double *VA, *VB;             // recurrence buffers: V_0 in VA, V_1 in VB, then alternating
    double *dS;                  // accumulated noise (3N x m)
    float *X32[2];               // FP32 operand, [column][xs], ping-pong by term parity
    double *lq[3];               // q_{j-1}, q_j, w
    double *lab;                 // alpha [kMaxLanczos], beta [kMaxLanczos]
    double *lan_part;            // per item: q_j.w, q_{j-1}.w, w.w
    unsigned *lan_count;         // items of the current term done (self-resetting)
    int32_t *err;                // the replica's status word (BD_ERR_TIMEOUT)
};

int rows_items(int n3);
// allocate the plan's FP32 operand, item table and partials (first use)
bd_status rows_plan_init(Plan &P);
// Y = D16 X, 1 <= m <= kRowsMaxCols columns (X, Y FP64, 3N x m)
bd_status rows_apply(Plan &P, const void *D16, const double *X, int m, double *Y, cudaStream_t s);
// the replica's table entry for a Chebyshev loop on D16
RowsRep rows_rep(Plan &P, const void *D16, const double *coef, const double *bounds, int m,
                 int lan, double *dS);
// term 2's operand (V_1 and, with lan, q_j) and the table entry into *dst
void rows_cheb_prepare(Plan &P, const RowsRep &rep, RowsRep *dst, const double *V1, int lan,
                       cudaStream_t s);
// terms 2 .. nch - 1 of every replica in the table, one cooperative launch;
// lan_from >= 0: term p takes Lanczos step lan_from + p - 1
bd_status rows_cheb_launch(const RowsRep *reps, int nreps, const int *item_rep, int nitems, int cols,
                           int nch, int lan_from, unsigned *bar, int device, cudaStream_t s);

// parts of bd_step for the batch (bd_api.cu): 1 = forces .. V_1 and the
// loop's table entry in *slot (item0: the replica's first item), 2 = E_f ..
// Euler update; the plan must be step_batchable
bool step_batchable(bd_plan *plan, const bd_step_opts *o);
bd_status step_part(bd_plan *plan, double *R, void *D, const bd_step_opts *o,
                    bd_step_stats *stats, cudaStream_t s, int part, RowsRep *slot, int item0);
// after a front part: 1 if the Lanczos vector rides in the loop's products
int step_part_lag(bd_plan *plan);
// items of the plan's row-streamed products (32 rows each)
int step_part_items(bd_plan *plan);
int plan_device(bd_plan *plan);

}  // namespace bd
