// batch.cu -- many independent replicas (uneven N) advanced together.
//
// One plan per replica.  A step of the batch forks `count` branches from the
// caller's stream (one non-blocking stream per replica) and joins them back.
// Mixed plans with a few Wiener columns (max_rhs <= 4) take the row-streamed
// product shape, and their step runs in three parts: every replica's front
// (forces, D(R), bounds, the first product, V_1) on its branch; then the
// Chebyshev loops of ALL replicas in one persistent launch, a work queue over
// {replica, 64-row block} (rows_gemm.cu); then every replica's back (E_f,
// lagged bounds, Euler update) on its branch.  Otherwise each branch runs a
// whole bd_step.  From the second call on, the sequence is recorded once into
// a CUDA graph and replayed with a single cudaGraphLaunch per step.  Wiener
// increments are drawn on the device with the plan's device step counter,
// so every replay draws new noise.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bd_internal.cuh"
#include "rows_gemm.cuh"

struct bd_batch {
    int count = 0;
    std::vector<bd_plan *> plans;
    std::vector<int64_t> r_off, d_off;
    int64_t r_total = 0, d_total = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join_ev;
    cudaEvent_t fork_ev = nullptr;
    cudaStream_t origin = nullptr;   // capture origin (the legacy stream cannot capture)
    cudaGraphExec_t exec = nullptr;
    // arguments the recorded graph was made with
    double *key_R = nullptr;
    void *key_D = nullptr;
    bd_step_stats *key_stats = nullptr;
    bd_step_opts key_opts;
    int calls = 0;
    // the batched Chebyshev loop (all plans in the row-streamed shape)
    int rows = 0;                    // 1: the plans use launch shape 5
    std::vector<int> item0;          // first work item of each replica
    int nitems = 0;
    bd::RowsRep *d_reps = nullptr;   // [count] table entries, written by each front part
    int *d_items = nullptr;          // item -> replica
    unsigned *d_bar = nullptr;       // grid barrier words
    cudaEvent_t mid_ev = nullptr;    // fork of the back parts
};

using namespace bd;

static void destroy_batch(bd_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto s : b->streams) if (s) cudaStreamDestroy(s);
    for (auto e : b->join_ev) if (e) cudaEventDestroy(e);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->mid_ev) cudaEventDestroy(b->mid_ev);
    if (b->d_reps) cudaFree(b->d_reps);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_bar) cudaFree(b->d_bar);
    if (b->origin) cudaStreamDestroy(b->origin);
    for (auto p : b->plans) bd_plan_destroy(p);
    delete b;
}

extern "C" {

bd_status bd_batch_create(const bd_params *params, int32_t count, bd_batch **out_batch)
{
    if (!params || !out_batch || count < 1 || count > 4096)
        return set_error(BD_ERR_INVALID, "need params, out_batch and 1 <= count <= 4096");
    *out_batch = nullptr;
    bd_batch *b = new (std::nothrow) bd_batch();
    if (!b) return set_error(BD_ERR_OOM, "host allocation failed");
    b->count = count;
    b->plans.assign(count, nullptr);
    b->streams.assign(count, nullptr);
    b->join_ev.assign(count, nullptr);
    memset(&b->key_opts, 0, sizeof(b->key_opts));
    for (int i = 0; i < count; i++) {
        bd_status st = bd_plan_create(&params[i], &b->plans[i]);
        if (st != BD_OK) {
            destroy_batch(b);
            return st;
        }
        bd_plan_info info;
        bd_plan_query(b->plans[i], &info);
        b->r_off.push_back(b->r_total);
        b->d_off.push_back(b->d_total);
        b->r_total += info.n3;
        b->d_total += (info.d_bytes + 255) / 256 * 256;
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming) != cudaSuccess) {
            destroy_batch(b);
            return set_error(BD_ERR_CUDA, "stream/event creation failed");
        }
    }
    if (cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->mid_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) {
        destroy_batch(b);
        return set_error(BD_ERR_CUDA, "event creation failed");
    }
    // mixed replicas with few columns: the row-streamed shape and one
    // persistent Chebyshev launch for all of them
    bool rows = true;
    for (int i = 0; i < count; i++)
        rows = rows && params[i].precision != BD_FP64 && params[i].max_rhs + 4 <= kRowsMaxCols;
    if (rows) {
        for (int i = 0; i < count; i++) {
            bd_status st = bd_plan_set_shape(b->plans[i], kRowsShape);
            if (st != BD_OK) {
                destroy_batch(b);
                return st;
            }
        }
        // the item table lists the replicas with the longest rows (largest N)
        // first: items are claimed in table order, so the long ones start
        // early and the short ones fill in at the end of each term
        std::vector<int> order(count), items;
        for (int i = 0; i < count; i++) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return params[x].n_beads > params[y].n_beads; });
        b->item0.assign(count, 0);
        for (int i : order) {
            b->item0[i] = b->nitems;
            const int k = step_part_items(b->plans[i]);
            for (int t = 0; t < k; t++) items.push_back(i);
            b->nitems += k;
        }
        cudaError_t e = cudaMalloc(&b->d_reps, sizeof(RowsRep) * count);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int) * items.size());
        if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, kRowsBarAlloc * sizeof(unsigned));
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, kRowsBarAlloc * sizeof(unsigned));
        if (e != cudaSuccess) {
            cudaGetLastError();
            destroy_batch(b);
            return set_error(BD_ERR_OOM, "batch work queue: %s", cudaGetErrorString(e));
        }
        b->rows = 1;
    }
    *out_batch = b;
    return BD_OK;
}

void bd_batch_destroy(bd_batch *batch) { destroy_batch(batch); }

bd_status bd_batch_query(const bd_batch *b, int32_t index, bd_plan_info *info, int64_t *r_offset,
                         int64_t *d_offset, int64_t *r_total, int64_t *d_total)
{
    if (!b) return set_error(BD_ERR_INVALID, "NULL batch");
    if (r_total) *r_total = b->r_total;
    if (d_total) *d_total = b->d_total;
    if (index < 0) return BD_OK;
    if (index >= b->count) return set_error(BD_ERR_INVALID, "index %d >= count %d", index, b->count);
    if (info) bd_plan_query(b->plans[index], info);
    if (r_offset) *r_offset = b->r_off[index];
    if (d_offset) *d_offset = b->d_off[index];
    return BD_OK;
}

// fork from `stream`, the replicas' fronts, one launch of all their
// Chebyshev loops, the replicas' backs, join back
static bd_status batch_body_rows(bd_batch *b, double *R, void *D, const bd_step_opts *opts,
                                 bd_step_stats *stats, cudaStream_t stream)
{
    if (cudaEventRecord(b->fork_ev, stream) != cudaSuccess) return check_launch("batch fork");
    int lag = 0;
    for (int i = 0; i < b->count; i++) {
        cudaStreamWaitEvent(b->streams[i], b->fork_ev, 0);
        bd_step_opts o = *opts;
        o.seed = opts->seed + (uint64_t)i;
        o.flags |= BD_STEP_DEVICE_COUNTER;
        bd_status st = step_part(b->plans[i], R + b->r_off[i], (char *)D + b->d_off[i], &o,
                                 stats ? stats + i : nullptr, b->streams[i], 1, b->d_reps + i,
                                 b->item0[i]);
        if (st != BD_OK) return st;
        lag = step_part_lag(b->plans[i]);
        cudaEventRecord(b->join_ev[i], b->streams[i]);
        cudaStreamWaitEvent(stream, b->join_ev[i], 0);
    }
    bd_status st = rows_cheb_launch(b->d_reps, b->count, b->d_items, b->nitems, opts->m + lag,
                                    opts->n_cheb, lag ? 0 : -1, b->d_bar,
                                    plan_device(b->plans[0]), stream);
    if (st != BD_OK) return st;
    if (cudaEventRecord(b->mid_ev, stream) != cudaSuccess) return check_launch("batch fork");
    for (int i = 0; i < b->count; i++) {
        cudaStreamWaitEvent(b->streams[i], b->mid_ev, 0);
        st = step_part(b->plans[i], R + b->r_off[i], (char *)D + b->d_off[i], opts,
                       stats ? stats + i : nullptr, b->streams[i], 2, nullptr, 0);
        if (st != BD_OK) return st;
        cudaEventRecord(b->join_ev[i], b->streams[i]);
        cudaStreamWaitEvent(stream, b->join_ev[i], 0);
    }
    return check_launch("batch step");
}

// fork from `stream`, one bd_step per replica on its branch, join back
static bd_status batch_body(bd_batch *b, double *R, void *D, const bd_step_opts *opts,
                            bd_step_stats *stats, cudaStream_t stream)
{
    if (b->rows && step_batchable(b->plans[0], opts))
        return batch_body_rows(b, R, D, opts, stats, stream);
    if (cudaEventRecord(b->fork_ev, stream) != cudaSuccess) return check_launch("batch fork");
    for (int i = 0; i < b->count; i++) {
        cudaStreamWaitEvent(b->streams[i], b->fork_ev, 0);
        bd_step_opts o = *opts;
        o.seed = opts->seed + (uint64_t)i;
        o.flags |= BD_STEP_DEVICE_COUNTER;
        bd_status st = bd_step(b->plans[i], R + b->r_off[i], (char *)D + b->d_off[i], nullptr, &o,
                               nullptr, nullptr, stats ? stats + i : nullptr, b->streams[i]);
        if (st != BD_OK) return st;
        cudaEventRecord(b->join_ev[i], b->streams[i]);
        cudaStreamWaitEvent(stream, b->join_ev[i], 0);
    }
    return check_launch("batch step");
}

bd_status bd_batch_step(bd_batch *b, double *R, void *D, const bd_step_opts *opts,
                        bd_step_stats *stats, bd_stream stream)
{
    if (!b || !R || !D || !opts) return set_error(BD_ERR_INVALID, "NULL argument");
    if (opts->n_cheb == 0)
        return set_error(BD_ERR_INVALID, "adaptive N_Ch synchronises and cannot run in a batch");
    if (((uintptr_t)D & 255) != 0) return set_error(BD_ERR_INVALID, "D must be 256-byte aligned");
    cudaStream_t s = stream;
    if (b->calls == 0) {
        // direct run: set the device counters, prime lagged bounds
        for (int i = 0; i < b->count; i++) {
            bd_status st = bd_plan_set_step_counter(b->plans[i], opts->step_index, s);
            if (st != BD_OK) return st;
        }
        b->calls = 1;
        return batch_body(b, R, D, opts, stats, s);
    }
    const bool same = b->exec && b->key_R == R && b->key_D == D && b->key_stats == stats &&
                      memcmp(&b->key_opts, opts, sizeof(*opts)) == 0;
    if (!same) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        // recorded on the batch's own stream; the graph is then launched on
        // the caller's stream, which may be the legacy default stream
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return check_launch("batch capture begin");
        bd_status st = batch_body(b, R, D, opts, stats, b->origin);
        cudaError_t e = cudaStreamEndCapture(b->origin, &g);
        if (st != BD_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess || !g)
            return set_error(BD_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return set_error(BD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        b->key_R = R;
        b->key_D = D;
        b->key_stats = stats;
        b->key_opts = *opts;
    }
    b->calls++;
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return check_launch("batch graph launch");
    count_launches(1);
    return BD_OK;
}

}  // extern "C"
