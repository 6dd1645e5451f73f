// batch.cu -- the batch calls of the C ABI.
//
// Many grids of one storage type advance together: every step is one launch of
// the persistent step kernel over a packed tile work-list of all grids (each
// item: grid, tile column/row, z range of at most kBatchZChunk planes) plus one
// launch of the ghost-face kernel over all grids.  The per-grid records (step
// coefficients, buffers, TMA maps) live in the caller's scratch and are read
// by the kernels at run time, so a captured CUDA graph of kGraphSteps steps is
// replayed unchanged across calls; parameters can change between calls.  Each
// grid's arithmetic is exactly the single-grid step's.
#include <math.h>
#include <string.h>

#include <vector>

#include "host_internal.h"

using namespace spfm;
using namespace spfm_host;

namespace {

constexpr int kBatchZChunk = 32;   // z-march depth of the items until tuned
constexpr int kGraphSteps = 16;    // steps per captured graph (even: parity repeats)
// depths the autotuner tries; the scratch holds the work-list of the shallowest
constexpr int kDepths[] = {8, 12, 16, 24, 32, 48, 64};
constexpr int kNDepths = (int)(sizeof(kDepths) / sizeof(kDepths[0]));
constexpr int kMinDepth = 8;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    size_t grids, items, ghosts, stats_jobs, partials, finals, err, steps, total;
};

size_t grid_record_bytes(int dtype)
{
    return dtype == SPFM_F64 ? batch_grid_bytes_f64()
                             : (dtype == SPFM_F32 ? batch_grid_bytes_f32() : batch_grid_bytes_bf16());
}

int items_of(int dtype, const GridGeom &g, int gi, int depth, BatchItem *out, int shape)
{
    return dtype == SPFM_F64   ? batch_items_f64(g, gi, depth, out, shape)
           : dtype == SPFM_F32 ? batch_items_f32(g, gi, depth, out, shape)
                               : batch_items_bf16(g, gi, depth, out, shape);
}

// Tile shapes of FP32 batch items: 0 = 64 x 16 cells (the single-grid tile),
// 1 = 32 x 32.  A tile policy gives every grid one of them:
//   SPFM_TILES_WIDE all 0, SPFM_TILES_SQUARE all 1, SPFM_TILES_FIT the shape
//   whose tiles pad the grid's xy extent least (ties keep 0).
// Other storage types have the one shape 0.
int shape_for(int dtype, const GridGeom &g, int policy)
{
    if (dtype != SPFM_F32 || policy == SPFM_TILES_WIDE) return 0;
    if (policy == SPFM_TILES_SQUARE) return 1;
    const long long wide = (long long)((g.nx + 63) / 64 * 64) * ((g.ny + 15) / 16 * 16);
    const long long sq = (long long)((g.nx + 31) / 32 * 32) * ((g.ny + 31) / 32 * 32);
    return sq < wide ? 1 : 0;
}

Layout layout_for(int dtype, int n, int nitems)
{
    Layout L;
    size_t off = 0;
    L.grids = off;
    off = align_up(off + grid_record_bytes(dtype) * n, 256);
    L.items = off;
    off = align_up(off + sizeof(BatchItem) * nitems, 256);
    L.ghosts = off;
    off = align_up(off + sizeof(GhostJob) * n, 256);
    L.stats_jobs = off;
    off = align_up(off + sizeof(StatsJob) * n, 256);
    L.partials = off;
    off = align_up(off + sizeof(double) * kNStat * kBatchStatsBlocks * n, 256);
    L.finals = off;
    off = align_up(off + sizeof(double) * (kNStat * n + 1), 256);
    L.err = off;
    off = align_up(off + 16, 256);
    L.steps = off;   // each grid's step count: the step keys of stochastic rounding
    off = align_up(off + sizeof(long long) * n, 256);
    L.total = off;
    return L;
}

int check_grids(spfm_grid *const *grids, int n, int *dtype, int *nitems)
{
    if (!grids || n < 1) return fail(nullptr, SPFM_EINVAL, "spfm_batch: need at least one grid");
    int items = 0;
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return fail(nullptr, SPFM_EINVAL, "spfm_batch: grid %d is NULL", i);
        if (grids[i]->d.dtype != grids[0]->d.dtype)
            return fail(nullptr, SPFM_EINVAL, "spfm_batch: grid %d has another dtype", i);
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i]) return fail(nullptr, SPFM_EINVAL, "spfm_batch: grid %d repeated", i);
        const int a = items_of(grids[i]->d.dtype, grids[i]->geom, i, kMinDepth, nullptr, 0);
        const int b = grids[i]->d.dtype == SPFM_F32 ? items_of(SPFM_F32, grids[i]->geom, i, kMinDepth, nullptr, 1) : 0;
        items += a > b ? a : b;
    }
    *dtype = grids[0]->d.dtype;
    *nitems = items;   // the longest work-list (shallowest depth, either shape): the scratch size
    return SPFM_OK;
}

}  // namespace

struct spfm_batch {
    std::vector<spfm_grid *> grids;
    int n = 0, dtype = 0, nitems = 0, depth = kBatchZChunk, policy = SPFM_TILES_FIT;
    int nitems0 = 0;   // items of shape 0; the shape-1 items follow them in the list
    char *scratch = nullptr;
    cudaStream_t stream = nullptr;
    Layout L;
    std::vector<BatchItem> h_items;
    std::vector<char> h_grids;
    std::vector<GhostJob> h_ghosts;
    std::vector<StatsJob> h_stats;
    std::vector<double> h_finals;
    std::vector<long long> h_steps;
    int sr = 0;   // the grids round their updates stochastically (they share the mode)
    // no grid has a periodic face: the step kernels compute the ghosts as they
    // read them and no ghost kernel runs between steps
    bool inline_faces = false;
    cudaGraphExec_t exec = nullptr;
    int graph_stencil = -1, graph_kind = -1, graph_sr = -1;
    std::string err;
    ~spfm_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

static int bfail(spfm_batch *b, int code, const char *msg)
{
    if (b) b->err = msg;
    return fail(nullptr, code, "%s", msg);
}

// the work-list of z-march depth `depth` under the batch's tile policy,
// uploaded on the batch's stream (the captured graph holds the item count, so
// it is dropped)
static cudaError_t set_depth(spfm_batch *b, int depth)
{
    int k = 0;
    for (int i = 0; i < b->n; ++i) {
        const GridGeom &g = b->grids[i]->geom;
        k += items_of(b->dtype, g, i, depth, nullptr, shape_for(b->dtype, g, b->policy));
    }
    b->h_items.resize(k);
    k = 0;
    for (int shape = 0; shape < 2; ++shape) {   // shape 0 items first, one launch per shape
        for (int i = 0; i < b->n; ++i) {
            const GridGeom &g = b->grids[i]->geom;
            if (shape_for(b->dtype, g, b->policy) == shape)
                k += items_of(b->dtype, g, i, depth, b->h_items.data() + k, shape);
        }
        if (shape == 0) b->nitems0 = k;
    }
    b->nitems = k;
    b->depth = depth;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return cudaMemcpyAsync(b->scratch + b->L.items, b->h_items.data(), sizeof(BatchItem) * k,
                           cudaMemcpyHostToDevice, b->stream);
}

// one step of every grid: persistent step kernel (one per tile shape in the
// list), then the ghost faces of the buffers it wrote; sub: the step's index
// since the device step counters were last advanced
static cudaError_t launch_one(spfm_batch *b, int parity, int stencil, int kind, int sub)
{
    const void *grids = b->scratch + b->L.grids;
    const BatchItem *items = (const BatchItem *)(b->scratch + b->L.items);
    int *err = (int *)(b->scratch + b->L.err);
    const long long *steps = (const long long *)(b->scratch + b->L.steps);
    cudaError_t e;
    const int fwd = b->inline_faces ? 1 : 0;
    if (b->dtype == SPFM_F64) {
        e = launch_batch_f64(grids, items, b->nitems, parity, err, stencil, kind, b->stream, fwd);
    } else if (b->dtype == SPFM_F32) {
        // the two tile shapes run as two persistent launches over their parts of
        // the list (their grids differ, so the second needs nothing of the first)
        e = cudaSuccess;
        if (b->nitems0 > 0)
            e = launch_batch_f32(grids, items, b->nitems0, parity, err, stencil, kind, b->stream, 0, b->sr, steps,
                                 sub, fwd);
        if (e == cudaSuccess && b->nitems > b->nitems0)
            e = launch_batch_f32(grids, items + b->nitems0, b->nitems - b->nitems0, parity, err, stencil, kind,
                                 b->stream, 1, b->sr, steps, sub, fwd);
    } else {
        e = launch_batch_bf16(grids, items, b->nitems, parity, err, stencil, kind, b->stream, b->sr, steps, sub,
                              fwd);
    }
    if (e != cudaSuccess || b->inline_faces) return e;
    return launch_fill_ghosts_batch((const GhostJob *)(b->scratch + b->L.ghosts), b->n, b->dtype,
                                    parity ^ 1, b->stream);
}

static cudaError_t capture_graph(spfm_batch *b, int stencil, int kind)
{
    if (b->exec && b->graph_stencil == stencil && b->graph_kind == kind && b->graph_sr == b->sr) return cudaSuccess;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < kGraphSteps && le == cudaSuccess; ++s) le = launch_one(b, s & 1, stencil, kind, s);
    if (le == cudaSuccess && b->sr)
        le = launch_advance_steps((long long *)(b->scratch + b->L.steps), b->n, kGraphSteps, b->stream);
    e = cudaStreamEndCapture(b->stream, &graph);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess) {
        b->graph_stencil = stencil;
        b->graph_kind = kind;
        b->graph_sr = b->sr;
    } else {
        b->exec = nullptr;
    }
    return e;
}

namespace spfm {

__global__ void advance_steps_kernel(long long *steps, int n, int k)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) steps[i] += k;
}

cudaError_t launch_advance_steps(long long *steps, int n, int k, cudaStream_t st)
{
    advance_steps_kernel<<<(n + 255) / 256, 256, 0, st>>>(steps, n, k);
    return cudaGetLastError();
}

}  // namespace spfm

extern "C" {

spfm_status spfm_batch_scratch_bytes(spfm_grid *const *grids, int n, size_t *bytes)
{
    int dtype = 0, nitems = 0;
    spfm_status st = check_grids(grids, n, &dtype, &nitems);
    if (st != SPFM_OK) return st;
    if (bytes) *bytes = layout_for(dtype, n, nitems).total;
    return SPFM_OK;
}

spfm_status spfm_batch_create(spfm_grid *const *grids, int n, void *scratch, size_t scratch_bytes,
                              void *stream, spfm_batch **out)
{
    if (!out) return fail(nullptr, SPFM_EINVAL, "spfm_batch_create: out is NULL");
    *out = nullptr;
    int dtype = 0, nitems = 0;
    spfm_status st = check_grids(grids, n, &dtype, &nitems);
    if (st != SPFM_OK) return st;
    const Layout L = layout_for(dtype, n, nitems);
    if (!scratch || ((uintptr_t)scratch & 255) || scratch_bytes < L.total)
        return fail(nullptr, SPFM_ENOMEM, "spfm_batch_create: scratch NULL, not 256-byte aligned or below %zu bytes",
                    L.total);
    spfm_batch *b = new spfm_batch();
    b->grids.assign(grids, grids + n);
    b->n = n;
    b->dtype = dtype;
    b->nitems = nitems;
    b->scratch = (char *)scratch;
    b->stream = (cudaStream_t)stream;
    b->L = L;
    b->inline_faces = true;
    for (int i = 0; i < n; ++i) b->inline_faces = b->inline_faces && faces_inline(grids[i]);
    b->h_grids.assign(grid_record_bytes(dtype) * n, 0);
    b->h_ghosts.resize(n);
    b->h_stats.resize(n);
    b->h_finals.resize((size_t)kNStat * n + 1);
    b->h_steps.resize(n);
    cudaError_t e = set_depth(b, kBatchZChunk);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->scratch + L.err, 0, 16, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        delete b;
        return fail(nullptr, SPFM_ECUDA, "spfm_batch_create: %s", cudaGetErrorString(e));
    }
    *out = b;
    return SPFM_OK;
}

spfm_status spfm_batch_step(spfm_batch *b, int n_steps, const spfm_step_args *args)
{
    if (!b || !args) return fail(nullptr, SPFM_EINVAL, "spfm_batch_step: NULL argument");
    if (n_steps < 0) return bfail(b, SPFM_EINVAL, "spfm_batch_step: n_steps < 0");
    const int stencil = args[0].stencil, scheme = args[0].scheme;
    if (scheme == SPFM_TI_LOCAL)
        return bfail(b, SPFM_EINVAL, "spfm_batch_step: SPFM_TI_LOCAL is not available for batches");
    const size_t rec = grid_record_bytes(b->dtype);
    cudaError_t e = cudaSuccess;
    b->sr = b->grids[0]->rounding == SPFM_ROUND_STOCHASTIC ? 1 : 0;
    for (int i = 0; i < b->n; ++i) {
        spfm_grid *g = b->grids[i];
        const spfm_step_args &a = args[i];
        if (a.stencil != stencil || a.scheme != scheme)
            return bfail(b, SPFM_EINVAL, "spfm_batch_step: all grids of a batch share stencil and scheme");
        if ((g->rounding == SPFM_ROUND_STOCHASTIC ? 1 : 0) != b->sr)
            return bfail(b, SPFM_EINVAL, "spfm_batch_step: all grids of a batch share the rounding mode");
        b->h_steps[i] = g->steps;
        Model m;
        spfm_status st = build_model(g, a.M, a.Gamma, a.lambda, a.dx, a.dt, a.dF, a.stencil, a.scheme, m);
        if (st != SPFM_OK) {
            char msg[600];
            snprintf(msg, sizeof msg, "grid %d: %s", i, g->err.c_str());
            return bfail(b, st, msg);
        }
        if (n_steps > 0 && !b->inline_faces &&
            (g->ghosts_dirty || g->ghost_lambda != a.lambda || g->ghost_dx != a.dx)) {
            e = launch_fill_ghosts(g->geom, g->d.dtype, m.aface, g->d.field[g->cur], b->stream, 1);
            if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
            g->ghosts_dirty = false;
            g->ghost_lambda = a.lambda;
            g->ghost_dx = a.dx;
        }
        void *slot = b->h_grids.data() + rec * i;
        if (b->dtype == SPFM_F64) {
            StepCoef<double> c;
            fill_coef<double>(g, m, a.dt, a.stencil, c);
            batch_fill_grid_f64(slot, c, g->d.field, g->cur, &g->tma);
        } else {
            StepCoef<float> c;
            fill_coef<float>(g, m, a.dt, a.stencil, c);
            if (b->dtype == SPFM_F32) batch_fill_grid_f32(slot, c, g->d.field, g->cur, &g->tma);
            else batch_fill_grid_bf16(slot, c, g->d.field, g->cur, &g->tma);
        }
        GhostJob &gj = b->h_ghosts[i];
        gj.g = g->geom;
        for (int f = 0; f < 6; ++f) gj.aface[f] = m.aface[f];
        gj.field[0] = g->d.field[0];
        gj.field[1] = g->d.field[1];
        gj.cur = g->cur;
    }
    if (n_steps == 0) return SPFM_OK;
    const int kind = is_fd_scheme(scheme) ? 0 : 5;
    e = cudaMemcpyAsync(b->scratch + b->L.grids, b->h_grids.data(), rec * b->n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->scratch + b->L.ghosts, b->h_ghosts.data(), sizeof(GhostJob) * b->n,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && b->sr)
        e = cudaMemcpyAsync(b->scratch + b->L.steps, b->h_steps.data(), sizeof(long long) * b->n,
                            cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
    int s = 0;
    // graphs need a capturable stream (not the legacy default stream)
    if (n_steps >= kGraphSteps && b->stream != nullptr) {
        e = capture_graph(b, stencil, kind);
        if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
        for (; s + kGraphSteps <= n_steps; s += kGraphSteps) {
            e = cudaGraphLaunch(b->exec, b->stream);
            if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
        }
    }
    const int s0 = s;   // the graphs advanced the device step counters up to here
    for (; s < n_steps; ++s) {
        e = launch_one(b, s & 1, stencil, kind, s - s0);
        if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
    }
    if (b->sr && n_steps > s0) {
        e = launch_advance_steps((long long *)(b->scratch + b->L.steps), b->n, n_steps - s0, b->stream);
        if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
    }
    for (int i = 0; i < b->n; ++i) {
        spfm_grid *g = b->grids[i];
        const spfm_step_args &a = args[i];
        g->cur ^= (n_steps & 1);
        if (b->inline_faces && n_steps > 0) g->ghosts_dirty = true;   // the ghost layer in memory is stale
        g->steps += n_steps;
        g->time += n_steps * a.dt;
        g->M = a.M;
        g->Gamma = a.Gamma;
        g->lambda = a.lambda;
        g->dx = a.dx;
        g->dF = a.dF;
        g->stencil = a.stencil;
        g->scheme = a.scheme;
    }
    return SPFM_OK;
}

spfm_status spfm_batch_autotune(spfm_batch *b, const spfm_step_args *args, int steps_per_trial,
                                int *out_depth, double *out_ms)
{
    if (!b || !args) return fail(nullptr, SPFM_EINVAL, "spfm_batch_autotune: NULL argument");
    if (steps_per_trial < kGraphSteps || steps_per_trial % kGraphSteps)
        return bfail(b, SPFM_EINVAL, "spfm_batch_autotune: steps_per_trial must be a positive multiple of 16");
    if (!b->stream) return bfail(b, SPFM_EINVAL, "spfm_batch_autotune: needs a non-default stream");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
    }
    spfm_status st = SPFM_OK;
    // the tile policy first, at the current depth (FP32 only: one shape otherwise)
    if (b->dtype == SPFM_F32) {
        int best_policy = b->policy;
        double best_pol_ms = 0.0;
        const int policies[3] = {SPFM_TILES_WIDE, SPFM_TILES_SQUARE, SPFM_TILES_FIT};
        for (int c = 0; c < 3 && st == SPFM_OK; ++c) {
            b->policy = policies[c];
            e = set_depth(b, b->depth);
            if (e != cudaSuccess) {
                st = bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
                break;
            }
            st = spfm_batch_step(b, kGraphSteps, args);
            if (st != SPFM_OK) break;
            e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) st = spfm_batch_step(b, steps_per_trial, args);
            if (e == cudaSuccess && st == SPFM_OK) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess && st == SPFM_OK) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess && st == SPFM_OK) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) st = bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
            if (st != SPFM_OK) break;
            if (c == 0 || ms < best_pol_ms) {
                best_pol_ms = ms;
                best_policy = policies[c];
            }
        }
        b->policy = best_policy;
    }
    int best = kBatchZChunk;
    double best_ms = 0.0;
    for (int c = 0; c < kNDepths && st == SPFM_OK; ++c) {
        e = set_depth(b, kDepths[c]);
        if (e != cudaSuccess) {
            st = bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
            break;
        }
        st = spfm_batch_step(b, kGraphSteps, args);   // captures this depth's graph, warms up
        if (st != SPFM_OK) break;
        e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) st = spfm_batch_step(b, steps_per_trial, args);
        if (e == cudaSuccess && st == SPFM_OK) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess && st == SPFM_OK) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess && st == SPFM_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) st = bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
        if (st != SPFM_OK) break;
        const double per = (double)ms / steps_per_trial;
        if (out_ms) out_ms[c] = per;
        if (c == 0 || per < best_ms) {
            best_ms = per;
            best = kDepths[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SPFM_OK) return st;
    e = set_depth(b, best);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
    if (out_depth) *out_depth = best;
    return SPFM_OK;
}

spfm_status spfm_batch_set_tiles(spfm_batch *b, int policy)
{
    if (!b) return fail(nullptr, SPFM_EINVAL, "spfm_batch_set_tiles: batch is NULL");
    if (policy != SPFM_TILES_WIDE && policy != SPFM_TILES_SQUARE && policy != SPFM_TILES_FIT)
        return bfail(b, SPFM_EINVAL, "spfm_batch_set_tiles: unknown tile policy");
    b->policy = policy;
    cudaError_t e = set_depth(b, b->depth);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
    return SPFM_OK;
}

spfm_status spfm_batch_tiles(const spfm_batch *b, int *policy, int *depth)
{
    if (!b) return fail(nullptr, SPFM_EINVAL, "spfm_batch_tiles: batch is NULL");
    if (policy) *policy = b->policy;
    if (depth) *depth = b->depth;
    return SPFM_OK;
}

spfm_status spfm_batch_stats(spfm_batch *b, int flags, spfm_stats *out)
{
    if (!b || !out) return fail(nullptr, SPFM_EINVAL, "spfm_batch_stats: NULL argument");
    for (int i = 0; i < b->n; ++i) {
        spfm_grid *g = b->grids[i];
        if (!(g->lambda > 0.0)) return bfail(b, SPFM_EINVAL, "spfm_batch_stats: a grid has no model yet");
        StatsJob &j = b->h_stats[i];
        fill_stats_args(g, flags, j.a);
        // the energy reads the ghosts: refresh a stale layer (no periodic face:
        // the steps do not keep it in memory)
        if (j.a.energy && (g->ghosts_dirty || g->ghost_lambda != g->lambda || g->ghost_dx != g->dx)) {
            spfm_status st = refresh_ghosts(g, g->lambda, g->dx, b->stream);
            if (st != SPFM_OK) return bfail(b, st, "spfm_batch_stats: ghost refresh failed");
        }
        j.field[0] = g->d.field[0];
        j.field[1] = g->d.field[1];
        j.cur = g->cur;
    }
    double *finals = (double *)(b->scratch + b->L.finals);
    cudaError_t e = cudaMemcpyAsync(b->scratch + b->L.stats_jobs, b->h_stats.data(), sizeof(StatsJob) * b->n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = launch_stats_batch((const StatsJob *)(b->scratch + b->L.stats_jobs), b->n, b->dtype,
                               (double *)(b->scratch + b->L.partials), finals, b->stream);
    // the error word sits right after the finals region: copy both
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_finals.data(), finals, sizeof(double) * kNStat * b->n, cudaMemcpyDeviceToHost,
                            b->stream);
    int errw = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&errw, b->scratch + b->L.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SPFM_ECUDA, cudaGetErrorString(e));
    double nonfinite = 0.0;
    for (int i = 0; i < b->n; ++i) {
        stats_from_reduction(b->grids[i], b->h_finals.data() + (size_t)kNStat * i, b->h_stats[i].a.energy, &out[i]);
        nonfinite += out[i].nonfinite;
    }
    if (errw != 0) return bfail(b, SPFM_ETIMEOUT, "a bounded wait in the batch step kernel gave up");
    if (nonfinite > 0.0) return bfail(b, SPFM_ENONFINITE, "a grid of the batch holds non-finite cells");
    return SPFM_OK;
}

spfm_status spfm_batch_destroy(spfm_batch *b)
{
    delete b;
    return SPFM_OK;
}

}  // extern "C"
