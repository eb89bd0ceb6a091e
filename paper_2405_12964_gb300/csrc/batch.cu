// Batched reverse-mode runs: many independent problems (each a context with
// its own boundary, BVH, data, PDE and options) in one pass.
//
// All problems of one dimension share a persistent walk kernel launch over a
// table of problem descriptors (up to 64 per launch), so lanes move from one
// problem's walks to the next and the tail of long walks is paid once per
// launch instead of once per problem.  Each problem then gets its U-statistic
// scatter, adjoint GEMV, mean and loss.  A pass enqueues only kernels and
// memsets on the batch's stream, so it can be captured once into a CUDA graph
// and replayed.  An autotuner times the walk launch of each dimension group
// over block size, resident blocks per SM and the distance-query search order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"
#include "dwos_internal.h"

using namespace dwos;

namespace {
constexpr int kChunk = 64;   // problems per walk launch (descriptor table in shared memory)

struct Chunk {
    int dim = 0;
    std::vector<int> jobs;              // job indices
    DevProblem* d_probs = nullptr;      // descriptor table
    DevCounters* d_ctr = nullptr;
    unsigned long long total = 0;       // walks
};
}  // namespace

struct dwos_batch {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<dwos_batch_job> jobs;
    std::vector<Chunk> chunks;
    dwos_record* rec = nullptr;
    std::vector<size_t> rec_off;
    uint32_t* trace = nullptr;          // per job: (K + 1) words per walk, when traces are on
    std::vector<size_t> trace_off;
    double* acc = nullptr;              // per job: n_vert*dim + n_vert doubles
    std::vector<size_t> acc_off;
    unsigned char* active = nullptr;    // per job: n_vert vertex flags (nonzero Jacobian / dg row)
    std::vector<size_t> active_off;
    WalkLaunch cfg[4];                  // per dimension (index 2 and 3)
    int trav[4] = {0, 0, 3, 3};         // per dimension: routed search (order 3)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    float last_walk_ms[4] = {0, 0, 0, 0};
};

namespace {

thread_local std::string g_batch_err;

dwos_status bfail(dwos_batch* b, dwos_status s, const std::string& m) {
    if (b) b->err = m; else g_batch_err = m;
    return s;
}

dwos_status bcuda(dwos_batch* b, cudaError_t e, const char* where) {
    cudaGetLastError();
    return bfail(b, e == cudaErrorMemoryAllocation ? DWOS_ERR_OOM : DWOS_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define BK(call, where) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) return bcuda(b, e_, where); } while (0)

bool on_device(const void* p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

void fill_problem(const dwos_ctx* c, const dwos_batch_job& j, dwos_record* rec, uint32_t* trace,
                  unsigned long long begin, int traversal, DevProblem& P) {
    std::memset(&P, 0, sizeof(P));
    P.nodes = c->bvh.nodes;
    P.prims = c->bvh.prims;
    P.prim_elem = c->bvh.prim_elem;
    P.elem = c->elem;
    P.g_vert = c->g_vert;
    P.root = 0;
    P.n_internal = c->bvh.n_internal;
    P.n_tree = c->bvh.n_tree;
    P.n_big = c->bvh.n_big;
    P.leaf_parent = c->bvh.leaf_parent;
    P.node_cell = c->bvh.node_cell;
    P.r_max = c->bvh.r_max;
    P.traversal = (traversal == 1 && !c->bvh.cells_ok) ? 0 : traversal;   // order 1 needs a fresh build
    P.wnodes = c->bvh.wnodes;
    P.n_wide = c->bvh.n_wide;
    P.data_kind = c->data_kind;
    P.differential = 1;
    for (int i = 0; i < 10; ++i) P.field[i] = (float)c->field[i];
    P.sqrt_sigma = std::sqrt(c->sigma);
    P.f = c->f;
    P.eps = c->opt.eps;
    P.h = c->opt.h;
    P.inv_h = 1.0f / c->opt.h;
    P.K = c->opt.K;
    P.max_steps = c->opt.max_steps;
    P.dudn_mode = c->opt.dudn_estimator;
    P.seed_lo = (uint32_t)c->opt.seed;
    P.seed_hi = (uint32_t)(c->opt.seed >> 32);
    P.xq = j.xq;
    P.valid = nullptr;     // checked once at creation
    P.walks = j.walks_per_point;
    P.node_budget = c->node_budget;
    P.walk_id_base = j.walk_id_base;
    const unsigned long long n = (unsigned long long)j.n_query * (unsigned long long)j.walks_per_point;
    P.work_begin = begin;
    P.work_end = begin + n;
    P.rec = rec;
    P.trace = trace;
}

// The warp-wide search serves a launch only if every problem's tree supports it.
bool wide_ok_dim(const dwos_batch* b, int dim) {
    for (const auto& ch : b->chunks)
        if (ch.dim == dim)
            for (int ji : ch.jobs)
                if (!b->jobs[ji].ctx->bvh.wide_ok) return false;
    return true;
}

// Rewrite the descriptor tables (after an autotuner change of search order).
dwos_status upload_tables(dwos_batch* b) {
    for (int dim = 2; dim <= 3; ++dim)
        if ((b->trav[dim] == 2 || b->trav[dim] == 3) && !wide_ok_dim(b, dim)) b->trav[dim] = 0;
    for (auto& ch : b->chunks) {
        std::vector<DevProblem> tab(ch.jobs.size());
        unsigned long long begin = 0;
        b->cfg[ch.dim].traversal = b->trav[ch.dim];
        for (size_t k = 0; k < ch.jobs.size(); ++k) {
            const int ji = ch.jobs[k];
            const dwos_batch_job& j = b->jobs[ji];
            fill_problem(j.ctx, j, b->rec + b->rec_off[ji], b->trace ? b->trace + b->trace_off[ji] : nullptr, begin,
                         b->trav[ch.dim], tab[k]);
            begin = tab[k].work_end;
        }
        BK(cudaMemcpy(ch.d_probs, tab.data(), sizeof(DevProblem) * tab.size(), cudaMemcpyHostToDevice), "upload table");
    }
    return DWOS_OK;
}

dwos_status run_walks_only(dwos_batch* b, int dim_filter) {
    for (auto& ch : b->chunks) {
        if (dim_filter && ch.dim != dim_filter) continue;
        BK(cudaMemsetAsync(ch.d_ctr, 0, sizeof(DevCounters), b->stream), "reset counters");
        int blocks = 0;
        BK(launch_walks(b->cfg[ch.dim], ch.d_probs, (int)ch.jobs.size(), ch.total, ch.d_ctr, b->stream, &blocks),
           "walk kernel");
    }
    return DWOS_OK;
}

}  // namespace

extern "C" {

dwos_status dwos_batch_create(dwos_batch** out, const dwos_batch_job* jobs, int n_jobs, void* stream) {
    if (!out) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!jobs || n_jobs < 1) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "no jobs");
    dwos_batch* b = new dwos_batch();
    b->stream = (cudaStream_t)stream;
    b->jobs.assign(jobs, jobs + n_jobs);
    b->device = jobs[0].ctx ? jobs[0].ctx->device : 0;
    auto bail = [&](dwos_status s) { g_batch_err = b->err; dwos_batch_destroy(b); return s; };
    for (int i = 0; i < n_jobs; ++i) {
        const dwos_batch_job& j = jobs[i];
        const std::string tag = "job " + std::to_string(i) + ": ";
        if (!j.ctx) return bail(bfail(b, DWOS_ERR_INVALID_ARG, tag + "ctx is NULL"));
        if (j.ctx->device != b->device) return bail(bfail(b, DWOS_ERR_INVALID_ARG, tag + "contexts must share one device"));
        if (!j.ctx->have_boundary) return bail(bfail(b, DWOS_ERR_STATE, tag + "context has no boundary"));
        if (j.ctx->n_neumann > 0) return bail(bfail(b, DWOS_ERR_NOT_IMPLEMENTED, tag + "batches of problems with a Neumann part"));
        if (j.n_query < 1 || j.walks_per_point < 1) return bail(bfail(b, DWOS_ERR_INVALID_ARG, tag + "empty job"));
        if (j.walks_per_point % j.ctx->opt.B) return bail(bfail(b, DWOS_ERR_INVALID_ARG, tag + "walks_per_point must be a multiple of B"));
        if (!on_device(j.xq, b->device) || !on_device(j.uref, b->device) || !on_device(j.loss, b->device))
            return bail(bfail(b, DWOS_ERR_INVALID_ARG, tag + "xq, uref and loss must be device pointers"));
        if (j.ctx->n_param > 0 && !on_device(j.grad_param, b->device))
            return bail(bfail(b, DWOS_ERR_INVALID_ARG, tag + "grad_param must be a device pointer"));
        if (j.u_mean && !on_device(j.u_mean, b->device))
            return bail(bfail(b, DWOS_ERR_INVALID_ARG, tag + "u_mean must be a device pointer"));
    }
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bail(bcuda(b, e, "cudaSetDevice"));
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    // inside test once, here, so that a pass needs no host round trip
    {
        int max_q = 0;
        for (auto& j : b->jobs) max_q = std::max(max_q, j.n_query);
        int* flags = nullptr;
        if ((e = cudaMalloc(&flags, sizeof(int) * max_q)) != cudaSuccess) return bail(bcuda(b, e, "alloc"));
        std::vector<int> h(max_q);
        for (int i = 0; i < n_jobs; ++i) {
            const dwos_batch_job& j = b->jobs[i];
            if (!j.ctx->opt.check_inside) continue;
            e = launch_inside(j.ctx->bvh, j.n_query, j.xq, flags, b->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), flags, sizeof(int) * j.n_query, cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) { cudaFree(flags); return bail(bcuda(b, e, "inside test")); }
            for (int q = 0; q < j.n_query; ++q)
                if (!h[q]) { cudaFree(flags); return bail(bfail(b, DWOS_ERR_OUTSIDE, "job " + std::to_string(i) + ": a query point lies outside the domain")); }
        }
        cudaFree(flags);
    }
    // buffers
    size_t n_rec = 0, n_acc = 0;
    for (auto& j : b->jobs) {
        b->rec_off.push_back(n_rec);
        b->acc_off.push_back(n_acc);
        n_rec += (size_t)j.n_query * j.walks_per_point;
        n_acc += (size_t)j.ctx->n_vert * j.ctx->dim + j.ctx->n_vert + j.n_query;   // + per-point sums of u
    }
    if ((e = cudaMalloc(&b->rec, sizeof(dwos_record) * n_rec)) != cudaSuccess) return bail(bcuda(b, e, "alloc records"));
    if ((e = cudaMalloc(&b->acc, sizeof(double) * n_acc)) != cudaSuccess) return bail(bcuda(b, e, "alloc accumulators"));
    // vertices with zero Jacobian and dg rows cannot reach a job's parameter gradient: the
    // scatter skips them (the batch returns no vertex gradients)
    {
        size_t n_act = 0;
        for (auto& j : b->jobs) { b->active_off.push_back(n_act); n_act += (size_t)std::max(j.ctx->n_vert, 1); }
        if ((e = cudaMalloc(&b->active, n_act)) != cudaSuccess) return bail(bcuda(b, e, "alloc vertex flags"));
        for (int i = 0; i < n_jobs; ++i) {
            const dwos_ctx* c = b->jobs[i].ctx;
            if ((e = launch_vertex_active(c->jac, c->dg_vert, c->n_vert, c->dim, c->n_param, b->active + b->active_off[i],
                                          b->stream)) != cudaSuccess)
                return bail(bcuda(b, e, "vertex flags"));
        }
    }
    // chunks of up to 64 problems per dimension
    for (int dim = 2; dim <= 3; ++dim) {
        std::vector<int> ids;
        for (int i = 0; i < n_jobs; ++i) if (b->jobs[i].ctx->dim == dim) ids.push_back(i);
        for (size_t k = 0; k < ids.size(); k += kChunk) {
            Chunk ch;
            ch.dim = dim;
            ch.jobs.assign(ids.begin() + k, ids.begin() + std::min(ids.size(), k + kChunk));
            for (int ji : ch.jobs) ch.total += (unsigned long long)b->jobs[ji].n_query * b->jobs[ji].walks_per_point;
            if ((e = cudaMalloc(&ch.d_probs, sizeof(DevProblem) * ch.jobs.size())) != cudaSuccess) return bail(bcuda(b, e, "alloc table"));
            if ((e = cudaMalloc(&ch.d_ctr, sizeof(DevCounters))) != cudaSuccess) { cudaFree(ch.d_probs); return bail(bcuda(b, e, "alloc counters")); }
            b->chunks.push_back(ch);
        }
        b->cfg[dim].dim = dim;
        b->cfg[dim].block_size = 256;
        b->cfg[dim].blocks_per_sm = std::max(1, walk_max_blocks_per_sm(dim, 256));
        b->cfg[dim].n_sm = b->n_sm;
    }
    if (dwos_status s = upload_tables(b)) return bail(s);
    if ((e = cudaEventCreate(&b->ev0)) != cudaSuccess || (e = cudaEventCreate(&b->ev1)) != cudaSuccess)
        return bail(bcuda(b, e, "events"));
    *out = b;
    return DWOS_OK;
}

void dwos_batch_destroy(dwos_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto& ch : b->chunks) { cudaFree(ch.d_probs); cudaFree(ch.d_ctr); }
    cudaFree(b->rec);
    cudaFree(b->trace);
    cudaFree(b->acc);
    cudaFree(b->active);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

const char* dwos_batch_last_error(const dwos_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

dwos_status dwos_batch_run(dwos_batch* b) {
    if (!b) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "batch is NULL");
    BK(cudaSetDevice(b->device), "cudaSetDevice");
    if (dwos_status s = run_walks_only(b, 0)) return s;
    for (size_t i = 0; i < b->jobs.size(); ++i) {
        const dwos_batch_job& j = b->jobs[i];
        const dwos_ctx* c = j.ctx;
        double* acc = b->acc + b->acc_off[i];
        const size_t nvacc = (size_t)c->n_vert * c->dim + c->n_vert;
        double* acc_g = c->dg_vert ? acc + (size_t)c->n_vert * c->dim : nullptr;
        double* usum = acc + nvacc;
        const dwos_record* rec = b->rec + b->rec_off[i];
        BK(cudaMemsetAsync(acc, 0, (nvacc + j.n_query) * sizeof(double), b->stream), "zero accumulators");
        // the scatter also sums u per point and zeroes the gradient the GEMV accumulates into
        BK(launch_scatter(rec, c->elem, c->dim, j.n_query, j.walks_per_point, c->opt.B, 1, j.uref, acc, acc_g, b->stream,
                          nullptr, nullptr, nullptr, b->active + b->active_off[i], usum,
                          c->n_param > 0 ? j.grad_param : nullptr, c->n_param), "scatter");
        if (c->n_param > 0)
            BK(launch_gemv(c->jac, c->dg_vert, acc, acc_g, c->n_vert, c->dim, c->n_param, j.grad_param, b->stream), "gemv");
        BK(launch_loss(usum, j.uref, j.n_query, j.loss, b->stream, nullptr, 1.0 / j.walks_per_point, j.u_mean),
           "loss");
    }
    return DWOS_OK;
}

dwos_status dwos_batch_capture(dwos_batch* b) {
    if (!b) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "batch is NULL");
    BK(cudaSetDevice(b->device), "cudaSetDevice");
    if (!b->stream) return bfail(b, DWOS_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    dwos_status s = dwos_batch_run(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return bcuda(b, e, "end capture");
    b->graph = g;
    BK(cudaGraphInstantiate(&b->exec, g, 0), "instantiate graph");
    return DWOS_OK;
}

dwos_status dwos_batch_launch(dwos_batch* b) {
    if (!b) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "batch is NULL");
    if (!b->exec) return bfail(b, DWOS_ERR_STATE, "no graph: call dwos_batch_capture first");
    BK(cudaSetDevice(b->device), "cudaSetDevice");
    BK(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    return DWOS_OK;
}

dwos_status dwos_batch_autotune(dwos_batch* b, int reps) {
    if (!b) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "batch is NULL");
    BK(cudaSetDevice(b->device), "cudaSetDevice");
    if (reps < 1) reps = 1;
    const int sizes[] = {128, 256};
    for (int dim = 2; dim <= 3; ++dim) {
        bool any = false;
        for (auto& ch : b->chunks) any = any || ch.dim == dim;
        if (!any) continue;
        float best = 1e30f;
        WalkLaunch best_cfg = b->cfg[dim];
        int best_trav = b->trav[dim];
        for (int trav = 0; trav <= 3; ++trav) {
            if ((trav == 2 || trav == 3) && !wide_ok_dim(b, dim)) continue;
            b->trav[dim] = trav;
            if (dwos_status s = upload_tables(b)) return s;
            for (int bs : sizes) {
                const int maxb = std::max(1, walk_max_blocks_per_sm(dim, bs, trav));
                for (int per = 1; per <= maxb; per = per < maxb ? std::min(maxb, per * 2) : maxb + 1) {
                    WalkLaunch L = b->cfg[dim];
                    L.block_size = bs;
                    L.blocks_per_sm = per;
                    L.traversal = trav;
                    const WalkLaunch keep = b->cfg[dim];
                    b->cfg[dim] = L;
                    float t = 0.0f;
                    for (int r = 0; r < reps; ++r) {
                        BK(cudaEventRecord(b->ev0, b->stream), "event");
                        if (dwos_status s = run_walks_only(b, dim)) { b->cfg[dim] = keep; return s; }
                        BK(cudaEventRecord(b->ev1, b->stream), "event");
                        BK(cudaEventSynchronize(b->ev1), "sync");
                        float ms = 0.0f;
                        BK(cudaEventElapsedTime(&ms, b->ev0, b->ev1), "elapsed");
                        t += ms;
                    }
                    b->cfg[dim] = keep;
                    if (t < best) { best = t; best_cfg = L; best_trav = trav; }
                }
            }
        }
        b->cfg[dim] = best_cfg;
        b->trav[dim] = best_trav;
        b->last_walk_ms[dim] = best / reps;
    }
    if (dwos_status s = upload_tables(b)) return s;
    if (b->exec) return dwos_batch_capture(b);
    return DWOS_OK;
}

dwos_status dwos_batch_config(const dwos_batch* b, int dim, int* block_size, int* blocks_per_sm, int* traversal,
                              float* walk_ms) {
    if (!b || (dim != 2 && dim != 3)) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "bad arguments");
    if (block_size) *block_size = b->cfg[dim].block_size;
    if (blocks_per_sm) *blocks_per_sm = b->cfg[dim].blocks_per_sm;
    if (traversal) *traversal = b->trav[dim];
    if (walk_ms) *walk_ms = b->last_walk_ms[dim];
    return DWOS_OK;
}

dwos_status dwos_batch_trace(dwos_batch* b, int enable) {
    if (!b) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "batch is NULL");
    BK(cudaSetDevice(b->device), "cudaSetDevice");
    BK(cudaStreamSynchronize(b->stream), "synchronize");
    if (enable && !b->trace) {
        size_t n = 0;
        b->trace_off.clear();
        for (auto& j : b->jobs) {
            b->trace_off.push_back(n);
            n += (size_t)j.n_query * j.walks_per_point * (size_t)(j.ctx->opt.K + 1);
        }
        BK(cudaMalloc(&b->trace, sizeof(uint32_t) * std::max<size_t>(n, 1)), "alloc traces");
        BK(cudaMemset(b->trace, 0xff, sizeof(uint32_t) * std::max<size_t>(n, 1)), "init traces");
    } else if (!enable && b->trace) {
        cudaFree(b->trace);
        b->trace = nullptr;
    }
    if (dwos_status s = upload_tables(b)) return s;
    if (b->exec) return dwos_batch_capture(b);
    return DWOS_OK;
}

dwos_status dwos_batch_records(dwos_batch* b, int job, dwos_record* records, uint32_t* trace, int mem) {
    if (!b) return bfail(nullptr, DWOS_ERR_INVALID_ARG, "batch is NULL");
    if (job < 0 || job >= (int)b->jobs.size()) return bfail(b, DWOS_ERR_INVALID_ARG, "job index out of range");
    if (mem != DWOS_MEM_HOST && mem != DWOS_MEM_DEVICE) return bfail(b, DWOS_ERR_INVALID_ARG, "bad mem flag");
    if (!records) return bfail(b, DWOS_ERR_INVALID_ARG, "records is NULL");
    if (trace && !b->trace) return bfail(b, DWOS_ERR_STATE, "traces are off: call dwos_batch_trace(b, 1) first");
    BK(cudaSetDevice(b->device), "cudaSetDevice");
    const dwos_batch_job& j = b->jobs[job];
    const size_t n = (size_t)j.n_query * j.walks_per_point;
    const cudaMemcpyKind k = mem == DWOS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    BK(cudaMemcpyAsync(records, b->rec + b->rec_off[job], sizeof(dwos_record) * n, k, b->stream), "copy records");
    if (trace)
        BK(cudaMemcpyAsync(trace, b->trace + b->trace_off[job], sizeof(uint32_t) * n * (j.ctx->opt.K + 1), k,
                           b->stream), "copy traces");
    BK(cudaStreamSynchronize(b->stream), "synchronize");
    return DWOS_OK;
}

dwos_status dwos_batch_stats(dwos_batch* b, dwos_run_stats* out) {
    if (!b || !out) return bfail(b, DWOS_ERR_INVALID_ARG, "NULL argument");
    BK(cudaSetDevice(b->device), "cudaSetDevice");
    BK(cudaStreamSynchronize(b->stream), "synchronize");
    std::memset(out, 0, sizeof(*out));
    for (auto& ch : b->chunks) {
        DevCounters c;
        BK(cudaMemcpy(&c, ch.d_ctr, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
        out->steps_main += c.steps_main;
        out->steps_nested += c.steps_nested;
        out->walks += std::min<unsigned long long>(c.next_work, ch.total);
        out->capped += c.capped;
        out->nodes_visited += c.nodes;
        out->prims_tested += c.prims;
        out->wide_nodes_visited += c.wnodes;
        if (c.error & 4) return bfail(b, DWOS_ERR_INVALID_ARG, "a query point is not finite");
        if (c.error & 1) return bfail(b, DWOS_ERR_STEP_LIMIT, "BVH traversal exceeded its iteration bound");
    }
    return DWOS_OK;
}

}  // extern "C"
