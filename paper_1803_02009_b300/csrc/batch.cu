// batch.cu -- many independent registration problems per Gauss-Newton
// iteration (each problem is one frame of the method of Sec. II: its own
// model, node graph and depth map).
//
// One batched iteration: the per-problem kernels up to the normal equations
// (association, residuals, assembly, block inverses) run on a set of
// internal streams forked from the caller's stream; the PCG solves of a group
// of problems run as ONE persistent cooperative launch in which every problem
// owns a contiguous range of CTAs, its own grid barrier and its own partial
// sums; then the per-problem updates run forked again.  The iteration can be
// captured into a CUDA graph and replayed (one graph launch per iteration,
// or per several iterations).  The schedule -- PCG threads per CTA (node rows
// per pass), problems per persistent launch (CTAs per problem) and the
// number of streams -- is picked by a measuring autotuner (ed_batch_autotune).
#include <algorithm>
#include <vector>

#include "ed_internal.cuh"

#define ED_MAX_BATCH 64

struct ed_batch {
    int count;
    ed_context *ctx[ED_MAX_BATCH];
    ed_batch_schedule sched;
    int n_groups;
    int group_first[ED_MAX_BATCH + 1];         // into member[]
    int member[ED_MAX_BATCH];                  // problems ordered by group
    ed_pcg_batch_plan_t plan[ED_MAX_BATCH];    // per group
    cudaStream_t side[ED_MAX_BATCH];
    cudaEvent_t ev_fork;
    cudaEvent_t ev_join[ED_MAX_BATCH];
    cudaGraphExec_t exec;
    unsigned long long graph_kernels;
    char *save;                                // autotuner copies of x, x_master, pose
    size_t save_bytes;
    int num_sms;
};

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

static size_t save_need(ed_context *const *ctxs, int count)
{
    size_t b = 0;
    for (int p = 0; p < count; ++p) b += align256(48 * (size_t)ctxs[p]->m) + align256(96 * (size_t)ctxs[p]->m) + 256;
    return b;
}

// groups of problems sharing one persistent launch: problems sorted by stored
// blocks and dealt out in snake order so that every group gets a similar load
static ed_status batch_plan(ed_batch *b, const ed_batch_schedule &s)
{
    const int count = b->count;
    if ((s.pcg_threads != 256 && s.pcg_threads != 512) || s.problems_per_launch < 1 ||
        s.problems_per_launch > ED_MAX_BATCH_LAUNCH || s.streams < 1 ||
        (s.asm_blocks_per_warp != 1 && s.asm_blocks_per_warp != 2) || (s.point_chunk != 256 && s.point_chunk != 512))
        return ED_ERR_ARG;
    // the row starts of a batched launch are rewritten below: nothing may run
    if (cudaDeviceSynchronize() != cudaSuccess) return ED_ERR_CUDA;
    const int ppl = std::min(s.problems_per_launch, count);
    const int ng = (count + ppl - 1) / ppl;
    std::vector<int> order(count);
    for (int p = 0; p < count; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->ctx[a]->nnzb > b->ctx[c]->nnzb; });
    std::vector<std::vector<int>> groups(ng);
    for (int i = 0; i < count; ++i) {
        const int round = i / ng, pos = i % ng;
        groups[(round & 1) ? ng - 1 - pos : pos].push_back(order[i]);
    }
    const int grid_total = b->num_sms * (512 / s.pcg_threads);
    int k = 0;
    for (int g = 0; g < ng; ++g) {
        b->group_first[g] = k;
        ed_context *gc[ED_MAX_BATCH_LAUNCH];
        for (size_t i = 0; i < groups[g].size(); ++i) {
            b->member[k + (int)i] = groups[g][i];
            gc[i] = b->ctx[groups[g][i]];
        }
        ed_status st = ed_pcg_batch_plan(gc, (int)groups[g].size(), s.pcg_threads, grid_total, &b->plan[g]);
        if (st != ED_OK) return st;
        k += (int)groups[g].size();
    }
    b->group_first[ng] = k;
    b->n_groups = ng;
    for (int p = 0; p < count; ++p) {   // the assembly and point-pass schedule of every member
        b->ctx[p]->asm_pairs = s.asm_blocks_per_warp;
        b->ctx[p]->pt_chunk = s.point_chunk;
    }
    b->sched = s;
    b->sched.problems_per_launch = ppl;
    b->sched.streams = std::min(s.streams, count);
    return ED_OK;
}

static ed_stats *stat_at(ed_stats *const *stats, int p, int it)
{
    return (stats && stats[p]) ? stats[p] + it : nullptr;
}

// one batched Gauss-Newton iteration enqueued on st (stats[p] + it receives
// problem p's statistics)
static ed_status batch_enqueue(ed_batch *b, const ed_frame *frames, const ed_solver_params *params, float *const *x,
                               double *const *xm, double *const *pose, ed_stats *const *stats, int it, cudaStream_t st)
{
    const int count = b->count, W = b->sched.streams;
    for (int p = 0; p < count; ++p)
        if (params[p].precision != params[0].precision) return ED_ERR_ARG;
    ed_status first = ED_OK;
    auto fork = [&]() -> ed_status {
        ED_CUDA_TRY(cudaEventRecord(b->ev_fork, st));
        for (int i = 0; i < W; ++i) ED_CUDA_TRY(cudaStreamWaitEvent(b->side[i], b->ev_fork, 0));
        return ED_OK;
    };
    auto join = [&]() -> ed_status {
        ed_status r = ED_OK;
        for (int i = 0; i < W; ++i) {
            if (cudaEventRecord(b->ev_join[i], b->side[i]) != cudaSuccess ||
                cudaStreamWaitEvent(st, b->ev_join[i], 0) != cudaSuccess)
                r = ED_ERR_CUDA;
        }
        return r;
    };
    ed_status s = fork();
    if (s != ED_OK) return s;
    for (int p = 0; p < count && first == ED_OK; ++p)
        first = ed_gn_pre(b->ctx[p], &frames[p], &params[p], x[p], xm ? xm[p] : nullptr, pose[p],
                          stat_at(stats, p, it), b->side[p % W], false);
    s = join();   // always rejoin, also after an error (a capture must not end forked)
    if (first != ED_OK) return first;
    if (s != ED_OK) return s;
    for (int g = 0; g < b->n_groups; ++g) {
        const int k0 = b->group_first[g], n = b->group_first[g + 1] - k0;
        ed_context *gc[ED_MAX_BATCH_LAUNCH];
        const ed_solver_params *gp[ED_MAX_BATCH_LAUNCH];
        ed_stats *gs[ED_MAX_BATCH_LAUNCH];
        float *gx[ED_MAX_BATCH_LAUNCH];
        double *gxm[ED_MAX_BATCH_LAUNCH], *gpose[ED_MAX_BATCH_LAUNCH];
        for (int i = 0; i < n; ++i) {
            const int p = b->member[k0 + i];
            gc[i] = b->ctx[p];
            gp[i] = &params[p];
            gs[i] = stat_at(stats, p, it);
            gx[i] = x[p];
            gxm[i] = xm ? xm[p] : nullptr;
            gpose[i] = pose[p];
        }
        if ((s = ed_pcg_solve_batch(gc, &b->plan[g], gp, gx, gxm, gpose, gs, st)) != ED_OK) return s;
    }
    for (int p = 0; p < count; ++p) ed_gn_post(b->ctx[p]);
    return ED_OK;
}

static ed_status check_args(const ed_batch *b, const ed_frame *frames, const ed_solver_params *params,
                            float *const *x, double *const *pose)
{
    if (!b || !frames || !params || !x || !pose) return ED_ERR_ARG;
    for (int p = 0; p < b->count; ++p)
        if (!x[p] || !pose[p]) return ED_ERR_ARG;
    return ED_OK;
}

extern "C" ed_status ed_batch_query_workspace(ed_context *const *ctxs, int count, size_t *bytes)
{
    if (!ctxs || !bytes || count < 1 || count > ED_MAX_BATCH) return ED_ERR_ARG;
    for (int p = 0; p < count; ++p) {
        if (!ctxs[p]) return ED_ERR_ARG;
        ed_status s = ed_graph_ready(ctxs[p], 0);
        if (s != ED_OK) return s;
    }
    ED_CUDA_TRY(cudaStreamSynchronize(0));   // (the plans' copies on the legacy stream)
    *bytes = save_need(ctxs, count);
    return ED_OK;
}

extern "C" ed_status ed_batch_destroy(ed_batch *b)
{
    if (!b) return ED_ERR_ARG;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (int i = 0; i < b->count; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
    return ED_OK;
}

extern "C" ed_status ed_batch_create(ed_context *const *ctxs, int count, void *workspace, size_t workspace_bytes,
                                     ed_batch **out)
{
    size_t need = 0;
    ed_status s = ed_batch_query_workspace(ctxs, count, &need);
    if (s != ED_OK) return s;
    if (!out || !workspace || ((uintptr_t)workspace & 255)) return ED_ERR_ARG;
    if (workspace_bytes < need) return ED_ERR_CAPACITY;
    for (int p = 0; p < count; ++p)
        for (int q = 0; q < p; ++q)
            if (ctxs[p] == ctxs[q]) return ED_ERR_ARG;   // a context holds one problem's state
    ed_batch *b = new ed_batch();
    b->count = count;
    for (int p = 0; p < count; ++p) b->ctx[p] = ctxs[p];
    b->save = (char *)workspace;
    b->save_bytes = workspace_bytes;
    b->num_sms = ctxs[0]->num_sms;
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
        ed_batch_destroy(b);
        return ED_ERR_CUDA;
    }
    for (int i = 0; i < count; ++i) {
        if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming) != cudaSuccess) {
            ed_batch_destroy(b);
            return ED_ERR_CUDA;
        }
    }
    // default schedule: 512-thread PCG CTAs, as many problems per launch as fit
    ed_batch_schedule d;
    d.pcg_threads = 512;
    d.streams = std::min(count, 16);
    d.asm_blocks_per_warp = 2;
    d.point_chunk = 512;
    s = ED_ERR_CAPACITY;
    for (int ppl = std::min(count, ED_MAX_BATCH_LAUNCH); ppl >= 1 && s == ED_ERR_CAPACITY; ppl = ppl > 1 ? ppl / 2 : 0) {
        d.problems_per_launch = ppl;
        s = batch_plan(b, d);
        if (ppl == 1) break;
    }
    if (s != ED_OK) {
        ed_batch_destroy(b);
        return s;
    }
    *out = b;
    return ED_OK;
}

extern "C" ed_status ed_batch_set_schedule(ed_batch *b, const ed_batch_schedule *s)
{
    if (!b || !s) return ED_ERR_ARG;
    const ed_batch_schedule old = b->sched;
    ed_status r = batch_plan(b, *s);
    if (r != ED_OK) batch_plan(b, old);   // keep the previous, valid plan
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);   // a captured graph belongs to the old plan
        b->exec = nullptr;
    }
    return r;
}

extern "C" ed_status ed_batch_get_schedule(const ed_batch *b, ed_batch_schedule *s)
{
    if (!b || !s) return ED_ERR_ARG;
    *s = b->sched;
    return ED_OK;
}

extern "C" ed_status ed_batch_gn_step(ed_batch *b, const ed_frame *frames, const ed_solver_params *params,
                                      float *const *x, double *const *x_master, double *const *pose,
                                      ed_stats *const *stats, cudaStream_t st)
{
    ed_status s = check_args(b, frames, params, x, pose);
    if (s != ED_OK) return s;
    return batch_enqueue(b, frames, params, x, x_master, pose, stats, 0, st);
}

static ed_status batch_capture(ed_batch *b, const ed_frame *frames, const ed_solver_params *params, float *const *x,
                               double *const *xm, double *const *pose, ed_stats *const *stats, int n_iters,
                               cudaStream_t st, cudaGraphExec_t *exec_out, unsigned long long *kernels)
{
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) {
        fprintf(stderr, "libed: a CUDA graph cannot be captured on the default stream; pass a created stream\n");
        return ED_ERR_ARG;
    }
    int tm_saved[ED_MAX_BATCH];
    for (int p = 0; p < b->count; ++p) {
        tm_saved[p] = b->ctx[p]->tm_kernel;
        b->ctx[p]->tm_kernel = -1;   // no timing events inside a graph
    }
    unsigned long long l0 = 0, l1 = 0;
    ed_launch_count(&l0);
    cudaGraph_t graph = nullptr;
    ed_status s = ED_OK;
    cudaError_t eb = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (eb != cudaSuccess) {
        fprintf(stderr, "libed: cudaStreamBeginCapture failed: %s\n", cudaGetErrorString(eb));
        s = ED_ERR_CUDA;
    }
    for (int it = 0; it < n_iters && s == ED_OK; ++it) s = batch_enqueue(b, frames, params, x, xm, pose, stats, it, st);
    const cudaError_t ec = eb == cudaSuccess ? cudaStreamEndCapture(st, &graph) : cudaSuccess;   // always end it
    if (s == ED_OK && ec != cudaSuccess) {
        fprintf(stderr, "libed: cudaStreamEndCapture failed: %s\n", cudaGetErrorString(ec));
        s = ED_ERR_CUDA;
    }
    ed_launch_count(&l1);
    for (int p = 0; p < b->count; ++p) b->ctx[p]->tm_kernel = tm_saved[p];
    if (s == ED_OK) {
        const cudaError_t ei = cudaGraphInstantiate(exec_out, graph, 0);
        if (ei != cudaSuccess) {
            fprintf(stderr, "libed: cudaGraphInstantiate failed: %s\n", cudaGetErrorString(ei));
            s = ED_ERR_CUDA;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (s != ED_OK) {
        cudaGetLastError();
        fprintf(stderr, "libed: batch capture failed (%s)\n", ed_status_string(s));
        return s;
    }
    *kernels = l1 - l0;
    return ED_OK;
}

extern "C" ed_status ed_batch_capture(ed_batch *b, const ed_frame *frames, const ed_solver_params *params,
                                      float *const *x, double *const *x_master, double *const *pose,
                                      ed_stats *const *stats, int n_iters, cudaStream_t st)
{
    ed_status s = check_args(b, frames, params, x, pose);
    if (s != ED_OK) return s;
    if (n_iters < 1) return ED_ERR_ARG;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return batch_capture(b, frames, params, x, x_master, pose, stats, n_iters, st, &b->exec, &b->graph_kernels);
}

extern "C" ed_status ed_batch_launch(ed_batch *b, cudaStream_t st)
{
    if (!b) return ED_ERR_ARG;
    if (!b->exec) return ED_ERR_STATE;
    ED_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    ed_note_launches(b->graph_kernels);
    return ED_OK;
}

// copies of every problem's x, x_master and pose (save = true) or back
static ed_status batch_save(ed_batch *b, float *const *x, double *const *xm, double *const *pose, bool save,
                            cudaStream_t st)
{
    char *q = b->save;
    for (int p = 0; p < b->count; ++p) {
        const size_t m = b->ctx[p]->m;
        char *sx = q, *sxm = q + align256(48 * m), *sp = sxm + align256(96 * m);
        q = sp + 256;
        if (save) {
            ED_CUDA_TRY(cudaMemcpyAsync(sx, x[p], 48 * m, cudaMemcpyDeviceToDevice, st));
            if (xm && xm[p]) ED_CUDA_TRY(cudaMemcpyAsync(sxm, xm[p], 96 * m, cudaMemcpyDeviceToDevice, st));
            ED_CUDA_TRY(cudaMemcpyAsync(sp, pose[p], 48, cudaMemcpyDeviceToDevice, st));
        } else {
            ED_CUDA_TRY(cudaMemcpyAsync(x[p], sx, 48 * m, cudaMemcpyDeviceToDevice, st));
            if (xm && xm[p]) ED_CUDA_TRY(cudaMemcpyAsync(xm[p], sxm, 96 * m, cudaMemcpyDeviceToDevice, st));
            ED_CUDA_TRY(cudaMemcpyAsync(pose[p], sp, 48, cudaMemcpyDeviceToDevice, st));
        }
    }
    return ED_OK;
}

// Times schedules as captured one-iteration graphs, the problems' x, x_master
// and pose restored after each run, and keeps the fastest: first every
// feasible PCG schedule (threads 512 / 256; problems per launch 1, 2, 4, ...
// up to all; 4 or up to 16 streams) with the default assembly, then, with the
// best of those, the assembly and point-pass schedules (off-diagonal blocks
// per warp 2 / 1, points per CTA 512 / 256).  Any graph captured before is
// dropped.
extern "C" ed_status ed_batch_autotune(ed_batch *b, const ed_frame *frames, const ed_solver_params *params,
                                       float *const *x, double *const *x_master, double *const *pose,
                                       ed_stats *const *stats, cudaStream_t st, ed_batch_schedule *chosen,
                                       float *best_ms)
{
    ed_status s = check_args(b, frames, params, x, pose);
    if (s != ED_OK) return s;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const ed_batch_schedule orig = b->sched;
    std::vector<ed_batch_schedule> cands;
    const int nt_opts[2] = {512, 256};
    std::vector<int> ppl_opts;
    for (int v = 1; v < b->count; v *= 2) ppl_opts.push_back(v);
    ppl_opts.push_back(std::min(b->count, ED_MAX_BATCH_LAUNCH));
    std::vector<int> str_opts = {std::min(b->count, 4)};
    if (std::min(b->count, 16) != str_opts[0]) str_opts.push_back(std::min(b->count, 16));
    for (int nt : nt_opts)
        for (int ppl : ppl_opts)
            for (int w : str_opts) {
                ed_batch_schedule c;
                c.pcg_threads = nt;
                c.problems_per_launch = ppl;
                c.streams = w;
                c.asm_blocks_per_warp = 2;
                c.point_chunk = 512;
                cands.push_back(c);
            }
    cudaEvent_t e0, e1;
    ED_CUDA_TRY(cudaEventCreate(&e0));
    ED_CUDA_TRY(cudaEventCreate(&e1));
    if ((s = batch_save(b, x, x_master, pose, true, st)) != ED_OK) return s;
    float best = -1.f;
    ed_batch_schedule best_s = orig;
    for (int stage = 0; stage < 2 && s == ED_OK; ++stage) {
        if (stage == 1) {   // the assembly and point-pass options on the best PCG schedule
            if (best < 0.f) break;
            cands.clear();
            for (int bpw = 2; bpw >= 1; --bpw)
                for (int ch = 512; ch >= 256; ch /= 2) {
                    if (bpw == best_s.asm_blocks_per_warp && ch == best_s.point_chunk) continue;
                    ed_batch_schedule c = best_s;
                    c.asm_blocks_per_warp = bpw;
                    c.point_chunk = ch;
                    cands.push_back(c);
                }
        }
        for (const ed_batch_schedule &c : cands) {
            if (batch_plan(b, c) != ED_OK) continue;   // infeasible: a CTA share does not fit
            cudaGraphExec_t ex = nullptr;
            unsigned long long nk = 0;
            if (batch_capture(b, frames, params, x, x_master, pose, stats, 1, st, &ex, &nk) != ED_OK) continue;
            float ms = -1.f;
            bool ok = cudaGraphLaunch(ex, st) == cudaSuccess;                     // warm-up
            ok = ok && batch_save(b, x, x_master, pose, false, st) == ED_OK;
            ok = ok && cudaEventRecord(e0, st) == cudaSuccess && cudaGraphLaunch(ex, st) == cudaSuccess &&
                 cudaEventRecord(e1, st) == cudaSuccess;
            ok = ok && batch_save(b, x, x_master, pose, false, st) == ED_OK;
            ok = ok && cudaStreamSynchronize(st) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            ed_note_launches(2 * nk);
            cudaGraphExecDestroy(ex);
            if (!ok) {
                s = ED_ERR_CUDA;
                break;
            }
            if (best < 0.f || ms < best) {
                best = ms;
                best_s = b->sched;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != ED_OK) {
        batch_plan(b, orig);
        return s;
    }
    if (best < 0.f) {
        batch_plan(b, orig);
        return ED_ERR_CAPACITY;
    }
    if ((s = batch_plan(b, best_s)) != ED_OK) return s;
    if (chosen) *chosen = b->sched;
    if (best_ms) *best_ms = best;
    return ED_OK;
}
