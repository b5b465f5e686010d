// C ABI of the IFGF library: argument checks, plan lifetime, host/device pointer
// handling and introspection.  All numerical work is in ifgf_plan.cu and the
// ifgf_apply_*.cu kernels.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ifgf_device.cuh"

cudaError_t ifgf_run_typed_f64(const PlanDev &pd, int nrhs, const void *in_user, void *out_user,
                               void *in_sorted, void *out_sorted, int mode, int adjoint, cudaStream_t st,
                               StageTimer &tm);
cudaError_t ifgf_run_typed_f32(const PlanDev &pd, int nrhs, const void *in_user, void *out_user,
                               void *in_sorted, void *out_sorted, int mode, int adjoint, cudaStream_t st,
                               StageTimer &tm);

cudaError_t ifgf_run_batched(const PlanDev &pd, int nrhs, const void *in_user, void *out_user, void *in_sorted,
                             void *out_sorted, int mode, cudaStream_t st, StageTimer &tm);
cudaError_t ifgf_batched_prepare();
// shared-memory limits of the FP32 run kernels (one per translation unit that holds them)
cudaError_t ifgf_prepare_runs_r1();
cudaError_t ifgf_prepare_runs_r4();
cudaError_t ifgf_batched_autotune(PlanDev &pd, int nrhs, const void *sig, void *us, cudaStream_t st, int reps,
                                  float *ms);

static thread_local std::string g_create_error;

static bool is_device_pointer(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Drops the plan's captured evaluations (their kernels hold a copy of the plan's device
// description, which is stale once it changes).
static void graphs_clear(ifgf_plan *p)
{
    for (auto &g : p->graphs) cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
}

static void free_plan(ifgf_plan *p)
{
    graphs_clear(p);
    if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
    for (int i = 0; i < StageTimer::kMax; ++i)
        if (p->timer.ev[i]) cudaEventDestroy(p->timer.ev[i]);
    for (void *ptr : p->allocs) cudaFree(ptr);
    p->allocs.clear();
    delete p;
}

// Default leaf cones: (1, 2) for leaves up to a quarter wavelength (the setting of
// the paper's Sec. 4 experiments), doubled per doubling of H_D / (lambda / 4).
static void default_leaf_cones(double kappa, double HD, int *ns, int *nc)
{
    int m = 0;
    if (kappa > 0) {
        double lambda = 2.0 * M_PI / kappa;
        double ratio = HD / (0.25 * lambda);
        if (ratio > 1.0) m = (int)std::lround(std::log2(ratio));
    }
    if (m > 10) m = 10;
    *ns = 1 << m;
    *nc = 2 << m;
}

extern "C" ifgf_status ifgf_plan_create(const double *points, int64_t n, double kappa, int levels,
                                        int p_radial, int p_angular, const ifgf_options *opt,
                                        void *stream, ifgf_plan **out)
{
    NvtxRange range("ifgf_plan_create");
    if (out) *out = nullptr;
    g_create_error.clear();
    if (!points || !out) { g_create_error = "NULL argument"; return IFGF_EINVAL; }
    if (n < 2 || n >= ((int64_t)1 << 31) - 1) { g_create_error = "N must be in [2, 2^31)"; return IFGF_EINVAL; }
    if (!(kappa >= 0.0) || !std::isfinite(kappa)) { g_create_error = "kappa must be finite and >= 0"; return IFGF_EINVAL; }
    if (levels < 3 || levels > IFGF_MAX_LEVELS) { g_create_error = "levels must be in [3, 20]"; return IFGF_EINVAL; }
    if (!((p_radial == 3 && p_angular == 5) || (p_radial == 4 && p_angular == 7))) {
        g_create_error = "supported (P_s, P_ang): (3, 5) and (4, 7)";
        return IFGF_EINVAL;
    }

    ifgf_options o = {0, 0, 1, IFGF_FP64, 0, 0, 0.0, 0};
    if (opt) o = *opt;
    if (o.value_budget_bytes < 0) { g_create_error = "value_budget_bytes must be >= 0"; return IFGF_EINVAL; }
    if (!(o.timeout_s >= 0.0)) { g_create_error = "timeout_s must be >= 0"; return IFGF_EINVAL; }
    if (o.max_nrhs <= 0) o.max_nrhs = 1;
    if (o.max_nrhs > 1024) { g_create_error = "max_nrhs must be <= 1024"; return IFGF_EINVAL; }
    if (o.precision != IFGF_FP64 && o.precision != IFGF_MIXED && !ifgf_is_batched(o.precision)) {
        g_create_error = "unknown precision";
        return IFGF_EINVAL;
    }
    if (o.leaf_ns < 0 || o.leaf_nc < 0 || o.leaf_ns > 1024 || o.leaf_nc > 1024) {
        g_create_error = "leaf cone counts out of range";
        return IFGF_EINVAL;
    }
    if (o.leaf_max < 0) { g_create_error = "leaf_max must be >= 0"; return IFGF_EINVAL; }
    if (o.leaf_max > 0 && ifgf_is_batched(o.precision)) {
        g_create_error = "adaptive trees (leaf_max > 0) are supported by IFGF_FP64 and IFGF_MIXED plans";
        return IFGF_EINVAL;
    }
    ifgf_plan *p = new (std::nothrow) ifgf_plan();
    if (!p) { g_create_error = "host allocation failed"; return IFGF_ENOMEM; }
    p->n = n;
    p->D = levels;
    p->Ps = p_radial;
    p->Pang = p_angular;
    p->P = p_radial * p_angular * p_angular;
    p->kappa = kappa;
    p->precision = o.precision;
    p->max_nrhs = o.max_nrhs;
    p->flags = o.flags;
    p->dev.flags = o.flags;
    p->leaf_max = o.leaf_max;
    p->dev.batched_f16 = o.precision == IFGF_BATCHED_FP16 ? 1 : 0;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        g_create_error = "no CUDA device";
        return IFGF_ECUDA;
    }
    p->timeout_s = o.timeout_s;
    p->value_budget = (size_t)o.value_budget_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    p->build_stream = st;
    // leaf cones need H_D, known only after the root cube: the builder reads lh[D]
    // and a non-positive entry means "default"
    p->lh[levels].ns = o.leaf_ns;
    p->lh[levels].nc = o.leaf_nc;
    if (o.leaf_ns == 0 || o.leaf_nc == 0) {
        // the root cube is the bounding cube of the points; compute its side on the
        // host only for this default (the builder recomputes it on the GPU)
        std::vector<double> h;
        const double *hp = points;
        if (is_device_pointer(points)) {
            h.resize((size_t)n * 3);
            if (cudaMemcpy(h.data(), points, h.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
                g_create_error = "copy of points failed";
                delete p;
                return IFGF_ECUDA;
            }
            hp = h.data();
        }
        double lo[3] = {hp[0], hp[1], hp[2]}, hi[3] = {hp[0], hp[1], hp[2]};
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) {
                lo[c] = std::min(lo[c], hp[3 * i + c]);
                hi[c] = std::max(hi[c], hp[3 * i + c]);
            }
        double H1 = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
        int ns, nc;
        default_leaf_cones(kappa, std::ldexp(H1, -(levels - 1)), &ns, &nc);
        if (o.leaf_ns == 0) p->lh[levels].ns = ns;
        if (o.leaf_nc == 0) p->lh[levels].nc = nc;
    }
    ifgf_status s = ifgf_build_plan(p, points, st);
    // batched plans group evaluations by source cone with the transpose lists
    if (s == IFGF_OK && ((o.flags & 1) || ifgf_is_batched(o.precision))) s = ifgf_build_adjoint_lists(p, st);
    if (s == IFGF_OK && ifgf_is_batched(o.precision) && ifgf_batched_prepare() != cudaSuccess) {
        cudaGetLastError();
        p->last_error = "shared-memory limit of the tensor-core kernel";
        s = IFGF_ECUDA;
    }
    if (s == IFGF_OK && o.precision != IFGF_FP64 &&
        (ifgf_prepare_runs_r1() != cudaSuccess || ifgf_prepare_runs_r4() != cudaSuccess)) {
        cudaGetLastError();
        p->last_error = "shared-memory limit of the run kernel";
        s = IFGF_ECUDA;
    }
    if (s != IFGF_OK) {
        g_create_error = p->last_error;
        cudaStreamSynchronize(st);
        cudaGetLastError();
        free_plan(p);
        return s;
    }
    *out = p;
    return IFGF_OK;
}

// Host-side wait for the work queued on st, bounded by the plan's timeout_s: past it
// the call reports IFGF_ETIMEOUT and leaves the queued work to complete on its own.
// Flags bit 7 (testing) makes the device look unfinished.
static ifgf_status wait_stream(ifgf_plan *p, cudaStream_t st)
{
    const bool fake = (p->flags & 128) != 0;
    if (p->timeout_s <= 0.0 && !fake) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            p->last_error = std::string("stream synchronisation failed: ") + cudaGetErrorString(e);
            return IFGF_ECUDA;
        }
        return IFGF_OK;
    }
    const double limit = p->timeout_s > 0.0 ? p->timeout_s : 0.05;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ev, st) != cudaSuccess) {
        p->last_error = "event creation failed";
        return IFGF_ECUDA;
    }
    const auto t0 = std::chrono::steady_clock::now();
    ifgf_status s = IFGF_OK;
    for (;;) {
        const cudaError_t q = fake ? cudaErrorNotReady : cudaEventQuery(ev);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) {
            p->last_error = std::string("device error while waiting: ") + cudaGetErrorString(q);
            s = IFGF_ECUDA;
            break;
        }
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > limit) {
            p->last_error = "timed out waiting for the device";
            s = IFGF_ETIMEOUT;
            break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaEventDestroy(ev);
    return s;
}

// Queues the launches of one evaluation on st (device buffers in the caller's order):
// right-hand sides in chunks of at most rhs_chunk, a chunk being a contiguous block of
// rows of the [nrhs][N] arrays.  Launches only: no host synchronisation, so that the
// sequence can be captured into a CUDA graph.
static cudaError_t launch_evaluation(ifgf_plan *p, const void *din, void *dout, int nrhs, int mode, int adjoint,
                                     cudaStream_t st)
{
    const size_t eb = ifgf_elem_bytes(p->precision);
    cudaError_t e = cudaSuccess;
    for (int c0 = 0; c0 < nrhs && e == cudaSuccess; c0 += p->rhs_chunk) {
        const int nc = std::min(p->rhs_chunk, nrhs - c0);
        const void *cin = (const char *)din + (size_t)c0 * p->n * eb;
        void *cout = (char *)dout + (size_t)c0 * p->n * eb;
        if (p->precision == IFGF_FP64)
            e = ifgf_run_typed_f64(p->dev, nc, cin, cout, p->sig_sorted, p->u_sorted, mode, adjoint, st, p->timer);
        else if (ifgf_is_batched(p->precision) && !adjoint && nc % 2 == 0 && nc <= ifgf_batched_max_nrhs(p->Ps))
            e = ifgf_run_batched(p->dev, nc, cin, cout, p->sig_sorted, p->u_sorted, mode, st, p->timer);
        else
            e = ifgf_run_typed_f32(p->dev, nc, cin, cout, p->sig_sorted, p->u_sorted, mode, adjoint, st, p->timer);
    }
    return e;
}

// Replays the captured graph of this evaluation on st, capturing it first if needed (on
// the plan's own capture stream: capture does not run anything, and the caller's stream
// may be the legacy default stream, which cannot be captured).  At most kMaxGraphs are
// kept; the least recently used is dropped.
static ifgf_status replay_graph(ifgf_plan *p, const void *din, void *dout, int nrhs, int mode, int adjoint,
                                cudaStream_t st)
{
    const bool timed = p->timer.on;
    ifgf_plan::GraphEntry *g = nullptr;
    for (auto &x : p->graphs)
        if (x.in == din && x.out == dout && x.nrhs == nrhs && x.mode == mode && x.adjoint == adjoint &&
            x.timed == timed)
            g = &x;
    if (!g) {
        if (!p->capture_stream && cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            p->last_error = "capture stream creation failed";
            return IFGF_ECUDA;
        }
        if (cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            p->last_error = "graph capture could not start";
            return IFGF_ECUDA;
        }
        p->timer.n = 0;
        p->timer.external = true;
        const cudaError_t le = launch_evaluation(p, din, dout, nrhs, mode, adjoint, p->capture_stream);
        p->timer.external = false;
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(p->capture_stream, &graph);
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie =
            (le == cudaSuccess && ce == cudaSuccess) ? cudaGraphInstantiate(&exec, graph, 0) : cudaErrorUnknown;
        if (graph) cudaGraphDestroy(graph);
        if (le != cudaSuccess || ce != cudaSuccess || ie != cudaSuccess) {
            cudaGetLastError();
            p->last_error = std::string("graph capture failed: ") +
                            cudaGetErrorString(le != cudaSuccess ? le : ce != cudaSuccess ? ce : ie);
            return IFGF_ECUDA;
        }
        if ((int)p->graphs.size() >= ifgf_plan::kMaxGraphs) {
            size_t lru = 0;
            for (size_t i = 1; i < p->graphs.size(); ++i)
                if (p->graphs[i].used < p->graphs[lru].used) lru = i;
            cudaGraphExecDestroy(p->graphs[lru].exec);
            p->graphs.erase(p->graphs.begin() + lru);
        }
        ifgf_plan::GraphEntry ne{din, dout, nrhs, mode, adjoint, timed, exec, 0, p->timer.n, {}, {}};
        ne.tstage.assign(p->timer.stage, p->timer.stage + p->timer.n);
        ne.tlaunch.assign(p->timer.launches, p->timer.launches + p->timer.n);
        p->graphs.push_back(std::move(ne));
        g = &p->graphs.back();
        ++p->graph_captures;
    }
    g->used = ++p->graph_clock;
    // the marks this replay records, for the caller's attribution of stage times
    p->timer.n = g->tn;
    for (int i = 0; i < g->tn; ++i) {
        p->timer.stage[i] = g->tstage[i];
        p->timer.launches[i] = g->tlaunch[i];
    }
    if (cudaGraphLaunch(g->exec, st) != cudaSuccess) {
        cudaGetLastError();
        p->last_error = "graph launch failed";
        return IFGF_ECUDA;
    }
    ++p->graph_replays;
    return IFGF_OK;
}

ifgf_status ifgf_run_apply(ifgf_plan *p, const void *in, void *out, int nrhs, int mode, int adjoint,
                           cudaStream_t st)
{
    NvtxRange range(adjoint ? "ifgf_apply_adjoint" : "ifgf_apply");
    if (!p || !in || !out) return IFGF_EINVAL;
    if (nrhs < 1 || nrhs > p->max_nrhs) {
        p->last_error = "nrhs must be in [1, max_nrhs]";
        return IFGF_EINVAL;
    }
    if (mode < 1 || mode > 3) {
        p->last_error = "mode must be 1, 2 or 3";
        return IFGF_EINVAL;
    }
    const size_t eb = ifgf_elem_bytes(p->precision);
    const size_t bytes = (size_t)p->n * nrhs * eb;
    const bool in_dev = is_device_pointer(in), out_dev = is_device_pointer(out);
    if ((!in_dev || !out_dev) && !p->stage_in) {
        p->stage_in = ifgf_dalloc(p, (size_t)p->n * p->max_nrhs * eb);
        p->stage_out = ifgf_dalloc(p, (size_t)p->n * p->max_nrhs * eb);
        if (!p->stage_in || !p->stage_out) {
            p->last_error = "staging buffers";
            return IFGF_ENOMEM;
        }
    }
    const void *din = in;
    void *dout = out;
    if (!in_dev) {
        if (cudaMemcpyAsync(p->stage_in, in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            p->last_error = "host-to-device copy failed";
            return IFGF_ECUDA;
        }
        din = p->stage_in;
    }
    if (!out_dev) dout = p->stage_out;
    // two-buffer plans build their adjoint's transpose lists per level just in time
    // (resident lists for all levels would not fit beside the cone values)
    const bool jit = adjoint && p->pingpong && !p->adjoint_ready;
    if (adjoint && !p->adjoint_ready && !jit) {
        // first adjoint call: build the transpose lists (synchronises the stream)
        ifgf_status s = ifgf_build_adjoint_lists(p, st);
        if (s != IFGF_OK) return s;
        graphs_clear(p);
    }
    if (adjoint && !p->adjoint_values_ready) {
        ifgf_status s = ifgf_alloc_adjoint_values(p);
        if (s != IFGF_OK) return s;
        graphs_clear(p);
    }
    p->timer.n = 0;
    cudaError_t e = cudaSuccess;
    if (jit) {
        // right-hand sides in chunks of at most rhs_chunk (contiguous rows of the
        // caller's [nrhs][N] arrays); the lists are built and freed between launches
        for (int c0 = 0; c0 < nrhs; c0 += p->rhs_chunk) {
            const int nc = std::min(p->rhs_chunk, nrhs - c0);
            const void *cin = (const char *)din + (size_t)c0 * p->n * eb;
            void *cout = (char *)dout + (size_t)c0 * p->n * eb;
            ifgf_status s = p->precision == IFGF_FP64 ? ifgf_run_adjoint_jit_f64(p, nc, cin, cout, mode, st)
                                                      : ifgf_run_adjoint_jit_f32(p, nc, cin, cout, mode, st);
            if (s != IFGF_OK) return s;
        }
    } else if (p->use_graphs) {
        ifgf_status s = replay_graph(p, din, dout, nrhs, mode, adjoint, st);
        if (s != IFGF_OK) return s;
    } else {
        e = launch_evaluation(p, din, dout, nrhs, mode, adjoint, st);
    }
    if (e != cudaSuccess) {
        p->last_error = std::string("kernel launch failed: ") + cudaGetErrorString(e);
        return IFGF_ECUDA;
    }
    if (p->timer.on && p->timer.n > 1) {
        // profiling mode: wait for this call and attribute the time between marks
        const ifgf_status ws = wait_stream(p, st);
        if (ws != IFGF_OK) return ws;
        for (int i = 1; i < p->timer.n; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->timer.ev[i - 1], p->timer.ev[i]);
            int s = p->timer.stage[i];
            if (s >= 0 && s < STAGE_COUNT) {
                p->stage_ms[s] += ms;
                p->stage_launches[s] += p->timer.launches[i];
            }
        }
        p->stage_calls += 1;
    }
    p->last_nrhs = nrhs;
    if (!out_dev) {
        if (cudaMemcpyAsync(out, p->stage_out, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            p->last_error = "device-to-host copy failed";
            return IFGF_ECUDA;
        }
    }
    if (!in_dev || !out_dev) return wait_stream(p, st);
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_apply(ifgf_plan *plan, const void *sigma, void *u, int nrhs, void *stream)
{
    return ifgf_run_apply(plan, sigma, u, nrhs, 3, 0, (cudaStream_t)stream);
}

extern "C" ifgf_status ifgf_apply_adjoint(ifgf_plan *plan, const void *v, void *w, int nrhs, void *stream)
{
    return ifgf_run_apply(plan, v, w, nrhs, 3, 1, (cudaStream_t)stream);
}

extern "C" ifgf_status ifgf_apply_partial(ifgf_plan *plan, const void *in, void *out, int nrhs, int mode,
                                          int adjoint, void *stream)
{
    return ifgf_run_apply(plan, in, out, nrhs, mode, adjoint ? 1 : 0, (cudaStream_t)stream);
}

extern "C" ifgf_status ifgf_plan_destroy(ifgf_plan *plan)
{
    if (!plan) return IFGF_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return IFGF_OK;
}

// ---------------------------------------------------------------------------------
// Introspection
// ---------------------------------------------------------------------------------
static ifgf_status copy_i32_as_i64(ifgf_plan *p, const int *src, int64_t count, int64_t *dst)
{
    if (count <= 0) return IFGF_OK;
    std::vector<int> h((size_t)count);
    if (cudaMemcpy(h.data(), src, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        p->last_error = "device-to-host copy failed";
        return IFGF_ECUDA;
    }
    for (int64_t i = 0; i < count; ++i) dst[i] = h[(size_t)i];
    return IFGF_OK;
}

static bool level_ok(const ifgf_plan *p, int level, int min_level)
{
    return p && level >= min_level && level <= p->D;
}

extern "C" ifgf_status ifgf_plan_level_info(const ifgf_plan *plan, int level, int64_t *info)
{
    if (!level_ok(plan, level, 1) || !info) return IFGF_EINVAL;
    const LevelHost &h = plan->lh[level];
    const LevelDev &L = plan->dev.lev[level];
    info[0] = L.nbox;
    info[1] = 0;
    info[2] = level >= 3 ? h.ncous : 0;
    info[3] = level >= 3 ? L.nact : 0;
    info[4] = level >= 3 ? L.ns : 0;
    info[5] = level >= 3 ? L.nc : 0;
    info[6] = level >= 3 ? h.cousin_evals : 0;
    info[7] = level >= 4 ? h.upward_evals : 0;
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_get_perm(const ifgf_plan *plan, int64_t *perm)
{
    if (!plan || !perm) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    return copy_i32_as_i64((ifgf_plan *)plan, plan->dev.perm, plan->n, perm);
}

extern "C" ifgf_status ifgf_plan_get_boxes(const ifgf_plan *plan, int level, uint64_t *keys, int64_t *start)
{
    if (!level_ok(plan, level, 1) || !keys || !start) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    const LevelDev &L = plan->dev.lev[level];
    if (cudaMemcpy(keys, L.key, (size_t)L.nbox * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return IFGF_ECUDA;
    return copy_i32_as_i64((ifgf_plan *)plan, L.start, L.nbox + 1, start);
}

extern "C" ifgf_status ifgf_plan_get_box_ends(const ifgf_plan *plan, int level, int64_t *end, int64_t *leaf)
{
    if (!level_ok(plan, level, 1) || !end || !leaf) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    const LevelDev &L = plan->dev.lev[level];
    ifgf_status s = copy_i32_as_i64((ifgf_plan *)plan, L.end, L.nbox, end);
    if (s != IFGF_OK) return s;
    std::vector<unsigned char> h(L.nbox);
    if (L.nbox && cudaMemcpy(h.data(), L.leaf, L.nbox, cudaMemcpyDeviceToHost) != cudaSuccess) return IFGF_ECUDA;
    for (int b = 0; b < L.nbox; ++b) leaf[b] = h[b];
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_get_point_levels(const ifgf_plan *plan, int64_t *levels)
{
    if (!plan || !levels) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    return copy_i32_as_i64((ifgf_plan *)plan, plan->dev.ptlev, plan->n, levels);
}

extern "C" ifgf_status ifgf_plan_get_near(const ifgf_plan *plan, int level, int64_t *count, int64_t *start,
                                          int64_t *lo, int64_t *hi)
{
    if (!level_ok(plan, level, 3) || !count) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    const LevelDev &L = plan->dev.lev[level];
    int m = 0;
    if (cudaMemcpy(&m, L.near_start + L.nbox, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return IFGF_ECUDA;
    *count = m;
    if (!start) return IFGF_OK;
    if (!lo || !hi) return IFGF_EINVAL;
    ifgf_status s = copy_i32_as_i64((ifgf_plan *)plan, L.near_start, L.nbox + 1, start);
    if (s == IFGF_OK) s = copy_i32_as_i64((ifgf_plan *)plan, L.near_lo, m, lo);
    if (s == IFGF_OK) s = copy_i32_as_i64((ifgf_plan *)plan, L.near_hi, m, hi);
    return s;
}

extern "C" ifgf_status ifgf_plan_get_cousins(const ifgf_plan *plan, int level, int64_t *start, int64_t *list)
{
    if (!level_ok(plan, level, 3) || !start || !list) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    const LevelDev &L = plan->dev.lev[level];
    ifgf_status s = copy_i32_as_i64((ifgf_plan *)plan, L.cous_start, L.nbox + 1, start);
    if (s != IFGF_OK) return s;
    return copy_i32_as_i64((ifgf_plan *)plan, L.cous, plan->lh[level].ncous, list);
}

extern "C" ifgf_status ifgf_plan_get_active(const ifgf_plan *plan, int level, int64_t *start, int64_t *cones)
{
    if (!level_ok(plan, level, 3) || !start || !cones) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    const LevelDev &L = plan->dev.lev[level];
    ifgf_status s = copy_i32_as_i64((ifgf_plan *)plan, L.act_start, L.nbox + 1, start);
    if (s != IFGF_OK) return s;
    return copy_i32_as_i64((ifgf_plan *)plan, L.act_cone, L.nact, cones);
}

extern "C" ifgf_status ifgf_plan_get_values(const ifgf_plan *plan, int level, void *out)
{
    if (!level_ok(plan, level, 3) || !out) return IFGF_EINVAL;
    cudaDeviceSynchronize();
    const LevelDev &L = plan->dev.lev[level];
    size_t bytes = (size_t)L.nact * plan->P * plan->last_nrhs * ifgf_elem_bytes(plan->precision);
    if (bytes && cudaMemcpy(out, L.F, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return IFGF_ECUDA;
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_geometry(const ifgf_plan *plan, double *geom)
{
    if (!plan || !geom) return IFGF_EINVAL;
    geom[0] = plan->H1;
    geom[1] = plan->corner[0];
    geom[2] = plan->corner[1];
    geom[3] = plan->corner[2];
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_stats(const ifgf_plan *plan, char *buf, size_t cap)
{
    if (!plan || !buf || cap == 0) return IFGF_EINVAL;
    std::string s = "{";
    char tmp[512];
    snprintf(tmp, sizeof tmp,
             "\"n\": %lld, \"levels\": %d, \"P\": %d, \"kappa\": %.17g, \"precision\": %d, \"max_nrhs\": %d, "
             "\"near_pairs\": %lld, \"leaf_evals\": %lld, \"build_ms\": %.3f, \"device_bytes\": %zu, "
             "\"pingpong\": %d, \"rhs_chunk\": %d, \"cache_bytes\": %zu, \"graphs\": %d, "
             "\"graph_captures\": %lld, \"graph_replays\": %lld, \"tune_leaf\": %d, \"tune_cone_ctas\": %d, "
             "\"leaf_max\": %d, \"adaptive\": %d, \"level\": [",
             (long long)plan->n, plan->D, plan->P, plan->kappa, plan->precision, plan->max_nrhs,
             (long long)plan->near_pairs, (long long)plan->leaf_evals, plan->build_ms, plan->device_bytes,
             plan->pingpong ? 1 : 0, plan->rhs_chunk, plan->cache_bytes, (int)plan->graphs.size(),
             (long long)plan->graph_captures, (long long)plan->graph_replays, plan->dev.tune_leaf,
             plan->dev.tune_cone_ctas, plan->leaf_max, plan->dev.adaptive);
    s += tmp;
    for (int d = 1; d <= plan->D; ++d) {
        const LevelHost &h = plan->lh[d];
        const LevelDev &L = plan->dev.lev[d];
        snprintf(tmp, sizeof tmp,
                 "%s{\"d\": %d, \"nbox\": %d, \"ncous\": %lld, \"nact\": %d, \"ns\": %d, \"nc\": %d, "
                 "\"cousin_evals\": %lld, \"upward_evals\": %lld, \"table_rows\": %lld, \"union_rows\": %lld, "
                 "\"act_sets\": %d}",
                 d > 1 ? ", " : "", d, L.nbox, (long long)h.ncous, d >= 3 ? L.nact : 0, d >= 3 ? L.ns : 0,
                 d >= 3 ? L.nc : 0, (long long)h.cousin_evals, (long long)h.upward_evals, (long long)h.table_rows,
                 (long long)h.union_rows, h.act_sets);
        s += tmp;
    }
    s += "]}";
    if (s.size() + 1 > cap) return IFGF_EINVAL;
    memcpy(buf, s.c_str(), s.size() + 1);
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_check(ifgf_plan *plan, int *device_errors)
{
    if (!plan || !device_errors) return IFGF_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        plan->last_error = "device synchronisation failed";
        return IFGF_ECUDA;
    }
    int h = 0;
    if (cudaMemcpy(&h, plan->dev.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return IFGF_ECUDA;
    if (cudaMemset(plan->dev.err, 0, sizeof(int)) != cudaSuccess) return IFGF_ECUDA;
    *device_errors = h;
    return IFGF_OK;
}

__global__ void k_cone_ids(PlanDev pd, int d, int n, const double *v, int *exact, int *fast, int mixed)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const LevelDev &L = pd.lev[d];
    double x = v[3 * (size_t)i], y = v[3 * (size_t)i + 1], z = v[3 * (size_t)i + 2];
    exact[i] = ifgf::cone_of(L, x, y, z).cone;
    fast[i] = mixed ? ifgf::cone_of_mixed(L, x, y, z).cone : ifgf::cone_of_fast(L, x, y, z).cone;
}

extern "C" ifgf_status ifgf_plan_cone_ids(const ifgf_plan *plan, int level, int64_t n, const double *v,
                                          int32_t *exact, int32_t *fast)
{
    if (!level_ok(plan, level, 3) || n < 0 || n > (1 << 30) || (n > 0 && (!v || !exact || !fast)))
        return IFGF_EINVAL;
    if (n == 0) return IFGF_OK;
    ifgf_plan *p = (ifgf_plan *)plan;
    double *dv = nullptr;
    int *de = nullptr;
    if (cudaMalloc(&dv, (size_t)n * 3 * sizeof(double)) != cudaSuccess) return IFGF_ENOMEM;
    if (cudaMalloc(&de, (size_t)n * 2 * sizeof(int)) != cudaSuccess) {
        cudaFree(dv);
        return IFGF_ENOMEM;
    }
    ifgf_status st = IFGF_OK;
    if (cudaMemcpy(dv, v, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) st = IFGF_ECUDA;
    if (st == IFGF_OK) {
        k_cone_ids<<<(int)((n + 255) / 256), 256>>>(p->dev, level, (int)n, dv, de, de + n,
                                                     p->precision != IFGF_FP64);
        if (cudaDeviceSynchronize() != cudaSuccess) st = IFGF_ECUDA;
    }
    if (st == IFGF_OK && (cudaMemcpy(exact, de, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
                          cudaMemcpy(fast, de + n, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess))
        st = IFGF_ECUDA;
    cudaFree(dv);
    cudaFree(de);
    if (st != IFGF_OK) p->last_error = "cone id evaluation failed";
    return st;
}

extern "C" ifgf_status ifgf_plan_set_profiling(ifgf_plan *plan, int on)
{
    if (!plan) return IFGF_EINVAL;
    if (on && !plan->timer.ev[0]) {
        for (int i = 0; i < StageTimer::kMax; ++i)
            if (cudaEventCreate(&plan->timer.ev[i]) != cudaSuccess) {
                plan->last_error = "event creation failed";
                return IFGF_ECUDA;
            }
    }
    plan->timer.on = on != 0;
    for (int s = 0; s < STAGE_COUNT; ++s) {
        plan->stage_ms[s] = 0;
        plan->stage_launches[s] = 0;
    }
    plan->stage_calls = 0;
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_autotune(ifgf_plan *plan, int nrhs, int reps, double *ms, int *choice,
                                          void *stream)
{
    if (!plan) return IFGF_EINVAL;
    if (!ifgf_is_batched(plan->precision) || nrhs < 2 || nrhs > ifgf_batched_max_nrhs(plan->Ps) || nrhs % 2 ||
        nrhs > plan->max_nrhs ||
        reps < 1) {
        plan->last_error = "autotune: batched plan, even nrhs in [2, min(64, max_nrhs)] and reps >= 1";
        return IFGF_EINVAL;
    }
    NvtxRange range("ifgf_plan_autotune");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(plan->sig_sorted, 0, (size_t)plan->n * nrhs * 8, st) != cudaSuccess) {
        cudaGetLastError();
        plan->last_error = "autotune: clearing the density buffer";
        return IFGF_ECUDA;
    }
    float t[5] = {0, 0, 0, 0, 0};
    const cudaError_t e = ifgf_batched_autotune(plan->dev, nrhs, plan->sig_sorted, plan->u_sorted, st, reps, t);
    if (e != cudaSuccess) {
        plan->last_error = std::string("autotune: ") + cudaGetErrorString(e);
        return IFGF_ECUDA;
    }
    graphs_clear(plan);  // captured evaluations hold the previous tile shapes
    if (ms)
        for (int i = 0; i < 5; ++i) ms[i] = t[i];
    if (choice) {
        choice[0] = plan->dev.tune_leaf;
        choice[1] = plan->dev.tune_cone_ctas;
    }
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_set_tiles(ifgf_plan *plan, int leaf_shape, int cone_ctas_per_sm)
{
    if (!plan) return IFGF_EINVAL;
    if (leaf_shape < 0 || leaf_shape > 2 || cone_ctas_per_sm < 1 || cone_ctas_per_sm > 2) {
        plan->last_error = "tiles: leaf shape in [0, 2], CTAs per SM in [1, 2]";
        return IFGF_EINVAL;
    }
    plan->dev.tune_leaf = leaf_shape;
    plan->dev.tune_cone_ctas = cone_ctas_per_sm;
    graphs_clear(plan);
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_set_graphs(ifgf_plan *plan, int on)
{
    if (!plan) return IFGF_EINVAL;
    plan->use_graphs = on != 0;
    if (!on) graphs_clear(plan);
    return IFGF_OK;
}

extern "C" ifgf_status ifgf_plan_timings(const ifgf_plan *plan, double *ms, int64_t *launches, int64_t *calls,
                                         int count)
{
    if (!plan || !ms || !launches || !calls || count < STAGE_COUNT) return IFGF_EINVAL;
    for (int s = 0; s < STAGE_COUNT; ++s) {
        ms[s] = plan->stage_ms[s];
        launches[s] = plan->stage_launches[s];
    }
    *calls = plan->stage_calls;
    return IFGF_OK;
}

extern "C" const char *ifgf_last_error(const ifgf_plan *plan)
{
    if (!plan) return g_create_error.c_str();
    return plan->last_error.c_str();
}
