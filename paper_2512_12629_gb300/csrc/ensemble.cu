// Ensembles of independent boxes (many small simulations on one GPU) and the
// cost-ordered placement they share with a multi-GPU split.
//
// Placement follows the load balancing of the paper's Sec. 2.2.3 (Fig.
// balance): tasks sorted by decreasing cost and each given, in that order, to
// the least loaded worker (longest-processing-time-first).  Here a task is a
// box, its cost an estimate of one step's work (FFT N log N over every PM level
// plus a term linear in the particles), and a worker either a concurrent branch
// of one CUDA graph or a GPU rank.
//
// cube2_ensemble_create records n_steps KDK steps of every box into one CUDA
// graph: a fork from an internal capture stream into n_streams branch streams,
// the boxes of each branch one after another (each box's steps in order), and
// a join.  Replaying the graph runs the whole ensemble with one launch, the
// small boxes' kernels of different branches overlapping on the GPU.  The
// context calls are allocation- and synchronisation-free, which is what makes
// them capturable; each context's stream is redirected to its branch only
// while the graph is recorded.
#include "common.cuh"

#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

struct cube2_ensemble {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> branches;
    std::vector<cudaEvent_t> events;
    int64_t kernel_nodes = 0;
    int64_t particle_steps = 0;
    cube2_ensemble_opts opts{};
    int n_steps = 0;
    // persistent PP: per-step parameters of every box, the (box, block) items,
    // their per-step cost and order, the queue header, the host's publication
    void *pp_params = nullptr;      // [n_steps][n_boxes] PP parameters (device)
    int32_t *item_box = nullptr;    // [n_items]
    int32_t *item_base = nullptr;   // [n_boxes] first item of each box
    unsigned *item_cost = nullptr;  // [n_items]
    int32_t *item_order = nullptr;  // [n_items]
    void *queue = nullptr;          // queue header (device)
    int *publish = nullptr;         // [n_steps] pinned host: epoch published before step s (s + 1), 0 withholds it
};

namespace {

void ensemble_free(cube2_ensemble *e) {
    if (!e) return;
    cudaFree(e->pp_params);
    cudaFree(e->item_box);
    cudaFree(e->item_base);
    cudaFree(e->item_cost);
    cudaFree(e->item_order);
    cudaFree(e->queue);
    if (e->publish) cudaFreeHost(e->publish);
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    for (cudaEvent_t ev : e->events) cudaEventDestroy(ev);
    for (cudaStream_t s : e->branches) cudaStreamDestroy(s);
    if (e->origin) cudaStreamDestroy(e->origin);
    delete e;
}

// One step's work estimate of a box: FFT passes over every level plus the
// particle-linear kernels (deposit, interp, PP at mean density, re-bin).
double config_cost(const cube2_config *cfg) {
    double cost = 0.0;
    for (int l = 0; l < cfg->n_levels && l < CUBE2_MAX_LEVELS; ++l) {
        const double m = (double)cfg->n_mesh[l] * cfg->n_mesh[l] * cfg->n_mesh[l];
        cost += m * std::log2(std::max(m, 2.0));
    }
    return cost + 64.0 * (double)cfg->n_particles;
}

}  // namespace

extern "C" {

int cube2_lpt_partition(const double *cost, int n, int bins, int *bin_of) {
    if (n < 0 || bins < 1 || (n > 0 && (!cost || !bin_of))) return CUBE2_ERR_BAD_ARG;
    for (int i = 0; i < n; ++i)
        if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return CUBE2_ERR_BAD_ARG;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(bins, 0.0);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        bin_of[i] = k;
        load[k] += cost[i];
    }
    return CUBE2_OK;
}

int cube2_config_cost(const cube2_config *cfg, double *cost) {
    if (!cfg || !cost || cfg->n_levels < 1 || cfg->n_particles < 0) return CUBE2_ERR_BAD_ARG;
    *cost = config_cost(cfg);
    return CUBE2_OK;
}

int cube2_ensemble_create(cube2_ensemble **out, cube2_ctx *const *ctxs, cube2_particles *const *parts, int n_boxes,
                          const double *a, int n_steps, int n_streams) {
    cube2_ensemble_opts o{};
    o.n_streams = n_streams;
    o.persistent_pp = 0;
    o.pp_ctas_per_sm = 16;
    o.pp_wmax = 0;
    o.timeout_ms = 1000.0;
    return cube2_ensemble_create_ex(out, ctxs, parts, n_boxes, a, n_steps, &o);
}

int cube2_ensemble_create_ex(cube2_ensemble **out, cube2_ctx *const *ctxs, cube2_particles *const *parts, int n_boxes,
                             const double *a, int n_steps, const cube2_ensemble_opts *opts) {
    if (!out) return CUBE2_ERR_BAD_ARG;
    *out = nullptr;
    if (!opts || !ctxs || !parts || !a || n_boxes < 1 || n_steps < 1) return CUBE2_ERR_BAD_ARG;
    const int n_streams = opts->n_streams;
    const bool persistent = opts->persistent_pp != 0;
    if (n_streams < 1 || n_streams > 64 || (persistent && (opts->pp_ctas_per_sm < 1 || opts->pp_ctas_per_sm > 16)) ||
        opts->pp_wmax < 0 || opts->pp_wmax > 64 || !(opts->timeout_ms > 0))
        return CUBE2_ERR_BAD_ARG;
    for (int b = 0; b < n_boxes; ++b) {
        if (!ctxs[b] || !parts[b]) return CUBE2_ERR_BAD_ARG;
        if (ctxs[b]->prof) return cube2::set_error(ctxs[b], CUBE2_ERR_STATE, "profiling must be off to record an ensemble");
        if (ctxs[b]->device != ctxs[0]->device) return cube2::set_error(ctxs[b], CUBE2_ERR_BAD_ARG, "boxes on different devices");
        if (persistent && (ctxs[b]->pm3.on || ctxs[b]->vel32))
            return cube2::set_error(ctxs[b], CUBE2_ERR_STATE,
                                    "the persistent PP kernel takes boxes without the third level and FP16 velocities");
        for (int c = 0; c < b; ++c)
            if (ctxs[c] == ctxs[b]) return cube2::set_error(ctxs[b], CUBE2_ERR_BAD_ARG, "a context appears twice");
        for (int s = 0; s < n_steps; ++s)
            if (!(a[(size_t)b * (n_steps + 1) + s] > 0) ||
                !(a[(size_t)b * (n_steps + 1) + s + 1] > a[(size_t)b * (n_steps + 1) + s]))
                return cube2::set_error(ctxs[b], CUBE2_ERR_BAD_ARG, "scale factors must increase from > 0");
    }
    cudaError_t e = cudaSetDevice(ctxs[0]->device);
    if (e != cudaSuccess) return cube2::cuda_error(ctxs[0], e, "ensemble device");
    // every box's earlier work done before its stream is borrowed
    for (int b = 0; b < n_boxes && e == cudaSuccess; ++b) e = cudaStreamSynchronize(ctxs[b]->stream);
    if (e != cudaSuccess) return cube2::cuda_error(ctxs[0], e, "ensemble sync");

    std::vector<double> cost(n_boxes);
    for (int b = 0; b < n_boxes; ++b) cost[b] = config_cost(&ctxs[b]->cfg);
    const int nbr = std::min(n_streams, n_boxes);
    std::vector<int> bin(n_boxes);
    cube2_lpt_partition(cost.data(), n_boxes, nbr, bin.data());
    std::vector<int> order(n_boxes);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });

    cube2_ensemble *E = new cube2_ensemble();
    E->opts = *opts;
    E->n_steps = n_steps;
    e = cudaStreamCreateWithFlags(&E->origin, cudaStreamNonBlocking);
    E->branches.assign(nbr, nullptr);
    const int nev = persistent ? (nbr + 1) * n_steps : nbr + 1;
    E->events.assign(nev, nullptr);
    for (int k = 0; k < nbr && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&E->branches[k], cudaStreamNonBlocking);
    for (int k = 0; k < nev && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&E->events[k], cudaEventDisableTiming);
    // persistent PP: items (box, block of 128 slots), parameters per step, queue
    const size_t psz = cube2::pp_params_bytes();
    std::vector<int32_t> item_box, base(n_boxes);
    std::vector<unsigned char> params;
    if (persistent && e == cudaSuccess) {
        for (int b = 0; b < n_boxes; ++b) {
            base[b] = (int32_t)item_box.size();
            const int64_t nb = (ctxs[b]->N + 127) / 128;
            for (int64_t k = 0; k < nb; ++k) item_box.push_back(b);
        }
        params.assign((size_t)n_steps * n_boxes * psz, 0);
        const size_t ni = std::max<size_t>(item_box.size(), 1);
        e = cudaMalloc(&E->pp_params, params.size());
        if (e == cudaSuccess) e = cudaMalloc((void **)&E->item_box, ni * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&E->item_base, (size_t)n_boxes * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&E->item_cost, ni * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&E->item_order, ni * 4);
        if (e == cudaSuccess) e = cudaMalloc(&E->queue, cube2::pp_queue_bytes());
        if (e == cudaSuccess) e = cudaMemset(E->queue, 0, cube2::pp_queue_bytes());
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&E->publish, (size_t)n_steps * sizeof(int), cudaHostAllocDefault);
        if (e == cudaSuccess) {
            for (int s = 0; s < n_steps; ++s) E->publish[s] = s + 1;
            if (!item_box.empty())
                e = cudaMemcpy(E->item_box, item_box.data(), item_box.size() * 4, cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) e = cudaMemcpy(E->item_base, base.data(), (size_t)n_boxes * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        ensemble_free(E);
        return cube2::cuda_error(ctxs[0], e, "ensemble setup");
    }
    int num_sms = 152;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, ctxs[0]->device);
    std::vector<int> wmax_saved(n_boxes);
    for (int b = 0; b < n_boxes; ++b) {
        wmax_saved[b] = ctxs[b]->pp_wmax;
        if (opts->pp_wmax > 0) ctxs[b]->pp_wmax = opts->pp_wmax;
    }

    int status = CUBE2_OK;
    e = cudaStreamBeginCapture(E->origin, cudaStreamCaptureModeThreadLocal);
    if (!persistent) {
        // every box's steps in its branch, the branches joined once at the end
        if (e == cudaSuccess) e = cudaEventRecord(E->events[nbr], E->origin);
        for (int k = 0; k < nbr && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(E->branches[k], E->events[nbr], 0);
        for (int oi = 0; oi < n_boxes && e == cudaSuccess && status == CUBE2_OK; ++oi) {
            const int b = order[oi];
            cube2_ctx *c = ctxs[b];
            cudaStream_t own = c->stream;
            c->stream = E->branches[bin[b]];
            const double *ab = a + (size_t)b * (n_steps + 1);
            for (int s = 0; s < n_steps && status == CUBE2_OK; ++s) status = cube2_kdk_step(c, parts[b], ab[s], ab[s + 1]);
            c->stream = own;
        }
        for (int k = 0; k < nbr && e == cudaSuccess && status == CUBE2_OK; ++k) {
            e = cudaEventRecord(E->events[k], E->branches[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(E->origin, E->events[k], 0);
        }
    } else {
        // step by step: each box's step up to its PP inputs in its branch, then
        // one persistent PP kernel (with the second kick) over every box
        const unsigned long long timeout_ns = (unsigned long long)(opts->timeout_ms * 1e6);
        for (int s = 0; s < n_steps && e == cudaSuccess && status == CUBE2_OK; ++s) {
            cudaEvent_t *ev = &E->events[(size_t)s * (nbr + 1)];
            e = cudaEventRecord(ev[nbr], E->origin);
            for (int k = 0; k < nbr && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(E->branches[k], ev[nbr], 0);
            for (int oi = 0; oi < n_boxes && e == cudaSuccess && status == CUBE2_OK; ++oi) {
                const int b = order[oi];
                cube2_ctx *c = ctxs[b];
                cudaStream_t own = c->stream;
                c->stream = E->branches[bin[b]];
                c->defer_pp = true;
                const double *ab = a + (size_t)b * (n_steps + 1);
                status = cube2_kdk_step(c, parts[b], ab[s], ab[s + 1]);
                c->defer_pp = false;
                c->stream = own;
                memcpy(&params[((size_t)s * n_boxes + b) * psz], c->pp_deferred, psz);
            }
            for (int k = 0; k < nbr && e == cudaSuccess && status == CUBE2_OK; ++k) {
                e = cudaEventRecord(ev[k], E->branches[k]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(E->origin, ev[k], 0);
            }
            if (e == cudaSuccess && status == CUBE2_OK && !item_box.empty())
                e = cube2::launch_pp_persistent_step(
                    E->origin, static_cast<unsigned char *>(E->pp_params) + (size_t)s * n_boxes * psz, E->item_box,
                    E->item_base, (int)item_box.size(), E->item_cost, E->item_order, E->queue, &E->publish[s], s + 1,
                    timeout_ns, num_sms * opts->pp_ctas_per_sm);
        }
    }
    for (int b = 0; b < n_boxes; ++b) {
        ctxs[b]->pp_wmax = wmax_saved[b];
        ctxs[b]->defer_pp = false;
    }
    for (int b = 0; b < n_boxes; ++b) E->particle_steps += (int64_t)n_steps * ctxs[b]->N;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(E->origin, &g);
    E->graph = g;
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess && persistent) e = cudaMemcpy(E->pp_params, params.data(), params.size(), cudaMemcpyHostToDevice);
    if (status != CUBE2_OK || e != cudaSuccess) {
        ensemble_free(E);
        if (status != CUBE2_OK) return status;
        return cube2::cuda_error(ctxs[0], e, "ensemble capture");
    }
    size_t nn = 0;
    e = cudaGraphGetNodes(E->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(E->graph, nodes.data(), &nn);
    for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (t == cudaGraphNodeTypeKernel) ++E->kernel_nodes;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&E->exec, E->graph, 0);
    if (e != cudaSuccess) {
        ensemble_free(E);
        return cube2::cuda_error(ctxs[0], e, "ensemble instantiate");
    }
    *out = E;
    return CUBE2_OK;
}

int cube2_ensemble_check(cube2_ensemble *ens, void *stream) {
    if (!ens) return CUBE2_ERR_BAD_ARG;
    if (!ens->queue) return CUBE2_OK;
    int h[4] = {0, 0, 0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h, ens->queue, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return CUBE2_ERR_CUDA;
    if (!h[3]) return CUBE2_OK;
    e = cudaMemsetAsync(static_cast<int *>(ens->queue) + 3, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? CUBE2_ERR_TIMEOUT : CUBE2_ERR_CUDA;
}

int cube2_ensemble_publish(cube2_ensemble *ens, int on) {
    if (!ens) return CUBE2_ERR_BAD_ARG;
    if (!ens->publish) return CUBE2_OK;
    for (int s = 0; s < ens->n_steps; ++s) ens->publish[s] = on ? s + 1 : 0;
    return CUBE2_OK;
}

// Autotuner: coordinate search over the ensemble's runtime knobs, each
// candidate recorded as a graph and timed with CUDA events over `trials`
// launches from the same particle states (snapshotted first, restored before
// every launch and at the end).
namespace {

struct Snapshot {
    std::vector<void *> bufs;
    bool ok = true;
};

struct BoxArrays {
    void *dst;
    size_t bytes;
};

std::vector<BoxArrays> box_arrays(cube2_ctx *c, cube2_particles *p) {
    const size_t N = (size_t)c->N, C = (size_t)c->n_cells;
    std::vector<BoxArrays> v;
    for (int d = 0; d < 3; ++d) v.push_back({p->off[d], N * 2});
    v.push_back({p->count, C * 4});
    v.push_back({p->start, C * 4});
    for (int d = 0; d < 3; ++d) {
        if (c->vel32) v.push_back({p->vel16[d], N * 2});
        else v.push_back({p->vel[d], N * 4});
        v.push_back({p->acc[d], N * 4});
    }
    if (c->vel32) v.push_back({p->vscale, C * 4});
    return v;
}

}  // namespace

int cube2_ensemble_autotune(cube2_ctx *const *ctxs, cube2_particles *const *parts, int n_boxes, const double *a,
                            int n_steps, int trials, void *stream, cube2_ensemble_opts *best, double *best_ms) {
    if (!ctxs || !parts || !a || !best || !best_ms || n_boxes < 1 || n_steps < 1 || trials < 1)
        return CUBE2_ERR_BAD_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<std::pair<void *, BoxArrays>> snap;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < n_boxes && e == cudaSuccess; ++b) {
        if (!ctxs[b] || !parts[b]) e = cudaErrorInvalidValue;
        else
            for (const BoxArrays &x : box_arrays(ctxs[b], parts[b])) {
                void *buf = nullptr;
                e = cudaMalloc(&buf, x.bytes > 0 ? x.bytes : 16);
                if (e != cudaSuccess) break;
                snap.push_back({buf, x});
                if (x.bytes) e = cudaMemcpyAsync(buf, x.dst, x.bytes, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) break;
            }
    }
    auto restore = [&]() {
        cudaError_t r = cudaSuccess;
        for (auto &sx : snap)
            if (r == cudaSuccess && sx.second.bytes)
                r = cudaMemcpyAsync(sx.second.dst, sx.first, sx.second.bytes, cudaMemcpyDeviceToDevice, st);
        return r;
    };
    int status = e == cudaSuccess ? CUBE2_OK : CUBE2_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (status == CUBE2_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        status = CUBE2_ERR_CUDA;
    auto measure = [&](const cube2_ensemble_opts &o, double *ms) -> int {
        cube2_ensemble *E = nullptr;
        int r = cube2_ensemble_create_ex(&E, ctxs, parts, n_boxes, a, n_steps, &o);
        if (r != CUBE2_OK) return r;
        double bestt = 1e300;
        for (int t = 0; t < trials + 1 && r == CUBE2_OK; ++t) {   // the first launch warms up
            if (restore() != cudaSuccess) { r = CUBE2_ERR_CUDA; break; }
            if (cudaEventRecord(e0, st) != cudaSuccess || cube2_ensemble_launch(E, st) != CUBE2_OK ||
                cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                r = CUBE2_ERR_CUDA;
                break;
            }
            r = cube2_ensemble_check(E, st);
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            if (t > 0) bestt = std::min(bestt, (double)f);
        }
        cube2_ensemble_destroy(E);
        *ms = bestt;
        return r;
    };
    cube2_ensemble_opts cur = *best;
    double cur_ms = 0.0;
    if (status == CUBE2_OK) status = measure(cur, &cur_ms);
    const int ctas[] = {4, 8, 16}, wmax[] = {8, 16, 24}, streams[] = {8, 16, 32};
    for (int knob = 0; knob < 3 && status == CUBE2_OK; ++knob) {
        if (knob == 0 && !cur.persistent_pp) continue;
        for (int i = 0; i < 3 && status == CUBE2_OK; ++i) {
            cube2_ensemble_opts t = cur;
            if (knob == 0) t.pp_ctas_per_sm = ctas[i];
            if (knob == 1) t.pp_wmax = wmax[i];
            if (knob == 2) t.n_streams = streams[i];
            if (t.pp_ctas_per_sm == cur.pp_ctas_per_sm && t.pp_wmax == cur.pp_wmax && t.n_streams == cur.n_streams)
                continue;
            double ms = 0.0;
            status = measure(t, &ms);
            if (status == CUBE2_OK && ms < cur_ms) {
                cur = t;
                cur_ms = ms;
            }
        }
    }
    if (restore() != cudaSuccess && status == CUBE2_OK) status = CUBE2_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && status == CUBE2_OK) status = CUBE2_ERR_CUDA;
    for (auto &sx : snap) cudaFree(sx.first);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (status == CUBE2_OK) {
        *best = cur;
        *best_ms = cur_ms;
    }
    return status;
}

int cube2_ensemble_launch(cube2_ensemble *ens, void *stream) {
    if (!ens) return CUBE2_ERR_BAD_ARG;
    const cudaError_t e = cudaGraphLaunch(ens->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? CUBE2_OK : CUBE2_ERR_CUDA;
}

int cube2_ensemble_info(const cube2_ensemble *ens, int64_t out[2]) {
    if (!ens || !out) return CUBE2_ERR_BAD_ARG;
    out[0] = ens->kernel_nodes;
    out[1] = ens->particle_steps;
    return CUBE2_OK;
}

void cube2_ensemble_destroy(cube2_ensemble *ens) {
    if (!ens) return;
    cudaStreamSynchronize(ens->origin);
    ensemble_free(ens);
}

}  // extern "C"
