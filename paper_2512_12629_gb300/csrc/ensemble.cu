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
};

namespace {

void ensemble_free(cube2_ensemble *e) {
    if (!e) return;
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
    if (!out) return CUBE2_ERR_BAD_ARG;
    *out = nullptr;
    if (!ctxs || !parts || !a || n_boxes < 1 || n_steps < 1 || n_streams < 1 || n_streams > 64)
        return CUBE2_ERR_BAD_ARG;
    for (int b = 0; b < n_boxes; ++b) {
        if (!ctxs[b] || !parts[b]) return CUBE2_ERR_BAD_ARG;
        if (ctxs[b]->prof) return cube2::set_error(ctxs[b], CUBE2_ERR_STATE, "profiling must be off to record an ensemble");
        if (ctxs[b]->device != ctxs[0]->device) return cube2::set_error(ctxs[b], CUBE2_ERR_BAD_ARG, "boxes on different devices");
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
    e = cudaStreamCreateWithFlags(&E->origin, cudaStreamNonBlocking);
    E->branches.assign(nbr, nullptr);
    E->events.assign(nbr + 1, nullptr);
    for (int k = 0; k < nbr && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&E->branches[k], cudaStreamNonBlocking);
    for (int k = 0; k <= nbr && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&E->events[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ensemble_free(E);
        return cube2::cuda_error(ctxs[0], e, "ensemble streams");
    }

    int status = CUBE2_OK;
    e = cudaStreamBeginCapture(E->origin, cudaStreamCaptureModeThreadLocal);
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
        E->particle_steps += (int64_t)n_steps * c->N;
    }
    for (int k = 0; k < nbr && e == cudaSuccess && status == CUBE2_OK; ++k) {
        e = cudaEventRecord(E->events[k], E->branches[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(E->origin, E->events[k], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(E->origin, &g);
    E->graph = g;
    if (e == cudaSuccess) e = ec;
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
