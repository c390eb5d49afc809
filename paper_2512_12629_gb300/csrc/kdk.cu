// Kick, fixed-point drift and IOS re-binning of the kick-drift-kick step (paper
// Secs. 2.2.3 and 2.3; constant Delta a, Sec. 3.2).
//
// Drift: X_d <- (X_d + rint(p_d Dr 2^16 / s_ios)) mod n_ios 2^16 (round half to
// even), X_d = c_d 2^16 + off_d.  Re-bin: a stable counting sort by the new
// cell id (ties keep the previous order) rebuilds count/start and permutes the
// offsets and momenta, so the IOS order stays the cell list.
//   1. kick_drift : new coordinates into scratch; ncount[new cell] += 1; flag
//                   any particle that moved more than one cell along an axis
//   2. scan       : nstart = exclusive prefix sum of ncount (multi-level)
//   3a. local re-bin (no far mover): one thread per new cell c walks the 27
//       old cells around c in increasing old-cell id, each in particle order,
//       and keeps the particles whose new cell is c.  Old order is (old cell,
//       rank), so this emits exactly the stable order, with no atomics and no
//       sort, and writes the permuted offsets/momenta directly.
//   3b. general re-bin (some far mover; the kernels of 3a return at once):
//       perm[nstart[cell] + atomic slot] = i, each cell's perm segment sorted
//       by old index, then gathered.  The flag is read on the device, so the
//       step needs no host synchronisation.
//   4. ncount/nstart copied into the caller's count/start.
#include "common.cuh"

namespace cube2 {
namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;   // 4096 elements per block

__global__ void kick_kernel(float *v0, float *v1, float *v2, const float *a0, const float *a1,
                            const float *a2, int64_t n, float kick, int *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = v0[i] + kick * a0[i], y = v1[i] + kick * a1[i], z = v2[i] + kick * a2[i];
    v0[i] = x;
    v1[i] = y;
    v2[i] = z;
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) set_status(status, ST_NONFINITE);
}

struct DriftParams {
    const uint16_t *off0, *off1, *off2;
    const float *vel0, *vel1, *vel2;
    const float *acc0, *acc1, *acc2;
    const int32_t *cellid;
    int32_t *count;           // zeroed before the launch, receives the new histogram
    int *far;
    uint16_t *toff;           // [3][N]
    float *tvel;              // [3][N]
    int32_t *tcell, *tslot;
    int64_t N;
    int n_ios;
    float kick, drift_fix;    // drift_fix = Dr 2^16 / s_ios
    int *status;
};

__global__ void __launch_bounds__(256) kick_drift_kernel(DriftParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int n = P.n_ios;
    const int c = P.cellid[i];
    const int cc[3] = {c % n, (c / n) % n, c / (n * n)};
    const uint16_t off[3] = {P.off0[i], P.off1[i], P.off2[i]};
    const float v[3] = {P.vel0[i] + P.kick * P.acc0[i], P.vel1[i] + P.kick * P.acc1[i],
                        P.vel2[i] + P.kick * P.acc2[i]};
    const int period = n * FIX;
    int nc[3];
    uint16_t no[3];
    bool bad = false, far = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = v[a] * P.drift_fix;
        if (!(fabsf(d) < 0.5f * (float)period)) bad = true;   // also catches NaN
        const int disp = bad ? 0 : __float2int_rn(d);
        int X = cc[a] * FIX + (int)off[a] + disp;
        X = X < 0 ? X + period : (X >= period ? X - period : X);
        nc[a] = X >> FIX_BITS;
        no[a] = (uint16_t)(X & (FIX - 1));
        const int dc = nc[a] - cc[a];
        if (!(dc == 0 || dc == 1 || dc == -1 || dc == n - 1 || dc == 1 - n)) far = true;
    }
    if (far) *P.far = 1;
    if (bad) set_status(P.status, isfinite(v[0] + v[1] + v[2]) ? ST_DISPLACEMENT : ST_NONFINITE);
    const int cell = (nc[2] * n + nc[1]) * n + nc[0];
    const int slot = atomicAdd(&P.count[cell], 1);
    P.toff[i] = no[0];
    P.toff[P.N + i] = no[1];
    P.toff[2 * P.N + i] = no[2];
    P.tvel[i] = v[0];
    P.tvel[P.N + i] = v[1];
    P.tvel[2 * P.N + i] = v[2];
    P.tcell[i] = cell;
    P.tslot[i] = slot;
}

// -------------------------------------------------------------- scan
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sums[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == nw - 1) warp_sums[32] = wi;
    }
    __syncthreads();
    const int out = warp_sums[warp] + incl - v;
    total = warp_sums[32];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const int32_t *in, int32_t *sums, int64_t n) {
    __shared__ int ws[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) s += (base + k < n) ? in[base + k] : 0;
    int total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// exclusive scan of in[0, n) into out, adding offsets[blockIdx] (if non-null)
__global__ void __launch_bounds__(SCAN_THREADS) scan_apply_kernel(const int32_t *in, int32_t *out, int64_t n,
                                                                  const int32_t *offsets) {
    __shared__ int ws[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan(s, ws, total) + (offsets ? offsets[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ------------------------------------------------------------- rebin
__global__ void scatter_kernel(const int32_t *tcell, const int32_t *tslot, const int32_t *start,
                               int32_t *perm, int64_t n, const int *far) {
    if (!*far) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[start[tcell[i]] + tslot[i]] = (int32_t)i;
}

// Sort each cell's segment of perm ascending (old index = stable order).  One
// thread per cell, insertion sort: segments are short and arrive nearly sorted.
__global__ void sort_cells_kernel(const int32_t *count, const int32_t *start, int32_t *perm, int64_t n_cells,
                                  const int *far) {
    if (!*far) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int cnt = count[c];
    if (cnt < 2) return;
    int32_t *seg = perm + start[c];
    for (int a = 1; a < cnt; ++a) {
        const int32_t key = seg[a];
        int b = a - 1;
        while (b >= 0 && seg[b] > key) {
            seg[b + 1] = seg[b];
            --b;
        }
        seg[b + 1] = key;
    }
}

struct GatherParams {
    const int32_t *perm, *tcell;
    const uint16_t *toff;
    const float *tvel;
    uint16_t *off0, *off1, *off2;
    float *vel0, *vel1, *vel2;
    int32_t *cellid;
    int64_t N;
    const int *far;
};

__global__ void gather_kernel(GatherParams P) {
    if (!*P.far) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int64_t j = P.perm[i];
    P.off0[i] = P.toff[j];
    P.off1[i] = P.toff[P.N + j];
    P.off2[i] = P.toff[2 * P.N + j];
    P.vel0[i] = P.tvel[j];
    P.vel1[i] = P.tvel[P.N + j];
    P.vel2[i] = P.tvel[2 * P.N + j];
    P.cellid[i] = P.tcell[j];
}

struct LocalParams {
    const int32_t *ocount, *ostart;   // old cell list
    const int32_t *ncount, *nstart;   // new cell list
    const int32_t *tcell;
    const uint16_t *toff;
    const float *tvel;
    uint16_t *off0, *off1, *off2;
    float *vel0, *vel1, *vel2;
    int32_t *cellid;
    int64_t N, n_cells;
    int n_ios;
    const int *far;
};

// the three wrapped neighbour coordinates of c in increasing order
__device__ __forceinline__ void sorted_neighbours(int c, int n, int out[3]) {
    if (c == 0) { out[0] = 0; out[1] = 1; out[2] = n - 1; }
    else if (c == n - 1) { out[0] = 0; out[1] = n - 2; out[2] = n - 1; }
    else { out[0] = c - 1; out[1] = c; out[2] = c + 1; }
}

__global__ void __launch_bounds__(256) rebin_local_kernel(LocalParams P) {
    if (*P.far) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.n_cells) return;
    const int cnt = P.ncount[c];
    if (cnt == 0) return;
    const int n = P.n_ios;
    const int cx = (int)(c % n), cy = (int)((c / n) % n), cz = (int)(c / ((int64_t)n * n));
    int xs[3], ys[3], zs[3];
    sorted_neighbours(cx, n, xs);
    sorted_neighbours(cy, n, ys);
    sorted_neighbours(cz, n, zs);
    int64_t out = P.nstart[c];
    const int64_t end = out + cnt;
    const int32_t me = (int32_t)c;
    for (int a = 0; a < 3 && out < end; ++a) {
        for (int b = 0; b < 3 && out < end; ++b) {
            const int64_t row = ((int64_t)zs[a] * n + ys[b]) * n;
            for (int e = 0; e < 3 && out < end; ++e) {
                const int64_t o = row + xs[e];
                const int s = P.ostart[o], stop = s + P.ocount[o];
                for (int j = s; j < stop; ++j) {
                    if (P.tcell[j] != me) continue;
                    P.off0[out] = P.toff[j];
                    P.off1[out] = P.toff[P.N + j];
                    P.off2[out] = P.toff[2 * P.N + j];
                    P.vel0[out] = P.tvel[j];
                    P.vel1[out] = P.tvel[P.N + j];
                    P.vel2[out] = P.tvel[2 * P.N + j];
                    P.cellid[out] = me;
                    if (++out == end) break;
                }
            }
        }
    }
}

}  // namespace

int64_t scan_scratch_len(int64_t n) {
    int64_t total = 0;
    while (n > SCAN_CHUNK) {
        n = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
        total += n;
    }
    return total + 1;
}

cudaError_t launch_scan(cube2_ctx *ctx, const int32_t *in, int32_t *out, int64_t n) {
    if (n <= SCAN_CHUNK) {
        scan_apply_kernel<<<1, SCAN_THREADS, 0, ctx->stream>>>(in, out, n, nullptr);
        ctx->launches++;
        return cudaGetLastError();
    }
    // level sums live in ctx->scan_tmp, consumed recursively
    const int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    int32_t *sums = ctx->scan_tmp;
    // reserve this level's sums, recurse on the remainder of the scratch
    scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, sums, n);
    ctx->launches++;
    int32_t *saved = ctx->scan_tmp;
    ctx->scan_tmp = saved + nb;
    cudaError_t e = launch_scan(ctx, sums, sums, nb);
    ctx->scan_tmp = saved;
    if (e != cudaSuccess) return e;
    scan_apply_kernel<<<(unsigned)nb, SCAN_THREADS, 0, ctx->stream>>>(in, out, n, sums);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_kick(cube2_ctx *ctx, const cube2_particles *p, float kick) {
    const int64_t blocks = (ctx->N + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    ProfScope prof(ctx, P_KICK, 0);
    kick_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(p->vel[0], p->vel[1], p->vel[2], p->acc[0], p->acc[1],
                                                          p->acc[2], ctx->N, kick, ctx->dev_status);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_kick_drift(cube2_ctx *ctx, const cube2_particles *p, float kick, float drift_fix) {
    DriftParams P{};
    P.off0 = p->off[0]; P.off1 = p->off[1]; P.off2 = p->off[2];
    P.vel0 = p->vel[0]; P.vel1 = p->vel[1]; P.vel2 = p->vel[2];
    P.acc0 = p->acc[0]; P.acc1 = p->acc[1]; P.acc2 = p->acc[2];
    P.cellid = ctx->cellid;
    P.count = ctx->ncount;
    P.far = ctx->far;
    P.toff = ctx->toff;
    P.tvel = ctx->tvel;
    P.tcell = ctx->tcell;
    P.tslot = ctx->tslot;
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.kick = kick;
    P.drift_fix = drift_fix;
    P.status = ctx->dev_status;
    ProfScope prof(ctx, P_KICK_DRIFT, 0);
    cudaError_t e = cudaMemsetAsync(ctx->ncount, 0, sizeof(int32_t) * ctx->n_cells, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->far, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (ctx->N + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    kick_drift_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_rebin(cube2_ctx *ctx, const cube2_particles *p) {
    cudaError_t e;
    {
        ProfScope prof(ctx, P_SCAN, 0);
        e = launch_scan(ctx, ctx->ncount, ctx->nstart, ctx->n_cells);
    }
    if (e != cudaSuccess) return e;
    const int64_t pb = (ctx->N + 255) / 256, cb = (ctx->n_cells + 255) / 256;
    if (pb > 0) {
        {
            ProfScope prof(ctx, P_GATHER, 0);
            LocalParams L{};
            L.ocount = p->count; L.ostart = p->start;
            L.ncount = ctx->ncount; L.nstart = ctx->nstart;
            L.tcell = ctx->tcell; L.toff = ctx->toff; L.tvel = ctx->tvel;
            L.off0 = p->off[0]; L.off1 = p->off[1]; L.off2 = p->off[2];
            L.vel0 = p->vel[0]; L.vel1 = p->vel[1]; L.vel2 = p->vel[2];
            L.cellid = ctx->cellid;
            L.N = ctx->N;
            L.n_cells = ctx->n_cells;
            L.n_ios = ctx->n_ios;
            L.far = ctx->far;
            rebin_local_kernel<<<(unsigned)cb, 256, 0, ctx->stream>>>(L);
            ctx->launches++;
        }
        {
            ProfScope prof(ctx, P_SCATTER, 0);
            scatter_kernel<<<(unsigned)pb, 256, 0, ctx->stream>>>(ctx->tcell, ctx->tslot, ctx->nstart, ctx->perm,
                                                                  ctx->N, ctx->far);
        }
        {
            ProfScope prof(ctx, P_SORT, 0);
            sort_cells_kernel<<<(unsigned)cb, 256, 0, ctx->stream>>>(ctx->ncount, ctx->nstart, ctx->perm,
                                                                     ctx->n_cells, ctx->far);
        }
        GatherParams G{};
        G.perm = ctx->perm;
        G.tcell = ctx->tcell;
        G.toff = ctx->toff;
        G.tvel = ctx->tvel;
        G.off0 = p->off[0]; G.off1 = p->off[1]; G.off2 = p->off[2];
        G.vel0 = p->vel[0]; G.vel1 = p->vel[1]; G.vel2 = p->vel[2];
        G.cellid = ctx->cellid;
        G.N = ctx->N;
        G.far = ctx->far;
        {
            ProfScope prof(ctx, P_GATHER, 0);
            gather_kernel<<<(unsigned)pb, 256, 0, ctx->stream>>>(G);
        }
        ctx->launches += 3;
    }
    e = cudaMemcpyAsync(p->count, ctx->ncount, sizeof(int32_t) * ctx->n_cells, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->start, ctx->nstart, sizeof(int32_t) * ctx->n_cells, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace cube2
