// Kick, fixed-point drift and IOS re-binning of the kick-drift-kick step (paper
// Secs. 2.2.3 and 2.3; constant Delta a, Sec. 3.2).
//
// Drift: X_d <- (X_d + rint(p_d Dr 2^16 / s_ios)) mod n_ios 2^16 (round half to
// even), X_d = c_d 2^16 + off_d.  Re-bin: a stable counting sort by the new
// cell id (ties keep the previous order) rebuilds count/start and permutes the
// offsets and momenta, so the IOS order stays the cell list.
//   1. kick_drift : new coordinates into scratch; slot = ncount[new cell]++
//                   (atomic: a provisional, order-dependent rank in the cell)
//   2. scan       : nstart = exclusive prefix sum of ncount (multi-level)
//   3. scatter    : perm[nstart[cell] + slot] = old index
//   4. sort       : every cell's perm segment sorted by old index, which makes
//                   the result stable and independent of the atomics' order:
//                   cells of <= 32 particles by one thread (insertion sort),
//                   larger ones by a CTA (bitonic in shared memory up to 8192,
//                   beyond that sorted 8192-runs merged through global scratch)
//   5. gather     : off, vel, cellid of new index i from old index perm[i]
//   6. ncount/nstart copied into the caller's count/start
#include "common.cuh"

#include <cuda_fp16.h>

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
    const uint16_t *v16_0, *v16_1, *v16_2;   // FP16 storage (null: FP32 vel)
    const float *vscale;                     // its per-cell scale
    const float *acc0, *acc1, *acc2;
    const int32_t *cellid;
    int32_t *count;           // zeroed before the launch, receives the new histogram
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
    float v0[3];
    if (P.v16_0) {
        const float sc = P.vscale[c];
        v0[0] = __half2float(__ushort_as_half(P.v16_0[i])) * sc;
        v0[1] = __half2float(__ushort_as_half(P.v16_1[i])) * sc;
        v0[2] = __half2float(__ushort_as_half(P.v16_2[i])) * sc;
    } else {
        v0[0] = P.vel0[i];
        v0[1] = P.vel1[i];
        v0[2] = P.vel2[i];
    }
    const float v[3] = {v0[0] + P.kick * P.acc0[i], v0[1] + P.kick * P.acc1[i], v0[2] + P.kick * P.acc2[i]};
    const int period = n * FIX;
    int nc[3];
    uint16_t no[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = v[a] * P.drift_fix;
        if (!(fabsf(d) < 0.5f * (float)period)) bad = true;   // also catches NaN
        const int disp = bad ? 0 : __float2int_rn(d);
        int X = cc[a] * FIX + (int)off[a] + disp;
        X = X < 0 ? X + period : (X >= period ? X - period : X);
        nc[a] = X >> FIX_BITS;
        no[a] = (uint16_t)(X & (FIX - 1));
    }
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

// Placement of arbitrary positions into IOS (the entry of a differentiable
// run): X_d = rint(x_d / s_ios * 2^16) mod n_ios 2^16 in FP64 (round half to
// even), then the same stable counting sort as the re-bin, ties in input order.
struct PlaceParams {
    const double *pos0, *pos1, *pos2;
    const float *mom0, *mom1, *mom2;   // may be null: zero momenta
    int32_t *count;
    uint16_t *toff;
    float *tvel;
    int32_t *tcell, *tslot;
    int64_t N;
    int n_ios;
    double s_ios;
    int *status;
};

__global__ void __launch_bounds__(256) place_kernel(PlaceParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int n = P.n_ios;
    const int64_t period = (int64_t)n * FIX;
    const double x[3] = {P.pos0[i], P.pos1[i], P.pos2[i]};
    int nc[3];
    uint16_t no[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double u = rint(x[a] / P.s_ios * (double)FIX);
        if (!(fabs(u) < 4.0e18)) bad = true;   // also catches NaN
        int64_t X = bad ? 0 : (int64_t)u % period;
        if (X < 0) X += period;
        nc[a] = (int)(X >> FIX_BITS);
        no[a] = (uint16_t)(X & (FIX - 1));
    }
    if (bad) set_status(P.status, ST_NONFINITE);
    const int cell = (nc[2] * n + nc[1]) * n + nc[0];
    const int slot = atomicAdd(&P.count[cell], 1);
    P.toff[i] = no[0];
    P.toff[P.N + i] = no[1];
    P.toff[2 * P.N + i] = no[2];
    P.tvel[i] = P.mom0 ? P.mom0[i] : 0.0f;
    P.tvel[P.N + i] = P.mom1 ? P.mom1[i] : 0.0f;
    P.tvel[2 * P.N + i] = P.mom2 ? P.mom2[i] : 0.0f;
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
                               int32_t *perm, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[start[tcell[i]] + tslot[i]] = (int32_t)i;
}

// Sort each cell's segment of perm ascending (old index = stable order).  One
// thread per cell sorts segments of up to 32 by insertion; cells of up to
// WARP_SORT are listed from the front of `big` for sort_mid_kernel (one warp
// per cell), larger ones from the back for sort_big_kernel (one CTA per cell).
constexpr int SMALL_SORT = 32;
constexpr int WARP_SORT = 1024;
constexpr int MID_WARPS = 8;
constexpr int BIG_SORT_SMEM = 8192;
constexpr int BIG_SORT_THREADS = 512;

__global__ void sort_small_kernel(const int32_t *count, const int32_t *start, int32_t *perm, int64_t n_cells,
                                  int32_t *big, int *big_n) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int cnt = count[c];
    if (cnt < 2) return;
    if (cnt > SMALL_SORT) {
        if (cnt <= WARP_SORT)
            big[atomicAdd(&big_n[0], 1)] = (int32_t)c;
        else
            big[n_cells - 1 - atomicAdd(&big_n[1], 1)] = (int32_t)c;
        return;
    }
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

__device__ void bitonic_smem(int32_t *s, int np2) {
    for (int k = 2; k <= np2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const int32_t a = s[i], b = s[ixj];
                    if ((a > b) == up) { s[i] = b; s[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// sort keys[0, n) (n <= BIG_SORT_SMEM) in place through shared memory
__device__ void sort_run_smem(int32_t *keys, int n, int32_t *s) {
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (int i = threadIdx.x; i < np2; i += blockDim.x) s[i] = i < n ? keys[i] : 0x7fffffff;
    __syncthreads();
    bitonic_smem(s, np2);
    for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = s[i];
    __syncthreads();
}

// merge sorted a[0, la) and b[0, lb) into out (keys unique), CTA-cooperative
__device__ void merge_runs(const int32_t *a, int la, const int32_t *b, int lb, int32_t *out) {
    const int total = la + lb;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int d0 = min(total, (int)threadIdx.x * per), d1 = min(total, d0 + per);
    if (d0 >= d1) return;
    int lo = max(0, d0 - lb), hi = min(d0, la);
    while (lo < hi) {                      // merge-path split of diagonal d0
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= b[d0 - mid - 1]) lo = mid + 1; else hi = mid;
    }
    int i = lo, j = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        if (j >= lb || (i < la && a[i] <= b[j])) out[d] = a[i++];
        else out[d] = b[j++];
    }
}

// Cells of 33 .. WARP_SORT particles: one warp per cell, a bitonic sort of the
// segment (padded to a power of two) in the warp's own shared buffer, every
// lane exchanging pairs at each stage, with warp barriers only.
__global__ void __launch_bounds__(MID_WARPS * 32) sort_mid_kernel(const int32_t *count, const int32_t *start,
                                                                 int32_t *perm, const int32_t *big,
                                                                 const int *big_n) {
    __shared__ int32_t buf[MID_WARPS][WARP_SORT];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *s = buf[w];
    const int total = big_n[0];
    for (int item = blockIdx.x * MID_WARPS + w; item < total; item += gridDim.x * MID_WARPS) {
        const int64_t c = big[item];
        const int n = count[c];
        int32_t *seg = perm + start[c];
        int np2 = 64;
        while (np2 < n) np2 <<= 1;
        for (int i = lane; i < np2; i += 32) s[i] = i < n ? seg[i] : 0x7fffffff;
        __syncwarp();
        for (int k = 2; k <= np2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int q = lane; q < (np2 >> 1); q += 32) {
                    const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));   // lower index of pair q
                    const int ixj = i | j;
                    const bool up = (i & k) == 0;
                    const int32_t a = s[i], b = s[ixj];
                    if ((a > b) == up) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
                __syncwarp();
            }
        for (int i = lane; i < n; i += 32) seg[i] = s[i];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(BIG_SORT_THREADS) sort_big_kernel(const int32_t *count, const int32_t *start,
                                                                    int32_t *perm, int32_t *perm2,
                                                                    const int32_t *big, const int *big_n,
                                                                    int64_t n_cells) {
    __shared__ int32_t s[BIG_SORT_SMEM];
    const int total = big_n[1];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int64_t c = big[n_cells - 1 - item];
        const int n = count[c];
        int32_t *seg = perm + start[c];
        if (n <= BIG_SORT_SMEM) {
            sort_run_smem(seg, n, s);
            continue;
        }
        for (int r = 0; r < n; r += BIG_SORT_SMEM) sort_run_smem(seg + r, min(BIG_SORT_SMEM, n - r), s);
        int32_t *src = seg, *dst = perm2 + start[c];
        for (int w = BIG_SORT_SMEM; w < n; w <<= 1) {
            for (int lo = 0; lo < n; lo += 2 * w) {
                const int la = min(w, n - lo), lb = max(0, min(w, n - lo - w));
                merge_runs(src + lo, la, src + lo + la, lb, dst + lo);
            }
            __syncthreads();
            int32_t *t = src; src = dst; dst = t;
        }
        if (src != seg)
            for (int i = threadIdx.x; i < n; i += blockDim.x) seg[i] = src[i];
        __syncthreads();
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
};

__global__ void gather_kernel(GatherParams P) {
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

// FP16 velocity codec: per IOS cell the FP32 scale max_p,d |v_d| (an atomic
// max on the bit patterns, which order like the values for v >= 0, so the
// result does not depend on order), then code = RN_half(RN32(v / scale)).
__global__ void vel_scale_kernel(const float *__restrict__ v0, const float *__restrict__ v1,
                                 const float *__restrict__ v2, const int32_t *__restrict__ cellid,
                                 float *__restrict__ vscale, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float m = fmaxf(fabsf(v0[i]), fmaxf(fabsf(v1[i]), fabsf(v2[i])));
    atomicMax(reinterpret_cast<int *>(&vscale[cellid[i]]), __float_as_int(m));
}

__global__ void vel_encode_kernel(const float *__restrict__ v0, const float *__restrict__ v1,
                                  const float *__restrict__ v2, const int32_t *__restrict__ cellid,
                                  const float *__restrict__ vscale, uint16_t *__restrict__ c0,
                                  uint16_t *__restrict__ c1, uint16_t *__restrict__ c2, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float s = vscale[cellid[i]];
    if (s > 0.0f) {
        c0[i] = __half_as_ushort(__float2half_rn(__fdiv_rn(v0[i], s)));
        c1[i] = __half_as_ushort(__float2half_rn(__fdiv_rn(v1[i], s)));
        c2[i] = __half_as_ushort(__float2half_rn(__fdiv_rn(v2[i], s)));
    } else {
        c0[i] = c1[i] = c2[i] = 0;
    }
}

__global__ void vel_decode_kernel(const uint16_t *__restrict__ c0, const uint16_t *__restrict__ c1,
                                  const uint16_t *__restrict__ c2, const int32_t *__restrict__ cellid,
                                  const float *__restrict__ vscale, float *__restrict__ v0, float *__restrict__ v1,
                                  float *__restrict__ v2, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float s = vscale[cellid[i]];
    v0[i] = __half2float(__ushort_as_half(c0[i])) * s;
    v1[i] = __half2float(__ushort_as_half(c1[i])) * s;
    v2[i] = __half2float(__ushort_as_half(c2[i])) * s;
}

}  // namespace

// p->vel16 / p->vscale from FP32 momenta v (ctx->cellid must hold p's cells).
cudaError_t launch_vel_encode(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3]) {
    cudaError_t e = cudaMemsetAsync(p->vscale, 0, sizeof(float) * ctx->n_cells, ctx->stream);
    const int64_t blocks = (ctx->N + 255) / 256;
    if (e != cudaSuccess || blocks == 0) return e;
    ProfScope prof(ctx, P_KICK, 0);
    vel_scale_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(v[0], v[1], v[2], ctx->cellid, p->vscale, ctx->N);
    vel_encode_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(v[0], v[1], v[2], ctx->cellid, p->vscale, p->vel16[0],
                                                                p->vel16[1], p->vel16[2], ctx->N);
    ctx->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_vel_decode(cube2_ctx *ctx, const cube2_particles *p, float *const v[3]) {
    const int64_t blocks = (ctx->N + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    vel_decode_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(p->vel16[0], p->vel16[1], p->vel16[2], ctx->cellid,
                                                                p->vscale, v[0], v[1], v[2], ctx->N);
    ctx->launches++;
    return cudaGetLastError();
}

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
    if (ctx->vel32) {
        P.v16_0 = p->vel16[0]; P.v16_1 = p->vel16[1]; P.v16_2 = p->vel16[2];
        P.vscale = p->vscale;
    }
    P.acc0 = p->acc[0]; P.acc1 = p->acc[1]; P.acc2 = p->acc[2];
    P.cellid = ctx->cellid;
    P.count = ctx->ncount;
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
    if (e != cudaSuccess) return e;
    const int64_t blocks = (ctx->N + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    kick_drift_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_place(cube2_ctx *ctx, const double *const pos[3], const float *const mom[3]) {
    PlaceParams P{};
    P.pos0 = pos[0]; P.pos1 = pos[1]; P.pos2 = pos[2];
    if (mom) { P.mom0 = mom[0]; P.mom1 = mom[1]; P.mom2 = mom[2]; }
    P.count = ctx->ncount;
    P.toff = ctx->toff;
    P.tvel = ctx->tvel;
    P.tcell = ctx->tcell;
    P.tslot = ctx->tslot;
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.s_ios = ctx->s_ios;
    P.status = ctx->dev_status;
    cudaError_t e = cudaMemsetAsync(ctx->ncount, 0, sizeof(int32_t) * ctx->n_cells, ctx->stream);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (ctx->N + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    place_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P);
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
            ProfScope prof(ctx, P_SCATTER, 0);
            scatter_kernel<<<(unsigned)pb, 256, 0, ctx->stream>>>(ctx->tcell, ctx->tslot, ctx->nstart, ctx->perm,
                                                                  ctx->N);
        }
        e = cudaMemsetAsync(ctx->big_n, 0, 2 * sizeof(int), ctx->stream);
        if (e != cudaSuccess) return e;
        {
            ProfScope prof(ctx, P_SORT, 0);
            sort_small_kernel<<<(unsigned)cb, 256, 0, ctx->stream>>>(ctx->ncount, ctx->nstart, ctx->perm,
                                                                     ctx->n_cells, ctx->big, ctx->big_n);
        }
        {
            ProfScope prof(ctx, P_SORT_BIG, 0);
            sort_mid_kernel<<<(unsigned)(ctx->num_sms * 6), MID_WARPS * 32, 0, ctx->stream>>>(
                ctx->ncount, ctx->nstart, ctx->perm, ctx->big, ctx->big_n);
            sort_big_kernel<<<(unsigned)(ctx->num_sms * 2), BIG_SORT_THREADS, 0, ctx->stream>>>(
                ctx->ncount, ctx->nstart, ctx->perm, ctx->perm2, ctx->big, ctx->big_n, ctx->n_cells);
        }
        ctx->launches++;
        GatherParams G{};
        G.perm = ctx->perm;
        G.tcell = ctx->tcell;
        G.toff = ctx->toff;
        G.tvel = ctx->tvel;
        G.off0 = p->off[0]; G.off1 = p->off[1]; G.off2 = p->off[2];
        if (ctx->vel32) {   // FP16 storage: the step's FP32 working copy
            G.vel0 = ctx->vel32; G.vel1 = ctx->vel32 + ctx->N; G.vel2 = ctx->vel32 + 2 * ctx->N;
        } else {
            G.vel0 = p->vel[0]; G.vel1 = p->vel[1]; G.vel2 = p->vel[2];
        }
        G.cellid = ctx->cellid;
        G.N = ctx->N;
        {
            ProfScope prof(ctx, P_GATHER, 0);
            gather_kernel<<<(unsigned)pb, 256, 0, ctx->stream>>>(G);
        }
        ctx->launches += 4;
    }
    e = cudaMemcpyAsync(p->count, ctx->ncount, sizeof(int32_t) * ctx->n_cells, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->start, ctx->nstart, sizeof(int32_t) * ctx->n_cells, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace cube2
