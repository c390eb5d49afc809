// Adaptive third PM level (paper Sec. 2.1.1 Eq. PM3; Sec. 2.2.3, local force and
// the resolution chosen from rho_max).
//
// The box of n_ios^3 IOS cells is cut into subtiles of T^3 IOS cells.  A
// subtile whose densest IOS cell holds at least rho_min particles is refined:
// it gets a local periodic mesh of spacing H_3 = H_finest / r over the
// subtile plus a buffer of B local cells on each side (m^3 cells in all),
// softening b_3 = beta_3 H_3 and the kernel R(r, b_3) - R(r, b_finest) of
// Eq. (PM3) in its Green's table (Eq. Gk with the truncation at the finest
// global softening).  Every particle inside the local box is a source; the
// subtile's own particles receive the force, and their PP range (Eq. PP)
// shrinks from b_finest to b_3.  Unrefined subtiles keep the two-level method.
//
// Steps, all asynchronous on the context stream:
//   map      per subtile the densest IOS cell (one warp per subtile), an
//            exclusive scan of the refinement flags, and the slot of each
//            refined subtile (subtile order; slots beyond the capacity stay
//            unrefined); the number of slots in use stays on the device.
//   deposit  one CTA per slot: the IOS cells under the local box, one warp per
//            cell, exact integer CIC at 2^-16 of a local cell into uint64
//            accumulators (the local cell is a power-of-two fraction of the IOS
//            cell, so positions are exact fixed point and the sum is order-free)
//   convert  accumulator -> FP32 density V_p/H_3^3 sum_i W, and the
//            accumulator back to zero for the next evaluation
//   solve    the FFT passes of the global levels, batched over the slots
//            (blocks of unused slots return at once)
//   gather   one thread per particle of a refined subtile: the 4-point
//            difference of Eq. (diff) at its 8 CIC cells, F += -H_3 E.
#include "common.cuh"

#include <algorithm>

namespace cube2 {
namespace {

struct Pm3Geo {
    int n_ios, T, ns, m, B, q_shift;
    int64_t period;          // n_ios 2^16
    int64_t m3;
};

__host__ __device__ inline Pm3Geo pm3_geo(const cube2_ctx *ctx) {
    Pm3Geo g;
    g.n_ios = ctx->n_ios;
    g.T = ctx->pm3.T;
    g.ns = ctx->pm3.ns;
    g.m = ctx->pm3.m;
    g.B = ctx->pm3.B;
    g.q_shift = ctx->pm3.q_shift;
    g.period = (int64_t)ctx->n_ios << FIX_BITS;
    g.m3 = (int64_t)g.m * g.m * g.m;
    return g;
}

// Fixed-point origin (one axis) of the local box of subtile coordinate s:
// s T 2^16 - B q, wrapped into [0, period).
__device__ __forceinline__ int64_t local_origin(const Pm3Geo &g, int s) {
    const int64_t q = (int64_t)1 << (FIX_BITS - g.q_shift);
    int64_t o = (int64_t)s * g.T * FIX - (int64_t)g.B * q;
    o %= g.period;
    return o < 0 ? o + g.period : o;
}

// x mod m in [0, m) for any int x (local mesh indices are periodic)
__device__ __forceinline__ int mod_mesh(int x, int m) {
    x %= m;
    return x < 0 ? x + m : x;
}

__global__ void __launch_bounds__(256) pm3_rho_max_kernel(const int32_t *__restrict__ count, Pm3Geo g, int rho_min,
                                                          int32_t *__restrict__ rho_max, int32_t *__restrict__ flag,
                                                          int64_t n_sub) {
    const int64_t sub = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (sub >= n_sub) return;
    const int sx = (int)(sub % g.ns), sy = (int)((sub / g.ns) % g.ns), sz = (int)(sub / ((int64_t)g.ns * g.ns));
    const int T = g.T, n = g.n_ios;
    int mx = 0;
    for (int k = lane; k < T * T * T; k += 32) {
        const int x = k % T, y = (k / T) % T, z = k / (T * T);
        const int64_t c = ((int64_t)(sz * T + z) * n + (sy * T + y)) * n + (sx * T + x);
        mx = max(mx, __ldg(&count[c]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        rho_max[sub] = mx;
        flag[sub] = mx >= rho_min ? 1 : 0;
    }
}

// slot[] holds the exclusive scan of the flags on entry; on exit the slot of
// each subtile (-1: not refined), list[slot] = subtile, count = {slots in use,
// subtiles that asked}.
__global__ void __launch_bounds__(256) pm3_slot_kernel(const int32_t *__restrict__ rho_max, int rho_min,
                                                       int32_t *__restrict__ slot, int32_t *__restrict__ list,
                                                       int *__restrict__ count, int64_t n_sub, int max_tiles) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sub) return;
    const int flag = rho_max[s] >= rho_min ? 1 : 0;
    const int k = slot[s];
    const bool use = flag && k < max_tiles;
    if (use) list[k] = (int32_t)s;
    slot[s] = use ? k : -1;
    if (s == n_sub - 1) {
        const int total = k + flag;
        count[0] = total < max_tiles ? total : max_tiles;
        count[1] = total;
    }
}

constexpr int PM3_DEP_THREADS = 512;

__global__ void __launch_bounds__(PM3_DEP_THREADS) pm3_deposit_kernel(
    const uint16_t *__restrict__ off0, const uint16_t *__restrict__ off1, const uint16_t *__restrict__ off2,
    const int32_t *__restrict__ cnt, const int32_t *__restrict__ start, const int32_t *__restrict__ list,
    const int *__restrict__ count, Pm3Geo g, unsigned long long *__restrict__ acc, int *status) {
    const int slot = blockIdx.x;
    if (slot >= count[0]) return;
    const int sub = list[slot];
    const int sxyz[3] = {sub % g.ns, (sub / g.ns) % g.ns, sub / (g.ns * g.ns)};
    int64_t org[3];
    int c_lo[3], span[3];
    const int64_t extent = (int64_t)g.m << (FIX_BITS - g.q_shift);   // local box side, fixed point
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        org[d] = local_origin(g, sxyz[d]);
        c_lo[d] = (int)(org[d] >> FIX_BITS);
        span[d] = (int)(((org[d] & (FIX - 1)) + extent + FIX - 1) >> FIX_BITS);
        if (span[d] > g.n_ios) span[d] = g.n_ios;
    }
    unsigned long long *a = acc + (int64_t)slot * g.m3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ncell = span[0] * span[1] * span[2];
    const int n = g.n_ios, m = g.m;
    for (int k = warp; k < ncell; k += nw) {
        const int kx = k % span[0], ky = (k / span[0]) % span[1], kz = k / (span[0] * span[1]);
        const int cx = wrap(c_lo[0] + kx, n), cy = wrap(c_lo[1] + ky, n), cz = wrap(c_lo[2] + kz, n);
        const int64_t c = ((int64_t)cz * n + cy) * n + cx;
        const int b = __ldg(&start[c]), e = b + __ldg(&cnt[c]);
        const int cc[3] = {cx, cy, cz};
        for (int j = b + lane; j < e; j += 32) {
            const unsigned o[3] = {off0[j], off1[j], off2[j]};
            int i0[3], w1[3];
            bool inside = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int64_t rel = (int64_t)cc[d] * FIX + o[d] - org[d];
                if (rel < 0) rel += g.period;
                inside = inside && rel < extent;
                const int64_t t = (rel << g.q_shift) - (FIX >> 1);   // local cells, 16 fractional bits
                const int64_t fl = t >> FIX_BITS;                    // floor, t may be negative
                i0[d] = (int)fl;
                w1[d] = (int)(t - (fl << FIX_BITS));
            }
            if (!inside) continue;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {
                const int iz = wrap(i0[2] + dz, m);
                const unsigned long long wz = dz ? w1[2] : FIX - w1[2];
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const int iy = wrap(i0[1] + dy, m);
                    const unsigned long long wyz = wz * (unsigned long long)(dy ? w1[1] : FIX - w1[1]);
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int ix = wrap(i0[0] + dx, m);
                        const unsigned long long w = wyz * (unsigned long long)(dx ? w1[0] : FIX - w1[0]);
                        if (w) {
                            const unsigned long long old = atomicAdd(&a[((int64_t)iz * m + iy) * m + ix], w);
                            if (old + w < old) set_status(status, ST_CAPACITY);
                        }
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) pm3_convert_kernel(unsigned long long *__restrict__ acc,
                                                          float *__restrict__ real, const int *__restrict__ count,
                                                          int64_t m3, float scale) {
    const int slot = blockIdx.y;
    if (slot >= count[0]) return;
    const int64_t base = (int64_t)slot * m3;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m3; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long v = acc[base + i];
        real[base + i] = (float)v * scale;
        acc[base + i] = 0ull;
    }
}

__global__ void __launch_bounds__(256) pm3_gather_kernel(
    const uint16_t *__restrict__ off0, const uint16_t *__restrict__ off1, const uint16_t *__restrict__ off2,
    const int32_t *__restrict__ cellid, const int32_t *__restrict__ slot_of, const float *__restrict__ phi,
    Pm3Geo g, float h3, float *__restrict__ acc0, float *__restrict__ acc1, float *__restrict__ acc2, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = g.n_ios, T = g.T, m = g.m;
    const int c = cellid[i];
    const int cc[3] = {c % n, (c / n) % n, c / (n * n)};
    const int sxyz[3] = {cc[0] / T, cc[1] / T, cc[2] / T};
    const int slot = slot_of[((int64_t)sxyz[2] * g.ns + sxyz[1]) * g.ns + sxyz[0]];
    if (slot < 0) return;
    const unsigned o[3] = {off0[i], off1[i], off2[i]};
    int i0[3];
    float w1[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int64_t rel = (int64_t)cc[d] * FIX + o[d] - local_origin(g, sxyz[d]);
        if (rel < 0) rel += g.period;
        const int64_t t = (rel << g.q_shift) - (FIX >> 1);
        const int64_t fl = t >> FIX_BITS;
        i0[d] = (int)fl;
        w1[d] = (float)(t - (fl << FIX_BITS)) * (1.0f / FIX);
    }
    const float *P = phi + (int64_t)slot * g.m3;
    float e[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const float wz = dz ? w1[2] : 1.0f - w1[2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float wyz = wz * (dy ? w1[1] : 1.0f - w1[1]);
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const float w = wyz * (dx ? w1[0] : 1.0f - w1[0]);
                const int j[3] = {i0[0] + dx, i0[1] + dy, i0[2] + dz};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    float v[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int step = k < 2 ? k - 2 : k - 1;   // -2, -1, +1, +2
                        int jj[3] = {j[0], j[1], j[2]};
                        jj[d] += step;
#pragma unroll
                        for (int a = 0; a < 3; ++a) jj[a] = mod_mesh(jj[a], m);
                        v[k] = __ldg(&P[((int64_t)jj[2] * m + jj[1]) * m + jj[0]]);
                    }
                    e[d] += w * (2.0f / 3.0f * (v[2] - v[1]) - 1.0f / 12.0f * (v[3] - v[0]));
                }
            }
        }
    }
    acc0[i] += -h3 * e[0];
    acc1[i] += -h3 * e[1];
    acc2[i] += -h3 * e[2];
}

}  // namespace

cudaError_t launch_pm3_map(cube2_ctx *ctx, const cube2_particles *p) {
    PM3 &M = ctx->pm3;
    const Pm3Geo g = pm3_geo(ctx);
    ProfScope prof(ctx, P_PM3_MAP, 0);
    const int64_t threads = M.n_sub * 32;
    pm3_rho_max_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->stream>>>(p->count, g, M.rho_min, M.rho_max,
                                                                                   M.slot, M.n_sub);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_scan(ctx, M.slot, M.slot, M.n_sub);
    if (e != cudaSuccess) return e;
    pm3_slot_kernel<<<(unsigned)((M.n_sub + 255) / 256), 256, 0, ctx->stream>>>(M.rho_max, M.rho_min, M.slot, M.list,
                                                                                M.count, M.n_sub, M.max_tiles);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_pm3(cube2_ctx *ctx, const cube2_particles *p) {
    PM3 &M = ctx->pm3;
    const Pm3Geo g = pm3_geo(ctx);
    cudaError_t e = launch_pm3_map(ctx, p);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof(ctx, P_PM3_DEPOSIT, 0);
        pm3_deposit_kernel<<<(unsigned)M.max_tiles, PM3_DEP_THREADS, 0, ctx->stream>>>(
            p->off[0], p->off[1], p->off[2], p->count, p->start, M.list, M.count, g, M.acc, ctx->dev_status);
        const unsigned gx = (unsigned)std::min<int64_t>((g.m3 + 255) / 256, 64);
        pm3_convert_kernel<<<dim3(gx, (unsigned)M.max_tiles), 256, 0, ctx->stream>>>(M.acc, M.lev.real, M.count, g.m3,
                                                                                    M.dens_scale);
        ctx->launches += 2;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    {
        ProfScope prof(ctx, P_PM3_FFT, 0);
        e = launch_fft_batched_solve(ctx, M.lev);
    }
    if (e != cudaSuccess || ctx->N == 0) return e;
    ProfScope prof(ctx, P_PM3_GATHER, 0);
    pm3_gather_kernel<<<(unsigned)((ctx->N + 255) / 256), 256, 0, ctx->stream>>>(
        p->off[0], p->off[1], p->off[2], ctx->cellid, M.slot, M.lev.real, g, (float)M.H, p->acc[0], p->acc[1],
        p->acc[2], ctx->N);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace cube2
