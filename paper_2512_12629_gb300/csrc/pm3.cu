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
//   deposit  one CTA per (z-slab, slot): the IOS cells under the slab's band of
//            the local box, one warp per cell, exact integer CIC at 2^-16 of a
//            local cell into 64-bit shared-memory sums (the local cell is a
//            power-of-two fraction of the IOS cell, so positions are exact
//            fixed point and the sum is order-free), then the slab's planes
//            written once as FP32 density V_p/H_3^3 sum_i W
//   solve    the FFT passes of the global levels, batched over the slots
//            (blocks of unused slots return at once)
//   gather   one CTA per slot, a warp per x-row of the subtile's IOS cells:
//            the 4-point difference of Eq. (diff) at each particle's 8 CIC
//            cells, F += -H_3 E.
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

// Owner-computes local deposit: CTA (slab, slot) owns `slab` consecutive
// z-planes of the slot's local mesh, accumulates the exact integer CIC weights
// that land in them in shared memory (64-bit sums as two 32-bit words, the
// high word taking the low word's carry), and writes its planes once as FP32
// density.  It visits the particles whose z-position lies within half a local
// cell of its planes (and, for the first and last planes, the band that wraps
// around the periodic local mesh): every particle is visited by at most three
// CTAs, with no global atomics.
__global__ void __launch_bounds__(256) pm3_slab_deposit_kernel(
    const uint16_t *__restrict__ off0, const uint16_t *__restrict__ off1, const uint16_t *__restrict__ off2,
    const int32_t *__restrict__ cnt, const int32_t *__restrict__ start, const int32_t *__restrict__ list,
    const int *__restrict__ count, Pm3Geo g, int slab, float *__restrict__ real, float scale, int *status) {
    const int slot = blockIdx.y;
    if (slot >= count[0]) return;
    const int m = g.m, n = g.n_ios;
    const int z0 = blockIdx.x * slab;
    const int nz = min(slab, m - z0);
    if (nz <= 0) return;
    extern __shared__ unsigned int sw[];
    const int plane = m * m;
    unsigned int *lo = sw, *hi = sw + slab * plane;
    for (int i = threadIdx.x; i < 2 * slab * plane; i += blockDim.x) sw[i] = 0u;
    const int sub = list[slot];
    const int sxyz[3] = {sub % g.ns, (sub / g.ns) % g.ns, sub / (g.ns * g.ns)};
    const int64_t q = (int64_t)1 << (FIX_BITS - g.q_shift);   // one local cell, fixed point
    const int64_t extent = (int64_t)m * q;
    int64_t org[3];
    int c_lo[2], span[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) org[d] = local_origin(g, sxyz[d]);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        c_lo[d] = (int)(org[d] >> FIX_BITS);
        span[d] = min((int)(((org[d] & (FIX - 1)) + extent + FIX - 1) >> FIX_BITS), n);
    }
    __syncthreads();
    // z bands (fixed point, relative to the local origin): the planes +- one cell,
    // and the wrapped band for the first or last plane of the mesh
    int64_t ba[3], bb[3];
    int nb = 0;
    ba[nb] = max((int64_t)0, (int64_t)(z0 - 1) * q);
    bb[nb] = min(extent, (int64_t)(z0 + nz + 1) * q);
    ++nb;
    // (a wrap band that meets the main band adds nothing: the main band holds it)
    if (z0 == 0 && extent - q >= bb[0]) { ba[nb] = extent - q; bb[nb] = extent; ++nb; }
    if (z0 + nz == m && q <= ba[0]) { ba[nb] = 0; bb[nb] = q; ++nb; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int bi = 0; bi < nb; ++bi) {
        if (bb[bi] <= ba[bi]) continue;
        // IOS z-planes holding fixed-point z in [org + ba, org + bb)
        const int64_t za = org[2] + ba[bi], zb = org[2] + bb[bi] - 1;
        const int pz0 = (int)(za >> FIX_BITS), npz = (int)((zb >> FIX_BITS) - (za >> FIX_BITS)) + 1;
        const int ncell = span[0] * span[1] * npz;
        for (int k = warp; k < ncell; k += nw) {
            const int kx = k % span[0], ky = (k / span[0]) % span[1], kz = k / (span[0] * span[1]);
            const int cx = wrap(c_lo[0] + kx, n), cy = wrap(c_lo[1] + ky, n);
            const int cz = (int)(((int64_t)pz0 + kz) % n);
            const int64_t c = ((int64_t)cz * n + cy) * n + cx;
            const int b = __ldg(&start[c]), e = b + __ldg(&cnt[c]);
            const int cc[3] = {cx, cy, cz};
            for (int j = b + lane; j < e; j += 32) {
                const unsigned o[3] = {off0[j], off1[j], off2[j]};
                int i0[3], w1[3];
                bool inside = true;
                int64_t relz = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    int64_t rel = (int64_t)cc[d] * FIX + o[d] - org[d];
                    if (rel < 0) rel += g.period;
                    inside = inside && rel < extent;
                    if (d == 2) relz = rel;
                    const int64_t t = (rel << g.q_shift) - (FIX >> 1);
                    const int64_t fl = t >> FIX_BITS;
                    i0[d] = (int)fl;
                    w1[d] = (int)(t - (fl << FIX_BITS));
                }
                if (!inside || relz < ba[bi] || relz >= bb[bi]) continue;
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    const int iz = wrap(i0[2] + dz, m) - z0;
                    if (iz < 0 || iz >= nz) continue;
                    const unsigned long long wz = dz ? w1[2] : FIX - w1[2];
#pragma unroll
                    for (int dy = 0; dy < 2; ++dy) {
                        const int iy = wrap(i0[1] + dy, m);
                        const unsigned long long wyz = wz * (unsigned long long)(dy ? w1[1] : FIX - w1[1]);
#pragma unroll
                        for (int dx = 0; dx < 2; ++dx) {
                            const int ix = wrap(i0[0] + dx, m);
                            const unsigned long long w = wyz * (unsigned long long)(dx ? w1[0] : FIX - w1[0]);
                            if (!w) continue;
                            const int cell = (iz * m + iy) * m + ix;
                            const unsigned int wl = (unsigned int)w, wh = (unsigned int)(w >> 32);
                            const unsigned int old = atomicAdd(&lo[cell], wl);
                            const unsigned int add_hi = wh + ((old + wl < old) ? 1u : 0u);
                            if (add_hi) {
                                const unsigned int oldh = atomicAdd(&hi[cell], add_hi);
                                if (oldh + add_hi < oldh) set_status(status, ST_CAPACITY);
                            }
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    float *out = real + (int64_t)slot * g.m3 + (int64_t)z0 * plane;
    for (int i = threadIdx.x; i < nz * plane; i += blockDim.x) {
        const unsigned long long v = ((unsigned long long)hi[i] << 32) | lo[i];
        out[i] = (float)v * scale;
    }
}

// -H_3 (D * phi) at the particles of one refined subtile per CTA: a warp per
// x-row of the subtile's IOS cells (their particles are contiguous).
__global__ void __launch_bounds__(256) pm3_slot_gather_kernel(
    const uint16_t *__restrict__ off0, const uint16_t *__restrict__ off1, const uint16_t *__restrict__ off2,
    const int32_t *__restrict__ cellid, const int32_t *__restrict__ cnt, const int32_t *__restrict__ start,
    const int32_t *__restrict__ list, const int *__restrict__ count, const float *__restrict__ phi, Pm3Geo g,
    float h3, float *__restrict__ acc0, float *__restrict__ acc1, float *__restrict__ acc2) {
    // grid: (row chunks, slots); the subtile's T^2 rows of IOS cells are dealt
    // to the warps of all its chunks so that a dense subtile spreads over SMs
    const int slot = blockIdx.y;
    if (slot >= count[0]) return;
    const int n = g.n_ios, T = g.T, m = g.m;
    const int sub = list[slot];
    const int sxyz[3] = {sub % g.ns, (sub / g.ns) % g.ns, sub / (g.ns * g.ns)};
    int64_t org[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) org[d] = local_origin(g, sxyz[d]);
    const float *P = phi + (int64_t)slot * g.m3;
    const int lane = threadIdx.x & 31, nw = (blockDim.x >> 5) * gridDim.x;
    const int warp = (threadIdx.x >> 5) + (blockDim.x >> 5) * blockIdx.x;
    for (int r = warp; r < T * T; r += nw) {
        const int cy = sxyz[1] * T + r % T, cz = sxyz[2] * T + r / T;
        const int64_t c0 = ((int64_t)cz * n + cy) * n + (int64_t)sxyz[0] * T;
        const int b = __ldg(&start[c0]), e = __ldg(&start[c0 + T - 1]) + __ldg(&cnt[c0 + T - 1]);
        for (int i = b + lane; i < e; i += 32) {
            const int cx = cellid[i] % n;
            const int cc[3] = {cx, cy, cz};
            const unsigned o[3] = {off0[i], off1[i], off2[i]};
            int i0[3];
            float w1[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int64_t rel = (int64_t)cc[d] * FIX + o[d] - org[d];
                if (rel < 0) rel += g.period;
                const int64_t t = (rel << g.q_shift) - (FIX >> 1);
                const int64_t fl = t >> FIX_BITS;
                i0[d] = (int)fl;
                w1[d] = (float)(t - (fl << FIX_BITS)) * (1.0f / FIX);
            }
            float e3[3] = {0.f, 0.f, 0.f};
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
                            e3[d] += w * (2.0f / 3.0f * (v[2] - v[1]) - 1.0f / 12.0f * (v[3] - v[0]));
                        }
                    }
                }
            }
            acc0[i] += -h3 * e3[0];
            acc1[i] += -h3 * e3[1];
            acc2[i] += -h3 * e3[2];
        }
    }
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

// z-planes of a local mesh per deposit CTA: as many as fit in 96 KB of shared
// 64-bit accumulators, at most 8
int pm3_slab_planes(int m) { return std::max(1, std::min(8, (96 * 1024) / (8 * m * m))); }

cudaError_t launch_pm3(cube2_ctx *ctx, const cube2_particles *p) {
    PM3 &M = ctx->pm3;
    const Pm3Geo g = pm3_geo(ctx);
    cudaError_t e = launch_pm3_map(ctx, p);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof(ctx, P_PM3_DEPOSIT, 0);
        const int slab = pm3_slab_planes(g.m);
        const size_t smem = (size_t)2 * slab * g.m * g.m * sizeof(unsigned int);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(pm3_slab_deposit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
            attr = true;
        }
        pm3_slab_deposit_kernel<<<dim3((unsigned)((g.m + slab - 1) / slab), (unsigned)M.max_tiles), 256, smem,
                                  ctx->stream>>>(p->off[0], p->off[1], p->off[2], p->count, p->start, M.list, M.count,
                                                 g, slab, M.lev.real, M.dens_scale, ctx->dev_status);
        ctx->launches += 1;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    {
        ProfScope prof(ctx, P_PM3_FFT, 0);
        e = launch_fft_batched_solve(ctx, M.lev);
    }
    if (e != cudaSuccess || ctx->N == 0) return e;
    ProfScope prof(ctx, P_PM3_GATHER, 0);
    const unsigned chunks = (unsigned)std::max(1, std::min(8, (M.T * M.T + 7) / 8));   // a row per warp at most
    pm3_slot_gather_kernel<<<dim3(chunks, (unsigned)M.max_tiles), 256, 0, ctx->stream>>>(
        p->off[0], p->off[1], p->off[2], ctx->cellid, p->count, p->start, M.list, M.count, M.lev.real, g, (float)M.H,
        p->acc[0], p->acc[1], p->acc[2]);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace cube2
