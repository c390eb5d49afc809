// Mesh kernels of the force's vector-Jacobian product (the PM part of the
// adjoint; the PP part is pp_vjp in pp.cu).
//
// For one PM level (n^3 cells, positions u in mesh cells, CIC W(u, c) of the
// forward deposit, rho = (n^3/N) sum W, phi = G * rho, E = D * phi with the
// 4-point difference of Eq. diff, F_i = -H sum_c W(u_i, c) E(c)), the product
// w_i = d<v, F>/dx_i of a cotangent v is, by the chain rule,
//
//   w_i = -sum_c grad_u W(u_i, c) (E(c) . v_i) + sum_c grad_u W(u_i, c) psi(c),
//   psi = G * s,   s = (n^3/N) sum_d D_d * mu_d,   mu_d(c) = sum_j W(u_j, c) v_{j,d},
//
// because G is even and D_d odd (the transpose of D_d * G * is -G * D_d *).
// H cancels: the forward multiplies by H, the derivative in x divides by it.
// The IOS quantisation is taken as the identity: W and grad_u W are the
// forward's exact integer CIC weights at the stored positions.
//
// Kernels: vjp_gather (mode E: the first sum with E from phi by the 4-point
// difference; mode PSI: the second sum), mu_deposit (three FP32 fields, float
// atomics, so the sum order and the last bits vary between runs) and
// div_stencil (s, written into the level's real grid for the Poisson solve).
#include "common.cuh"

namespace cube2 {
namespace {

struct CicPoint {
    int i0[3];        // lower corner (mesh cells, may be -1 or n-1 before wrapping)
    float w1[3];      // weight of the upper corner per axis (lower: 1 - w1)
};

__device__ __forceinline__ CicPoint cic_point(const uint16_t *off0, const uint16_t *off1, const uint16_t *off2,
                                              int64_t i, int cell, int n_ios, int shift) {
    const int c[3] = {cell % n_ios, (cell / n_ios) % n_ios, cell / (n_ios * n_ios)};
    const int o[3] = {(int)off0[i], (int)off1[i], (int)off2[i]};
    CicPoint P;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int X = c[d] * FIX + o[d];
        const int xm = shift >= 0 ? (X >> shift) : (X << (-shift));
        const int t = xm - (FIX >> 1);
        P.i0[d] = t >> FIX_BITS;
        P.w1[d] = (float)(t & (FIX - 1)) * (1.0f / FIX);
    }
    return P;
}

__device__ __forceinline__ int wrapn(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

__device__ __forceinline__ float at(const float *g, int n, int x, int y, int z) {
    return __ldg(&g[((int64_t)wrapn(z, n) * n + wrapn(y, n)) * n + wrapn(x, n)]);
}

struct VjpParams {
    const uint16_t *off0, *off1, *off2;
    const int32_t *cellid;
    const float *v0, *v1, *v2;
    float *w0, *w1, *w2;
    const float *grid;       // phi (mode E) or psi (mode PSI)
    float scale;             // factor on the gathered gradient
    int64_t N;
    int n_ios, n, shift;
};

template <bool MODE_E>
#ifndef VJP_MINB
#define VJP_MINB 1
#endif
__global__ void __launch_bounds__(256, VJP_MINB) vjp_gather_kernel(VjpParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const CicPoint C = cic_point(P.off0, P.off1, P.off2, i, P.cellid[i], P.n_ios, P.shift);
    float v[3] = {0.f, 0.f, 0.f};
    if (MODE_E) {   // the cotangent is read only in this mode (null otherwise)
        v[0] = P.v0[i];
        v[1] = P.v1[i];
        v[2] = P.v2[i];
    }
    const int n = P.n;
    float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                const int x = C.i0[0] + cx, y = C.i0[1] + cy, z = C.i0[2] + cz;
                const float wx = cx ? C.w1[0] : 1.0f - C.w1[0];
                const float wy = cy ? C.w1[1] : 1.0f - C.w1[1];
                const float wz = cz ? C.w1[2] : 1.0f - C.w1[2];
                const float sx = cx ? 1.0f : -1.0f, sy = cy ? 1.0f : -1.0f, sz = cz ? 1.0f : -1.0f;
                float val;
                if (MODE_E) {
                    const float *f = P.grid;
                    const float ex = (2.0f / 3.0f) * (at(f, n, x + 1, y, z) - at(f, n, x - 1, y, z)) -
                                     (1.0f / 12.0f) * (at(f, n, x + 2, y, z) - at(f, n, x - 2, y, z));
                    const float ey = (2.0f / 3.0f) * (at(f, n, x, y + 1, z) - at(f, n, x, y - 1, z)) -
                                     (1.0f / 12.0f) * (at(f, n, x, y + 2, z) - at(f, n, x, y - 2, z));
                    const float ez = (2.0f / 3.0f) * (at(f, n, x, y, z + 1) - at(f, n, x, y, z - 1)) -
                                     (1.0f / 12.0f) * (at(f, n, x, y, z + 2) - at(f, n, x, y, z - 2));
                    val = -(ex * v[0] + ey * v[1] + ez * v[2]);
                } else {
                    val = at(P.grid, n, x, y, z);
                }
                g[0] += sx * wy * wz * val;
                g[1] += wx * sy * wz * val;
                g[2] += wx * wy * sz * val;
            }
    P.w0[i] += P.scale * g[0];
    P.w1[i] += P.scale * g[1];
    P.w2[i] += P.scale * g[2];
}

__global__ void __launch_bounds__(256) mu_deposit_kernel(VjpParams P, float *mu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const CicPoint C = cic_point(P.off0, P.off1, P.off2, i, P.cellid[i], P.n_ios, P.shift);
    const float v[3] = {P.v0[i], P.v1[i], P.v2[i]};
    const int n = P.n;
    const int64_t n3 = (int64_t)n * n * n;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                const float W = (cx ? C.w1[0] : 1.0f - C.w1[0]) * (cy ? C.w1[1] : 1.0f - C.w1[1]) *
                                (cz ? C.w1[2] : 1.0f - C.w1[2]);
                const int64_t c = ((int64_t)wrapn(C.i0[2] + cz, n) * n + wrapn(C.i0[1] + cy, n)) * n +
                                  wrapn(C.i0[0] + cx, n);
                atomicAdd(&mu[c], W * v[0]);
                atomicAdd(&mu[n3 + c], W * v[1]);
                atomicAdd(&mu[2 * n3 + c], W * v[2]);
            }
}

__global__ void __launch_bounds__(256) div_stencil_kernel(const float *mu, float *s, int n, float scale) {
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n3) return;
    const int x = (int)(c % n), y = (int)((c / n) % n), z = (int)(c / ((int64_t)n * n));
    const float *mx = mu, *my = mu + n3, *mz = mu + 2 * n3;
    const float dx = (2.0f / 3.0f) * (at(mx, n, x + 1, y, z) - at(mx, n, x - 1, y, z)) -
                     (1.0f / 12.0f) * (at(mx, n, x + 2, y, z) - at(mx, n, x - 2, y, z));
    const float dy = (2.0f / 3.0f) * (at(my, n, x, y + 1, z) - at(my, n, x, y - 1, z)) -
                     (1.0f / 12.0f) * (at(my, n, x, y + 2, z) - at(my, n, x, y - 2, z));
    const float dz = (2.0f / 3.0f) * (at(mz, n, x, y, z + 1) - at(mz, n, x, y, z - 1)) -
                     (1.0f / 12.0f) * (at(mz, n, x, y, z + 2) - at(mz, n, x, y, z - 2));
    s[c] = scale * (dx + dy + dz);
}

VjpParams make_params(cube2_ctx *ctx, const Level &L, const cube2_particles *p, const float *const v[3],
                      float *const w[3], const float *grid) {
    VjpParams P{};
    P.off0 = p->off[0]; P.off1 = p->off[1]; P.off2 = p->off[2];
    P.cellid = ctx->cellid;
    P.v0 = v[0]; P.v1 = v[1]; P.v2 = v[2];
    P.w0 = w[0]; P.w1 = w[1]; P.w2 = w[2];
    P.grid = grid;
    P.scale = 1.0f;
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.n = L.n;
    P.shift = L.shift;
    return P;
}

// g(c) = 2 (delta(c) - target(c)) / n^3 in place of delta; sum of squares into *sq.
__global__ void __launch_bounds__(256) mse_residual_kernel(float *grid, const float *target, int64_t n3, double *sq) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double r2 = 0.0;
    if (c < n3) {
        const float r = grid[c] - target[c];
        r2 = (double)r * (double)r;
        grid[c] = r * (float)(2.0 / (double)n3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    if ((threadIdx.x & 31) == 0 && r2 != 0.0) atomicAdd(sq, r2);
}

// Reverse of one KDK step, part 1 (post-step order n -> pre-step order perm[n]):
// xs[perm[n]] = xbar[n] + k2 t[n],  ps[perm[n]] = pbar[n].
__global__ void __launch_bounds__(256) kdk_adjoint_scatter_kernel(const int32_t *perm, const float *xbar,
                                                                  const float *pbar, const float *t, float *xs,
                                                                  float *ps, int64_t N, float k2) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int64_t o = perm[n];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        xs[d * N + o] = xbar[d * N + n] + k2 * t[d * N + n];
        ps[d * N + o] = pbar[d * N + n];
    }
}

// Part 2 (pre-step order): xbar = xs, pbar = ps + drift * xs; part 3: xbar += k1 t.
struct Ptr3 {
    float *p[3];
};

__global__ void __launch_bounds__(256) kdk_adjoint_drift3_kernel(const float *xs, const float *ps, Ptr3 xbar, Ptr3 pbar,
                                                                 int64_t N, float drift) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float x = xs[d * N + i];
        xbar.p[d][i] = x;
        pbar.p[d][i] = ps[d * N + i] + drift * x;
    }
}

__global__ void __launch_bounds__(256) axpy3p_kernel(Ptr3 y, const float *t, int64_t N, float a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) y.p[d][i] += a * t[d * N + i];
}

}  // namespace

// w = (n^3 / (N H)) sum_c grad_u W(u_i, c) g(c) with g = 2 (delta - target)/n^3
// (the density's own grid must hold delta); adds sum (delta - target)^2 to *sq.
cudaError_t launch_density_mse_vjp(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *target,
                                   float *const w[3], double *sq) {
    const int64_t n3 = (int64_t)L.n * L.n * L.n;
    mse_residual_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, ctx->stream>>>(L.real, target, n3, sq);
    ctx->launches++;
    if (ctx->N == 0) return cudaGetLastError();
    const float *const nv[3] = {nullptr, nullptr, nullptr};
    VjpParams P = make_params(ctx, L, p, nv, w, L.real);
    P.v0 = P.v1 = P.v2 = nullptr;
    P.scale = (float)((double)n3 / ((double)ctx->N * L.H));
    vjp_gather_kernel<false><<<(unsigned)((ctx->N + 255) / 256), 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_density_vjp(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *g,
                               float *const w[3]) {
    const int64_t n3 = (int64_t)L.n * L.n * L.n;
    cudaError_t e = cudaMemcpyAsync(L.real, g, sizeof(float) * n3, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess || ctx->N == 0) return e;
    const float *const nv[3] = {nullptr, nullptr, nullptr};
    VjpParams P = make_params(ctx, L, p, nv, w, L.real);
    P.scale = (float)((double)n3 / ((double)ctx->N * L.H));
    vjp_gather_kernel<false><<<(unsigned)((ctx->N + 255) / 256), 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_kdk_adjoint_scatter(cube2_ctx *ctx, const int32_t *perm, float *const xbar[3],
                                       float *const pbar[3], const float *t, float k2) {
    // xbar/pbar are three separate arrays: gather them through the scratch rows
    const int64_t N = ctx->N;
    if (N == 0) return cudaSuccess;
    ProfScope prof(ctx, P_ADJ_KDK, 0);
    float *xs = ctx->vjp_u, *ps = ctx->vjp_u + 3 * N, *xc = ctx->vjp_u + 6 * N;
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
        e = cudaMemcpyAsync(xc + d * N, xbar[d], sizeof(float) * N, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(xc + (3 + d) * N, pbar[d], sizeof(float) * N, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    if (e != cudaSuccess) return e;
    kdk_adjoint_scatter_kernel<<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(perm, xc, xc + 3 * N, t, xs, ps,
                                                                                   N, k2);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_kdk_adjoint_drift(cube2_ctx *ctx, float *const xbar[3], float *const pbar[3], float drift) {
    const int64_t N = ctx->N;
    if (N == 0) return cudaSuccess;
    ProfScope prof(ctx, P_ADJ_KDK, 0);
    Ptr3 X{{xbar[0], xbar[1], xbar[2]}}, Pb{{pbar[0], pbar[1], pbar[2]}};
    kdk_adjoint_drift3_kernel<<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(ctx->vjp_u, ctx->vjp_u + 3 * N, X,
                                                                                   Pb, N, drift);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_axpy3(cube2_ctx *ctx, float *const y[3], const float *t, float a) {
    const int64_t N = ctx->N;
    if (N == 0) return cudaSuccess;
    Ptr3 Y{{y[0], y[1], y[2]}};
    axpy3p_kernel<<<(unsigned)((N + 255) / 256), 256, 0, ctx->stream>>>(Y, t, N, a);
    ctx->launches++;
    return cudaGetLastError();
}

// w += -sum_c grad W (E . v), E from the level's potential (in L.real).
cudaError_t launch_vjp_gather_e(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *const v[3],
                                float *const w[3]) {
    if (ctx->N == 0) return cudaSuccess;
    ProfScope prof(ctx, P_VJP_GATHER, L.index);
    VjpParams P = make_params(ctx, L, p, v, w, L.real);
    vjp_gather_kernel<true><<<(unsigned)((ctx->N + 255) / 256), 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

// w += sum_c grad W psi, psi in L.real.
cudaError_t launch_vjp_gather_psi(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *const v[3],
                                  float *const w[3]) {
    if (ctx->N == 0) return cudaSuccess;
    ProfScope prof(ctx, P_VJP_GATHER, L.index);
    VjpParams P = make_params(ctx, L, p, v, w, L.real);
    vjp_gather_kernel<false><<<(unsigned)((ctx->N + 255) / 256), 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

// L.real = (n^3/N) sum_d D_d * mu_d with mu_d the CIC deposit of v_d.
cudaError_t launch_vjp_source(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *const v[3]) {
    const int64_t n3 = (int64_t)L.n * L.n * L.n;
    ProfScope prof(ctx, P_VJP_SOURCE, L.index);
    cudaError_t e = cudaMemsetAsync(ctx->vjp_mu, 0, sizeof(float) * 3 * n3, ctx->stream);
    if (e != cudaSuccess) return e;
    if (ctx->N > 0) {
        float *const nw[3] = {nullptr, nullptr, nullptr};
        VjpParams P = make_params(ctx, L, p, v, nw, nullptr);
        mu_deposit_kernel<<<(unsigned)((ctx->N + 255) / 256), 256, 0, ctx->stream>>>(P, ctx->vjp_mu);
        ctx->launches++;
    }
    const float scale = (float)((double)n3 / (double)(ctx->N > 0 ? ctx->N : 1));
    div_stencil_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, ctx->stream>>>(ctx->vjp_mu, L.real, L.n, scale);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace cube2
