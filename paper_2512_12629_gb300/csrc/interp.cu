// Force interpolation F = -H_l sum_corners W E_l with E_l = D * phi_l (paper Sec. 2.1.2:
// Eq. diff for D, the deposit's CIC weights for W, so that momentum is conserved).
//
// One thread per particle, every level in one pass.  The 4-point difference is
// not stored as a field: along axis d the CIC pair of corners (weights w0 on
// i0, w1 on i0+1) sees phi at i0-2 .. i0+3 with the combined coefficients
//   i0-2: +w0/12      i0-1: -2/3 w0 + w1/12   i0: -2/3 w1
//   i0+1: +2/3 w0     i0+2: -w0/12 + 2/3 w1   i0+3: -w1/12
// applied on the 2x2 lines of the two other axes: 24 loads per component,
// 56 distinct phi values per level.  Particles are stored cell-sorted, so a warp
// reads a compact neighbourhood and phi comes from L1/L2 after the first touch.
#include "common.cuh"

namespace cube2 {
namespace {

struct InterpLevel {
    const float *phi;
    int n, shift;
    float scale;          // -H_l
};

struct InterpParams {
    const uint16_t *off0, *off1, *off2;
    const int32_t *cellid;
    float *acc0, *acc1, *acc2;
    int64_t N;
    int n_ios, nl, accumulate;
    InterpLevel lev[CUBE2_MAX_LEVELS];
};

__device__ __forceinline__ void fd_coeffs(float w0, float w1, float c[6]) {
    const float a = 2.0f / 3.0f, b = 1.0f / 12.0f;
    c[0] = b * w0;
    c[1] = -a * w0 + b * w1;
    c[2] = -a * w1;
    c[3] = a * w0;
    c[4] = -b * w0 + a * w1;
    c[5] = -b * w1;
}

__global__ void __launch_bounds__(256) interp_kernel(InterpParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int c = P.cellid[i];
    const int n_ios = P.n_ios;
    const int cx = c % n_ios, cy = (c / n_ios) % n_ios, cz = c / (n_ios * n_ios);
    const int X[3] = {cx * FIX + (int)P.off0[i], cy * FIX + (int)P.off1[i], cz * FIX + (int)P.off2[i]};
    float F[3] = {0.f, 0.f, 0.f};
    for (int l = 0; l < P.nl; ++l) {
        const InterpLevel &L = P.lev[l];
        const int n = L.n, s = L.shift;
        int i0[3];
        float w0[3], w1[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int xm = s >= 0 ? (X[a] >> s) : (X[a] * (1 << (-s)));
            const int t = xm - (FIX >> 1);
            i0[a] = t >> FIX_BITS;
            const int f = t & (FIX - 1);
            w1[a] = (float)f * (1.0f / FIX);
            w0[a] = (float)(FIX - f) * (1.0f / FIX);
        }
        // wrapped indices i0-2 .. i0+3 per axis
        int ix[6], iy[6], iz[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            ix[m] = wrap(i0[0] - 2 + m, n);
            iy[m] = wrap(i0[1] - 2 + m, n);
            iz[m] = wrap(i0[2] - 2 + m, n);
        }
        const float *phi = L.phi;
        const int64_t nn = (int64_t)n * n;
        float cx6[6], cy6[6], cz6[6];
        fd_coeffs(w0[0], w1[0], cx6);
        fd_coeffs(w0[1], w1[1], cy6);
        fd_coeffs(w0[2], w1[2], cz6);
        float ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
        for (int bz = 0; bz < 2; ++bz) {
            const float wz = bz ? w1[2] : w0[2];
#pragma unroll
            for (int by = 0; by < 2; ++by) {
                const float wy = by ? w1[1] : w0[1];
                // x component: line along x at (iy[2+by], iz[2+bz])
                const float *row = phi + (int64_t)iz[2 + bz] * nn + (int64_t)iy[2 + by] * n;
                float sx = 0.f;
#pragma unroll
                for (int m = 0; m < 6; ++m) sx += cx6[m] * __ldg(&row[ix[m]]);
                ex += wy * wz * sx;
            }
        }
#pragma unroll
        for (int bz = 0; bz < 2; ++bz) {
            const float wz = bz ? w1[2] : w0[2];
#pragma unroll
            for (int bx = 0; bx < 2; ++bx) {
                const float wx = bx ? w1[0] : w0[0];
                const float *col = phi + (int64_t)iz[2 + bz] * nn + ix[2 + bx];
                float sy = 0.f;
#pragma unroll
                for (int m = 0; m < 6; ++m) sy += cy6[m] * __ldg(&col[(int64_t)iy[m] * n]);
                ey += wx * wz * sy;
            }
        }
#pragma unroll
        for (int by = 0; by < 2; ++by) {
            const float wy = by ? w1[1] : w0[1];
#pragma unroll
            for (int bx = 0; bx < 2; ++bx) {
                const float wx = bx ? w1[0] : w0[0];
                const float *col = phi + (int64_t)iy[2 + by] * n + ix[2 + bx];
                float sz = 0.f;
#pragma unroll
                for (int m = 0; m < 6; ++m) sz += cz6[m] * __ldg(&col[(int64_t)iz[m] * nn]);
                ez += wx * wy * sz;
            }
        }
        F[0] += L.scale * ex;
        F[1] += L.scale * ey;
        F[2] += L.scale * ez;
    }
    if (P.accumulate) {
        P.acc0[i] += F[0];
        P.acc1[i] += F[1];
        P.acc2[i] += F[2];
    } else {
        P.acc0[i] = F[0];
        P.acc1[i] = F[1];
        P.acc2[i] = F[2];
    }
}

__global__ void cellid_kernel(const int32_t *__restrict__ count, const int32_t *__restrict__ start,
                              int32_t *__restrict__ cellid, int64_t n_cells) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const int s = start[c], e = s + count[c];
    for (int p = s; p < e; ++p) cellid[p] = (int32_t)c;
}

}  // namespace

cudaError_t launch_cellid(cube2_ctx *ctx, const cube2_particles *p) {
    const int64_t blocks = (ctx->n_cells + 255) / 256;
    ProfScope prof(ctx, P_CELLID, 0);
    cellid_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(p->count, p->start, ctx->cellid, ctx->n_cells);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_interp(cube2_ctx *ctx, int level, const cube2_particles *p, int accumulate) {
    InterpParams P{};
    P.off0 = p->off[0]; P.off1 = p->off[1]; P.off2 = p->off[2];
    P.cellid = ctx->cellid;
    P.acc0 = p->acc[0]; P.acc1 = p->acc[1]; P.acc2 = p->acc[2];
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.accumulate = accumulate;
    const int lo = level < 0 ? 0 : level, hi = level < 0 ? ctx->nl : level + 1;
    P.nl = hi - lo;
    for (int l = lo; l < hi; ++l) {
        const Level &L = ctx->lev[l];
        P.lev[l - lo] = InterpLevel{L.real, L.n, L.shift, (float)(-L.H)};
    }
    const int64_t blocks = (ctx->N + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    ProfScope prof(ctx, P_INTERP, 0);
    interp_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace cube2
