// Force interpolation F = -H_l sum_corners W E_l with E_l = D * phi_l (paper Sec. 2.1.2:
// Eq. diff for D, the deposit's CIC weights for W, so that momentum is conserved).
//
// One CTA per brick of BI^3 IOS cells, every level in one pass.  For each level
// the CTA stages in shared memory the phi tile its particles can reach: the
// brick's mesh cells, one more for the upper CIC corner and two on each side
// for the 4-point difference; along x the tile starts one more cell down, at
// a multiple of 4, and is a multiple of 4 long, so that it is staged in
// 16-byte copies (4-byte copies where a level's sizes do not allow it).  The 4-point difference is not stored as a
// field: along axis d the CIC pair of corners (weights w0 on i0, w1 on i0+1)
// sees phi at i0-2 .. i0+3 with the combined coefficients
//   i0-2: +w0/12      i0-1: -2/3 w0 + w1/12   i0: -2/3 w1
//   i0+1: +2/3 w0     i0+2: -w0/12 + 2/3 w1   i0+3: -w1/12
// applied on the 2x2 lines of the two other axes: 24 reads per component, 56
// distinct phi values per level, all from shared memory.  The brick's
// particles are the x-rows of its cells, contiguous in IOS order.
#include "common.cuh"

namespace cube2 {
namespace {

struct InterpLevel {
    const float *phi;
    int n, shift;
    float scale;          // -H_l
    int tile_off, D;      // tile offset in shared memory, tile edge
};

struct InterpParams {
    const uint16_t *off0, *off1, *off2;
    const int32_t *cellid, *count, *start;
    float *acc0, *acc1, *acc2;
    int64_t N;
    int n_ios, nl, accumulate, bi, nbx;
    InterpLevel lev[CUBE2_MAX_LEVELS];
};

constexpr int INTERP_THREADS = 256;
constexpr int INTERP_MAX_ROWS = DEPOSIT_BRICK * DEPOSIT_BRICK;

__device__ __forceinline__ void fd_coeffs(float w0, float w1, float c[6]) {
    const float a = 2.0f / 3.0f, b = 1.0f / 12.0f;
    c[0] = b * w0;
    c[1] = -a * w0 + b * w1;
    c[2] = -a * w1;
    c[3] = a * w0;
    c[4] = -b * w0 + a * w1;
    c[5] = -b * w1;
}

__device__ __forceinline__ int mod_n(int j, int n) {
    const int r = j % n;
    return r < 0 ? r + n : r;
}

// 7-point coefficients of the TSC-weighted 4-point difference along one axis
// (TSC weights w on cells i-1, i, i+1; coefficients on cells i-3 .. i+3).
__device__ __forceinline__ void fd7_coeffs(const float w[3], float c[7]) {
    const float a = 2.0f / 3.0f, b = 1.0f / 12.0f;
    c[0] = b * w[0];
    c[1] = -a * w[0] + b * w[1];
    c[2] = -a * w[1] + b * w[2];
    c[3] = a * (w[0] - w[2]);
    c[4] = -b * w[0] + a * w[1];
    c[5] = -b * w[1] + a * w[2];
    c[6] = -b * w[2];
}

// ORD 2: CIC; ORD 3: TSC (Eq. filter), whose 7-cell reach along each axis is
// the same tile as the CIC corner pair's 4-point difference.
template <int NL, int DA, int DB, int ORD>
__global__ void __launch_bounds__(INTERP_THREADS) interp_kernel(InterpParams P) {
    extern __shared__ __align__(16) float tiles[];
    __shared__ int row_pre[INTERP_MAX_ROWS + 1], row_start[INTERP_MAX_ROWS];
    const int n_ios = P.n_ios, bi = P.bi;
    const int brick = blockIdx.x;
    const int bx = brick % P.nbx, by = (brick / P.nbx) % P.nbx, bz = brick / (P.nbx * P.nbx);
    const int c0x = bx * bi, c0y = by * bi, c0z = bz * bi;
    const int ex = min(bi, n_ios - c0x), ey = min(bi, n_ios - c0y), ez = min(bi, n_ios - c0z);
    const int nrows = ey * ez;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        const int cy = c0y + r % ey, cz = c0z + r / ey;
        const int64_t rb = ((int64_t)cz * n_ios + cy) * n_ios;
        const int st = P.start[rb + c0x];
        row_start[r] = st;
        row_pre[r] = P.start[rb + c0x + ex - 1] + P.count[rb + c0x + ex - 1] - st;
    }
    // stage the phi tiles (origin three cells below the brick's mesh origin in
    // y and z, four in x): the wrapped per-axis indices of every level first,
    // then the copies
    static_assert(DA + 2 <= 32 && DB + 2 <= 32, "tile rows longer than the index table");
    __shared__ int widx[NL][3][32];
    for (int q = threadIdx.x; q < NL * 96; q += blockDim.x) {
        const int l = q / 96, a = (q / 32) % 3, k = q % 32;
        const int D = l == 0 ? DA : DB;
        if (k < (a == 0 ? D + 2 : D)) {
            const InterpLevel &L = P.lev[l];
            const int c0a = a == 0 ? c0x : (a == 1 ? c0y : c0z);
            widx[l][a][k] = mod_n((L.shift >= 0 ? (c0a >> L.shift) : (c0a << (-L.shift))) - (a == 0 ? 4 : 3) + k, L.n);
        }
    }
    __syncthreads();
    const int nwarps_s = blockDim.x >> 5, lane_s = threadIdx.x & 31, w_s = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const InterpLevel &L = P.lev[l];
        const int s = L.shift, n = L.n;
        const int D = l == 0 ? DA : DB, DX = D + 2;
        const int (*wi)[32] = widx[l];
        float *tile = tiles + L.tile_off;
        const int64_t nn = (int64_t)n * n;
        // 16-byte copies where the x origin, the row length and the mesh allow
        const int x0m = (s >= 0 ? (c0x >> s) : (c0x << (-s))) - 4;
        const bool vec = (x0m & 3) == 0 && (DX & 3) == 0 && (n & 3) == 0 && (L.tile_off & 3) == 0;
        if (vec) {
            // 16-byte chunks of all rows dealt to all threads: a warp copies
            // 32 chunks (about five rows) per instruction
            const int q = DX >> 2, chunks = D * D * q;
            for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
                const int row = c / q, x = (c - row * q) << 2;
                const int y = row % D, z = row / D;
                const float *src = L.phi + wi[2][z] * nn + (int64_t)wi[1][y] * n + wi[0][x];
                const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + row * DX + x);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
            }
        } else {
            for (int row = w_s; row < D * D; row += nwarps_s) {
                const int y = row % D, z = row / D;
                const float *src = L.phi + wi[2][z] * nn + (int64_t)wi[1][y] * n;
                for (int x = lane_s; x < DX; x += 32) {
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + row * DX + x);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src + wi[0][x])
                                 : "memory");
                }
            }
        }
    }
    // the row scan (row sizes written before the barrier above) while the
    // copies are in flight; one barrier then covers both
    if (threadIdx.x < 32) {            // exclusive scan of the row sizes
        const int lane = threadIdx.x;
        const int per = (nrows + 31) / 32;
        const int b0 = min(nrows, lane * per), b1 = min(nrows, b0 + per);
        int acc = 0;
        for (int i = b0; i < b1; ++i) acc += row_pre[i];
        int incl = acc;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - acc;
        for (int i = b0; i < b1; ++i) { const int v = row_pre[i]; row_pre[i] = run; run += v; }
        if (lane == 31) row_pre[nrows] = incl;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    const int total = row_pre[nrows];
    const int nwarps = blockDim.x >> 5, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per_w = ((total + nwarps - 1) / nwarps + 31) & ~31;
    const int it0 = w * per_w, it1 = min(total, it0 + per_w);
    int r = 0;
    if (it0 < it1) {
        int lo = 0, hi = nrows - 1;
        const int first = it0 + lane;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_pre[mid] <= first) lo = mid; else hi = mid - 1;
        }
        r = lo;
    }
    for (int t = it0 + lane; t < it1; t += 32) {
        while (row_pre[r + 1] <= t) ++r;
        const int64_t i = (int64_t)row_start[r] + (t - row_pre[r]);
        const int cx = P.cellid[i] % n_ios, cy = c0y + r % ey, cz = c0z + r / ey;
        const int X[3] = {cx * FIX + (int)P.off0[i], cy * FIX + (int)P.off1[i], cz * FIX + (int)P.off2[i]};
        const int c0[3] = {c0x, c0y, c0z};
        float F[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const InterpLevel &L = P.lev[l];
            const int s = L.shift;
            const int D = l == 0 ? DA : DB, DX = D + 2;
            if constexpr (ORD == 3) {
                // TSC: cell i holding the position, weights on i-1, i, i+1
                int ti[3];
                float tw[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int xm = s >= 0 ? (X[a] >> s) : (X[a] * (1 << (-s)));
                    const int org = (s >= 0 ? (c0[a] >> s) : (c0[a] << (-s))) - (a == 0 ? 4 : 3);
                    ti[a] = (xm >> FIX_BITS) - org;        // in the tile, >= 3
                    const float d = (float)(xm & (FIX - 1)) * (1.0f / FIX) - 0.5f;
                    tw[a][0] = 0.5f * (0.5f - d) * (0.5f - d);
                    tw[a][1] = 0.75f - d * d;
                    tw[a][2] = 0.5f * (0.5f + d) * (0.5f + d);
                }
                float c7x[7], c7y[7], c7z[7];
                fd7_coeffs(tw[0], c7x);
                fd7_coeffs(tw[1], c7y);
                fd7_coeffs(tw[2], c7z);
                const float *tile = tiles + L.tile_off;
                const int DD = D * DX;
                float ex_ = 0.f, ey_ = 0.f, ez_ = 0.f;
#pragma unroll
                for (int j1 = 0; j1 < 3; ++j1)
#pragma unroll
                    for (int j2 = 0; j2 < 3; ++j2) {
                        const float *rx = tile + (ti[2] + j2 - 1) * DD + (ti[1] + j1 - 1) * DX + ti[0] - 3;
                        const float *ry = tile + (ti[2] + j2 - 1) * DD + (ti[1] - 3) * DX + ti[0] + j1 - 1;
                        const float *rz = tile + (ti[2] - 3) * DD + (ti[1] + j2 - 1) * DX + ti[0] + j1 - 1;
                        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
                        for (int m = 0; m < 7; ++m) {
                            sx += c7x[m] * rx[m];
                            sy += c7y[m] * ry[m * DX];
                            sz += c7z[m] * rz[m * DD];
                        }
                        ex_ += tw[1][j1] * tw[2][j2] * sx;
                        ey_ += tw[0][j1] * tw[2][j2] * sy;
                        ez_ += tw[0][j1] * tw[1][j2] * sz;
                    }
                F[0] += L.scale * ex_;
                F[1] += L.scale * ey_;
                F[2] += L.scale * ez_;
                continue;
            }
            int li[3];
            float w0[3], w1[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int xm = s >= 0 ? (X[a] >> s) : (X[a] * (1 << (-s)));
                const int tt = xm - (FIX >> 1);
                const int org = (s >= 0 ? (c0[a] >> s) : (c0[a] << (-s))) - (a == 0 ? 4 : 3);
                li[a] = (tt >> FIX_BITS) - org;            // lower corner in the tile, >= 2
                const int f = tt & (FIX - 1);
                w1[a] = (float)f * (1.0f / FIX);
                w0[a] = (float)(FIX - f) * (1.0f / FIX);
            }
            const float *tile = tiles + L.tile_off;
            const int DD = D * DX;   // plane; rows are DX long
            float cx6[6], cy6[6], cz6[6];
            fd_coeffs(w0[0], w1[0], cx6);
            fd_coeffs(w0[1], w1[1], cy6);
            fd_coeffs(w0[2], w1[2], cz6);
            float ex_ = 0.f, ey_ = 0.f, ez_ = 0.f;
#pragma unroll
            for (int bz2 = 0; bz2 < 2; ++bz2) {
                const float wz = bz2 ? w1[2] : w0[2];
#pragma unroll
                for (int by2 = 0; by2 < 2; ++by2) {
                    const float wy = by2 ? w1[1] : w0[1];
                    const float *row = tile + (li[2] + bz2) * DD + (li[1] + by2) * DX + li[0] - 2;
                    float sx = 0.f;
#pragma unroll
                    for (int m = 0; m < 6; ++m) sx += cx6[m] * row[m];
                    ex_ += wy * wz * sx;
                }
            }
#pragma unroll
            for (int bz2 = 0; bz2 < 2; ++bz2) {
                const float wz = bz2 ? w1[2] : w0[2];
#pragma unroll
                for (int bx2 = 0; bx2 < 2; ++bx2) {
                    const float wx = bx2 ? w1[0] : w0[0];
                    const float *col = tile + (li[2] + bz2) * DD + (li[1] - 2) * DX + li[0] + bx2;
                    float sy = 0.f;
#pragma unroll
                    for (int m = 0; m < 6; ++m) sy += cy6[m] * col[m * DX];
                    ey_ += wx * wz * sy;
                }
            }
#pragma unroll
            for (int by2 = 0; by2 < 2; ++by2) {
                const float wy = by2 ? w1[1] : w0[1];
#pragma unroll
                for (int bx2 = 0; bx2 < 2; ++bx2) {
                    const float wx = bx2 ? w1[0] : w0[0];
                    const float *col = tile + (li[2] - 2) * DD + (li[1] + by2) * DX + li[0] + bx2;
                    float sz = 0.f;
#pragma unroll
                    for (int m = 0; m < 6; ++m) sz += cz6[m] * col[m * DD];
                    ez_ += wx * wy * sz;
                }
            }
            F[0] += L.scale * ex_;
            F[1] += L.scale * ey_;
            F[2] += L.scale * ez_;
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
    const int ord = ctx->cfg.assign_order == 3 ? 3 : 2;
    InterpParams P{};
    P.off0 = p->off[0]; P.off1 = p->off[1]; P.off2 = p->off[2];
    P.cellid = ctx->cellid;
    P.count = p->count; P.start = p->start;
    P.acc0 = p->acc[0]; P.acc1 = p->acc[1]; P.acc2 = p->acc[2];
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.accumulate = accumulate;
    const int lo = level < 0 ? 0 : level, hi = level < 0 ? ctx->nl : level + 1;
    int min_shift = 1;
    for (int l = lo; l < hi; ++l) min_shift = min(min_shift, ctx->lev[l].shift);
    P.bi = min_shift <= -2 ? DEPOSIT_BRICK / 2 : DEPOSIT_BRICK;
    P.nbx = (ctx->n_ios + P.bi - 1) / P.bi;
    P.nl = hi - lo;
    int off = 0;
    for (int l = lo; l < hi; ++l) {
        const Level &L = ctx->lev[l];
        InterpLevel &I = P.lev[l - lo];
        I.phi = L.real;
        I.n = L.n;
        I.shift = L.shift;
        I.scale = (float)(-L.H);
        const int E = L.shift >= 0 ? (P.bi >> L.shift) : (P.bi << (-L.shift));
        I.D = E + 6;
        I.tile_off = off;
        off += I.D * I.D * (I.D + 2);   // x rows are D + 2 long
    }
    if (ctx->N == 0) return cudaSuccess;
    const size_t smem = (size_t)off * sizeof(float);
    const int64_t blocks = (int64_t)P.nbx * P.nbx * P.nbx;
    ProfScope prof(ctx, P_INTERP, 0);
    const int d0 = P.lev[0].D, d1 = P.nl > 1 ? P.lev[1].D : d0;
    cudaError_t e = cudaErrorInvalidValue;
    // tile edges are 8, 10, 14 or 22 (brick 8 or 4, shifts -2..1); the coarse level has the smaller edge
#define CUBE2_INTERP_CASE_O(NL_, A_, B_, O_)                                                        \
    if (P.nl == NL_ && d0 == A_ && d1 == B_ && ord == O_) {                                         \
        static bool attr = false;                                                                   \
        if (!attr) {                                                                                \
            cudaFuncSetAttribute(interp_kernel<NL_, A_, B_, O_>,                                     \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);           \
            attr = true;                                                                            \
        }                                                                                           \
        interp_kernel<NL_, A_, B_, O_><<<(unsigned)blocks, INTERP_THREADS, smem, ctx->stream>>>(P); \
        e = cudaGetLastError();                                                                     \
    }
#define CUBE2_INTERP_CASE(NL_, A_, B_) CUBE2_INTERP_CASE_O(NL_, A_, B_, 2) CUBE2_INTERP_CASE_O(NL_, A_, B_, 3)
    CUBE2_INTERP_CASE(1, 8, 8)
    CUBE2_INTERP_CASE(1, 10, 10)
    CUBE2_INTERP_CASE(1, 14, 14)
    CUBE2_INTERP_CASE(1, 22, 22)
    CUBE2_INTERP_CASE(2, 8, 10)
    CUBE2_INTERP_CASE(2, 8, 14)
    CUBE2_INTERP_CASE(2, 8, 22)
    CUBE2_INTERP_CASE(2, 10, 14)
    CUBE2_INTERP_CASE(2, 10, 22)
    CUBE2_INTERP_CASE(2, 14, 22)
#undef CUBE2_INTERP_CASE
#undef CUBE2_INTERP_CASE_O
    ctx->launches++;
    return e;
}

}  // namespace cube2
