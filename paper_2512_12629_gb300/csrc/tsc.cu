// TSC mass assignment and force interpolation: the paper's own assignment
// window (Eq. filter, W(k) = prod_d sinc^3(k_d/2)), selected by
// cube2_config.assign_order = 3 in place of the workload's exact-integer CIC.
//
// Per axis, with the position in mesh cells u (the IOS fixed point in mesh
// units, floored to 2^-16 mesh cell as for CIC), i = floor(u) and
// d = u - (i + 1/2): weights (1/2 - d)^2/2, 3/4 - d^2, (1/2 + d)^2/2 on cells
// i - 1, i, i + 1.  A 3-D TSC weight would need 99 bits as an exact integer,
// so the deposit accumulates FP32 with global atomics onto a grid filled
// with -1 (the overdensity of an empty cell): sums are correct to FP32
// rounding, their last bits depend on the atomic order.
//
// Interpolation is the tiled gather of interp.cu (ORD = 3): it evaluates the
// 4-point difference of Eq. diff on the fly like the CIC gather; along axis d
// the three weights and the stencil combine into 7 coefficients on cells
// i-3 .. i+3,
//   c_m = sum_j w_j f_(m-j),  f = (1/12, -2/3, 0, 2/3, -1/12) on offsets -2..2,
// applied on the 3x3 lines of the two other axes (63 potential reads per
// component, from the shared-memory tile).
#include "common.cuh"

namespace cube2 {
namespace {

struct TscAxis {
    int i;        // cell holding the position
    float w[3];   // weights of cells i-1, i, i+1
};

__device__ __forceinline__ TscAxis tsc_axis(int X, int shift) {
    const int xm = shift >= 0 ? (X >> shift) : (X << (-shift));
    TscAxis a;
    a.i = xm >> FIX_BITS;
    const float d = (float)(xm & (FIX - 1)) * (1.0f / FIX) - 0.5f;
    a.w[0] = 0.5f * (0.5f - d) * (0.5f - d);
    a.w[1] = 0.75f - d * d;
    a.w[2] = 0.5f * (0.5f + d) * (0.5f + d);
    return a;
}

__device__ __forceinline__ int wrapc(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

struct TscParams {
    const uint16_t *off0, *off1, *off2;
    const int32_t *cellid;
    int64_t N;
    int n_ios, n, shift;
    float scale;         // n^3 / N (deposit)
    float *grid;         // density (deposit)
};

__device__ __forceinline__ void particle_axes(const TscParams &P, int64_t i, TscAxis a[3]) {
    const int cell = P.cellid[i], n = P.n_ios;
    const int c[3] = {cell % n, (cell / n) % n, cell / (n * n)};
    const int o[3] = {(int)P.off0[i], (int)P.off1[i], (int)P.off2[i]};
#pragma unroll
    for (int d = 0; d < 3; ++d) a[d] = tsc_axis(c[d] * FIX + o[d], P.shift);
}

__global__ void __launch_bounds__(256) fill_kernel(float *g, int64_t n, float v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g[i] = v;
}

// Particles are in IOS order, so on a coarse level the lanes of a warp come in
// runs that share the cell holding them, and with it all 27 target cells.  A
// warp with runs (at most 16 distinct cells) sums each target's weights over
// every run with a segmented shuffle scan and lets the run's last lane add the
// total; other warps add per lane.
__global__ void __launch_bounds__(256) tsc_deposit_kernel(TscParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = i < P.N;
    const int lane = threadIdx.x & 31;
    TscAxis a[3];
    if (has) {
        particle_axes(P, i, a);
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) a[d] = TscAxis{0, {0.f, 0.f, 0.f}};
    }
    const int n = P.n;
    const long long key = has ? ((long long)a[2].i * n + a[1].i) * n + a[0].i : -1ll;
    const long long prev = __shfl_up_sync(0xffffffffu, key, 1), next = __shfl_down_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || prev != key;
    const bool tail = lane == 31 || next != key;
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const bool agg = __popc(heads) <= 16;
    const int s0 = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));   // first lane of this lane's run
#pragma unroll
    for (int jz = 0; jz < 3; ++jz) {
        const int64_t z = wrapc(a[2].i + jz - 1, n);
        const float wz = P.scale * a[2].w[jz];
#pragma unroll
        for (int jy = 0; jy < 3; ++jy) {
            const int64_t row = (z * n + wrapc(a[1].i + jy - 1, n)) * n;
            const float wyz = wz * a[1].w[jy];
#pragma unroll
            for (int jx = 0; jx < 3; ++jx) {
                float v = wyz * a[0].w[jx];
                if (agg) {
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const float u = __shfl_up_sync(0xffffffffu, v, d);
                        if (lane - d >= s0) v += u;
                    }
                    if (has && tail) atomicAdd(&P.grid[row + wrapc(a[0].i + jx - 1, n)], v);
                } else if (has) {
                    atomicAdd(&P.grid[row + wrapc(a[0].i + jx - 1, n)], v);
                }
            }
        }
    }
}

TscParams tsc_params(cube2_ctx *ctx, const Level &L, const cube2_particles *p) {
    TscParams P{};
    P.off0 = p->off[0]; P.off1 = p->off[1]; P.off2 = p->off[2];
    P.cellid = ctx->cellid;
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.n = L.n;
    P.shift = L.shift;
    P.scale = (float)((double)L.n * L.n * L.n / (double)(ctx->N > 0 ? ctx->N : 1));
    P.grid = L.real;
    return P;
}

}  // namespace

// L.real = TSC overdensity of the particles (cell ids must be current).
cudaError_t launch_tsc_deposit(cube2_ctx *ctx, Level &L, const cube2_particles *p) {
    ProfScope prof(ctx, P_DEPOSIT, L.index);
    const int64_t n3 = (int64_t)L.n * L.n * L.n;
    fill_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, ctx->stream>>>(L.real, n3, -1.0f);
    ctx->launches++;
    if (ctx->N > 0) {
        tsc_deposit_kernel<<<(unsigned)((ctx->N + 255) / 256), 256, 0, ctx->stream>>>(tsc_params(ctx, L, p));
        ctx->launches++;
    }
    return cudaGetLastError();
}

}  // namespace cube2
