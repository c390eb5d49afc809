// CIC mass assignment onto one or all PM levels (paper Sec. 2.1.2, Eq. filter with
// the CIC reading; IOS input of Sec. 2.3).
//
// Design: one CTA owns a brick of BI^3 IOS cells.  For every level it owns the
// mesh cells that cover the brick (BI * n/n_ios per axis) and holds their uint64
// accumulators in shared memory.  It walks the particles of the brick and of a
// one-cell IOS halo (every particle whose CIC cloud can reach an owned cell),
// adds the exact integer weights of the corners that fall inside its owned
// region with shared-memory atomics, then converts each owned cell once and
// writes it with plain coalesced stores.  No global atomics and no uint64 mesh
// in HBM: HBM traffic is the particle offsets (x ~1.95 for the halo) plus one
// FP32 write per mesh cell.
//
// Integer CIC: X = c 2^16 + off is the IOS fixed-point coordinate; the mesh
// coordinate floored to 2^-16 cell is X >> s (s >= 0) or X << -s.  With
// T = Xm - 2^15 the lower corner is T >> 16 and the 1-D weights are
// 2^16 - (T & 0xffff) and (T & 0xffff); the 3-D weight is their exact product.
// A uint64 wrap in any add is detected from the atomic's old value.
#include "common.cuh"

namespace cube2 {
namespace {

struct DepLevel {
    int n;            // mesh cells per axis
    int shift;        // n_ios / n = 2^shift, shift in {-2,-1,0,1}
    int own;          // owned mesh cells per axis for a full brick
    int tile_off;     // offset of this level's tile in the shared uint64 array
    float *out_f32;   // FP32 overdensity grid (or null)
    uint64_t *out_u64;  // raw accumulator (or null)
    uint64_t mean_int;
    float scale;
};

struct DepParams {
    const uint16_t *off0, *off1, *off2;
    const int32_t *count, *start;
    int n_ios, bi, nbx;   // IOS cells per axis, brick edge, bricks per axis
    int nl;
    DepLevel lev[CUBE2_MAX_LEVELS];
    int *status;
};

__device__ __forceinline__ float u64_delta_to_f32(uint64_t acc, uint64_t m, float scale) {
    // RN32(acc - M) exactly (the magnitude is formed in uint64), then one FP32 multiply
    const float mag = acc >= m ? __ull2float_rn(acc - m) : -__ull2float_rn(m - acc);
    return __fmul_rn(mag, scale);
}

__global__ void __launch_bounds__(256) deposit_kernel(DepParams P) {
    extern __shared__ unsigned long long smem_u64[];
    const int bi = P.bi;
    const int hb = bi + 2;                                   // halo brick edge (IOS cells)
    const int brick = blockIdx.x;
    const int bx = brick % P.nbx, by = (brick / P.nbx) % P.nbx, bz = brick / (P.nbx * P.nbx);
    const int c0x = bx * bi, c0y = by * bi, c0z = bz * bi;
    const int ex = min(bi, P.n_ios - c0x), ey = min(bi, P.n_ios - c0y), ez = min(bi, P.n_ios - c0z);

    // shared layout: [tiles (uint64)] [halo prefix (int32, hb^3 + 1)] [halo starts (int32, hb^3)]
    int tile_total = 0;
    for (int l = 0; l < P.nl; ++l) tile_total += P.lev[l].own * P.lev[l].own * P.lev[l].own;
    int *hpre = reinterpret_cast<int *>(smem_u64 + tile_total);
    int *hstart = hpre + hb * hb * hb + 1;
    const int nh = hb * hb * hb;

    for (int i = threadIdx.x; i < tile_total; i += blockDim.x) smem_u64[i] = 0ull;
    // halo cell counts (cells beyond a partial brick's extent + 1 are excluded)
    for (int h = threadIdx.x; h < nh; h += blockDim.x) {
        const int hx = h % hb, hy = (h / hb) % hb, hz = h / (hb * hb);
        int cnt = 0, st = 0;
        if (hx <= ex + 1 && hy <= ey + 1 && hz <= ez + 1) {
            const int cx = wrap(c0x - 1 + hx, P.n_ios), cy = wrap(c0y - 1 + hy, P.n_ios),
                      cz = wrap(c0z - 1 + hz, P.n_ios);
            const int64_t c = ((int64_t)cz * P.n_ios + cy) * P.n_ios + cx;
            cnt = P.count[c];
            st = P.start[c];
        }
        hpre[h] = cnt;
        hstart[h] = st;
    }
    __syncthreads();
    // exclusive scan of the halo counts (single warp; nh <= 1000 for bi = 8)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int per = (nh + 31) / 32;
        const int b0 = lane * per, b1 = min(nh, b0 + per);
        int s = 0;
        for (int i = b0; i < b1; ++i) s += hpre[i];
        int incl = s;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - s;
        for (int i = b0; i < b1; ++i) { const int v = hpre[i]; hpre[i] = run; run += v; }
        if (lane == 31) hpre[nh] = incl;
    }
    __syncthreads();
    const int total = hpre[nh];

    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        // halo cell holding item t: largest h with hpre[h] <= t
        int lo = 0, hi = nh - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (hpre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int h = lo;
        const int64_t p = (int64_t)hstart[h] + (t - hpre[h]);
        const int hx = h % hb, hy = (h / hb) % hb, hz = h / (hb * hb);
        // unwrapped fixed-point coordinates relative to the grid origin
        const int X0 = (c0x - 1 + hx) * FIX + (int)P.off0[p];
        const int X1 = (c0y - 1 + hy) * FIX + (int)P.off1[p];
        const int X2 = (c0z - 1 + hz) * FIX + (int)P.off2[p];
        for (int l = 0; l < P.nl; ++l) {
            const DepLevel &L = P.lev[l];
            const int s = L.shift;
            int i0[3], w0[3], w1[3], ext[3];
            const int X[3] = {X0, X1, X2};
            const int c0[3] = {c0x, c0y, c0z};
            const int e[3] = {ex, ey, ez};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int xm = s >= 0 ? (X[a] >> s) : (X[a] * (1 << (-s)));
                const int tt = xm - (FIX >> 1);
                const int org = s >= 0 ? (c0[a] >> s) : (c0[a] << (-s));
                i0[a] = (tt >> FIX_BITS) - org;             // lower corner, owned-local
                w1[a] = tt & (FIX - 1);
                w0[a] = FIX - w1[a];
                ext[a] = s >= 0 ? (e[a] >> s) : (e[a] << (-s));
            }
            unsigned long long *tile = smem_u64 + L.tile_off;
            const int own = L.own;
#pragma unroll
            for (int cz = 0; cz < 2; ++cz) {
                const int iz = i0[2] + cz;
                if (iz < 0 || iz >= ext[2]) continue;
                const unsigned long long wz = (unsigned long long)(cz ? w1[2] : w0[2]);
#pragma unroll
                for (int cy = 0; cy < 2; ++cy) {
                    const int iy = i0[1] + cy;
                    if (iy < 0 || iy >= ext[1]) continue;
                    const unsigned long long wyz = wz * (unsigned long long)(cy ? w1[1] : w0[1]);
#pragma unroll
                    for (int cx = 0; cx < 2; ++cx) {
                        const int ix = i0[0] + cx;
                        if (ix < 0 || ix >= ext[0]) continue;
                        const unsigned long long w = wyz * (unsigned long long)(cx ? w1[0] : w0[0]);
                        if (w == 0ull) continue;
                        const unsigned long long old = atomicAdd(&tile[(iz * own + iy) * own + ix], w);
                        if (old + w < old) set_status(P.status, ST_CAPACITY);
                    }
                }
            }
        }
    }
    __syncthreads();

    // epilogue: each owned cell converted and written once
    for (int l = 0; l < P.nl; ++l) {
        const DepLevel &L = P.lev[l];
        const int s = L.shift;
        const int own = L.own;
        const int ox = s >= 0 ? (c0x >> s) : (c0x << (-s));
        const int oy = s >= 0 ? (c0y >> s) : (c0y << (-s));
        const int oz = s >= 0 ? (c0z >> s) : (c0z << (-s));
        const int exl = s >= 0 ? (ex >> s) : (ex << (-s));
        const int eyl = s >= 0 ? (ey >> s) : (ey << (-s));
        const int ezl = s >= 0 ? (ez >> s) : (ez << (-s));
        const unsigned long long *tile = smem_u64 + L.tile_off;
        const int cells = exl * eyl * ezl;
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            const int ix = i % exl, iy = (i / exl) % eyl, iz = i / (exl * eyl);
            const uint64_t v = tile[(iz * own + iy) * own + ix];
            const int64_t g = ((int64_t)(oz + iz) * L.n + (oy + iy)) * L.n + (ox + ix);
            if (L.out_u64) L.out_u64[g] = v;
            if (L.out_f32) L.out_f32[g] = u64_delta_to_f32(v, L.mean_int, L.scale);
        }
    }
}

}  // namespace

// level >= 0: that level only; level = -1: every level in one particle pass.
// out_u64 (level >= 0 only): write the raw accumulator instead of the FP32 grid.
cudaError_t launch_deposit(cube2_ctx *ctx, int level, const cube2_particles *p, uint64_t *out_u64) {
    DepParams P{};
    P.off0 = p->off[0]; P.off1 = p->off[1]; P.off2 = p->off[2];
    P.count = p->count; P.start = p->start;
    P.n_ios = ctx->n_ios;
    P.status = ctx->dev_status;
    int lo = level < 0 ? 0 : level, hi = level < 0 ? ctx->nl : level + 1;
    int min_shift = 1;
    for (int l = lo; l < hi; ++l) min_shift = min(min_shift, ctx->lev[l].shift);
    P.bi = min_shift <= -2 ? DEPOSIT_BRICK / 2 : DEPOSIT_BRICK;
    P.nbx = (ctx->n_ios + P.bi - 1) / P.bi;
    int tile = 0;
    P.nl = hi - lo;
    for (int l = lo; l < hi; ++l) {
        const Level &L = ctx->lev[l];
        DepLevel &D = P.lev[l - lo];
        D.n = L.n;
        D.shift = L.shift;
        D.own = L.shift >= 0 ? (P.bi >> L.shift) : (P.bi << (-L.shift));
        D.tile_off = tile;
        tile += D.own * D.own * D.own;
        D.out_u64 = out_u64;
        D.out_f32 = out_u64 ? nullptr : L.real;
        D.mean_int = L.mean_int;
        D.scale = L.dens_scale;
    }
    const int hb = P.bi + 2;
    const size_t smem = (size_t)tile * 8 + (size_t)(2 * hb * hb * hb + 1) * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(deposit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int64_t blocks = (int64_t)P.nbx * P.nbx * P.nbx;
    ProfScope prof(ctx, P_DEPOSIT, 0);
    deposit_kernel<<<(unsigned)blocks, 256, smem, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace cube2
