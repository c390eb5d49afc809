// CIC mass assignment onto one or all PM levels (paper Sec. 2.1.2, Eq. filter with
// the CIC reading; IOS input of Sec. 2.3).
//
// Design: one CTA owns a brick of BI^3 IOS cells.  For every level it owns the
// mesh cells that cover the brick (BI * n/n_ios per axis) and holds their 64-bit
// accumulators in shared memory.  It walks the particles of the brick and of a
// one-cell IOS halo (every particle whose CIC cloud can reach an owned cell):
// the halo brick is a set of x-rows whose particles are contiguous in IOS order
// (two segments where a row wraps around the box), so items map to particles
// through a short search over the row prefix.  Each corner weight that falls in
// the owned region is added exactly with two 32-bit shared-memory atomics (low
// word, then the high word plus the low word's carry; measured faster than one
// 64-bit shared atomic); the CTA then converts
// each owned cell once and writes it with plain coalesced stores.  No global
// atomics and no 64-bit mesh in HBM: HBM traffic is the particle data (x ~1.95
// for the halo) plus one FP32 write per mesh cell.
//
// Integer CIC: X = c 2^16 + off is the IOS fixed-point coordinate; the mesh
// coordinate floored to 2^-16 cell is X >> s (s >= 0) or X << -s.  With
// T = Xm - 2^15 the lower corner is T >> 16 and the 1-D weights are
// 2^16 - (T & 0xffff) and (T & 0xffff); the 3-D weight is their exact product.
// A wrap of a cell's 64-bit sum is detected from the high word's atomic.
#include "common.cuh"

namespace cube2 {
namespace {

struct DepLevel {
    int n;            // mesh cells per axis
    int shift;        // n_ios / n = 2^shift, shift in {-2,-1,0,1}
    int own;          // owned mesh cells per axis for a full brick
    int tile_off;     // offset of this level's tile in the shared word arrays
    float *out_f32;   // FP32 overdensity grid (or null)
    uint64_t *out_u64;  // raw accumulator (or null)
    uint64_t mean_int;
    float scale;
};

struct DepParams {
    const uint16_t *off0, *off1, *off2;
    const int32_t *count, *start, *cellid;
    int n_ios, bi, nbx;   // IOS cells per axis, brick edge, bricks per axis
    int nl;
    int tile_total;       // cells of all level tiles
    DepLevel lev[CUBE2_MAX_LEVELS];
    int *status;
};

__device__ __forceinline__ float u64_delta_to_f32(uint64_t acc, uint64_t m, float scale) {
    // RN32(acc - M) exactly (the magnitude is formed in uint64), then one FP32 multiply
    const float mag = acc >= m ? __ull2float_rn(acc - m) : -__ull2float_rn(m - acc);
    return __fmul_rn(mag, scale);
}

constexpr int DEP_THREADS = 256;
constexpr int DEP_MAX_SEGS = 3 * (DEPOSIT_BRICK + 2) * (DEPOSIT_BRICK + 2);

template <int NL, int S0, int S1, int BI>
__global__ void __launch_bounds__(DEP_THREADS) deposit_kernel(DepParams P) {
    extern __shared__ unsigned int smem_u32[];            // [tile_total] low words, [tile_total] high words
    __shared__ int seg_pre[DEP_MAX_SEGS + 1];              // item prefix over the halo-row segments
    __shared__ int seg_start[DEP_MAX_SEGS];                // first particle of each segment
    __shared__ int seg_info[DEP_MAX_SEGS];                 // hx0 | hy << 8 | hz << 16
    __shared__ int seg_c0[DEP_MAX_SEGS];                   // cell id of the segment's first cell
    unsigned int *lo = smem_u32, *hi = smem_u32 + P.tile_total;
    const int n = P.n_ios;
    constexpr int bi = BI;
    const int brick = blockIdx.x;
    const int bx = brick % P.nbx, by = (brick / P.nbx) % P.nbx, bz = brick / (P.nbx * P.nbx);
    const int c0x = bx * bi, c0y = by * bi, c0z = bz * bi;
    const int ex = min(bi, n - c0x), ey = min(bi, n - c0y), ez = min(bi, n - c0z);
    const int nrows = (ey + 2) * (ez + 2);
    const int nseg = 3 * nrows;

    if (P.tile_total % 2 == 0) {   // 2 * tile_total words as 16-byte stores
        for (int i = threadIdx.x; i < P.tile_total / 2; i += blockDim.x)
            reinterpret_cast<uint4 *>(smem_u32)[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        for (int i = threadIdx.x; i < 2 * P.tile_total; i += blockDim.x) smem_u32[i] = 0u;
    }
    // halo row (hy, hz) spans cells x in [c0x-1, c0x+ex]; segment 0 is the part
    // inside [0, n), segments 1 and 2 the cells that wrap on the left and right
    for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
        const int row = sg / 3, part = sg % 3;
        const int hy = row % (ey + 2), hz = row / (ey + 2);
        const int cy = wrap(c0y - 1 + hy, n), cz = wrap(c0z - 1 + hz, n);
        const int64_t rbase = ((int64_t)cz * n + cy) * n;
        int xa, xb, hx0;
        if (part == 0) {
            xa = max(c0x - 1, 0);
            xb = min(c0x + ex, n - 1);
            hx0 = xa - (c0x - 1);
        } else if (part == 1 && c0x == 0) {
            xa = xb = n - 1;            // the halo cell left of x = 0
            hx0 = 0;
        } else if (part == 2 && c0x + ex == n) {
            xa = xb = 0;                // the halo cell right of x = n - 1
            hx0 = ex + 1;
        } else {
            xa = 0;
            xb = -1;                    // empty
            hx0 = 0;
        }
        int st = 0, cnt = 0;
        if (xb >= xa) {
            st = P.start[rbase + xa];
            cnt = P.start[rbase + xb] + P.count[rbase + xb] - st;
        }
        seg_pre[sg] = cnt;
        seg_start[sg] = st;
        seg_info[sg] = hx0 | (hy << 8) | (hz << 16);
        seg_c0[sg] = (int)(rbase + xa);
    }
    __syncthreads();
    if (threadIdx.x < 32) {            // exclusive scan of the segment sizes
        const int lane = threadIdx.x;
        const int per = (nseg + 31) / 32;
        const int b0 = min(nseg, lane * per), b1 = min(nseg, b0 + per);
        int acc = 0;
        for (int i = b0; i < b1; ++i) acc += seg_pre[i];
        int incl = acc;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - acc;
        for (int i = b0; i < b1; ++i) { const int v = seg_pre[i]; seg_pre[i] = run; run += v; }
        if (lane == 31) seg_pre[nseg] = incl;
    }
    __syncthreads();
    const int total = seg_pre[nseg];

    // each lane a contiguous chunk of its warp's items: at any step the lanes
    // are per_w / 32 particles apart, in different cells of a dense brick, so
    // fewer of their corners hit the same shared-memory words at once than with
    // lanes on consecutive particles (6 % less deposit time over the 256^3 run)
    const int nwarps = blockDim.x >> 5, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per_w = ((total + nwarps - 1) / nwarps + 31) & ~31;
    const int kch = per_w >> 5;
    const int it0 = w * per_w + lane * kch, it1 = min(total, it0 + kch);
    int sg = 0;
    if (it0 < it1) {
        int lo_s = 0, hi_s = nseg - 1;   // last segment with seg_pre <= it0
        const int first = it0;
        while (lo_s < hi_s) {
            const int mid = (lo_s + hi_s + 1) >> 1;
            if (seg_pre[mid] <= first) lo_s = mid; else hi_s = mid - 1;
        }
        sg = lo_s;
    }
    for (int t = it0; t < it1; ++t) {
        while (seg_pre[sg + 1] <= t) ++sg;
        const int64_t p = (int64_t)seg_start[sg] + (t - seg_pre[sg]);
        const int info = seg_info[sg];
        const int hx = (info & 0xff) + (P.cellid[p] - seg_c0[sg]);
        const int hy = (info >> 8) & 0xff, hz = info >> 16;
        // unwrapped fixed-point coordinates relative to the grid origin
        const int X[3] = {(c0x - 1 + hx) * FIX + (int)P.off0[p], (c0y - 1 + hy) * FIX + (int)P.off1[p],
                          (c0z - 1 + hz) * FIX + (int)P.off2[p]};
        const int c0[3] = {c0x, c0y, c0z};
        const int e[3] = {ex, ey, ez};
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int s = l == 0 ? S0 : S1;
            constexpr int own0 = S0 >= 0 ? (BI >> S0) : (BI << (-S0));
            constexpr int own1 = S1 >= 0 ? (BI >> S1) : (BI << (-S1));
            const int own = l == 0 ? own0 : own1;
            const int tile_off = l == 0 ? 0 : own0 * own0 * own0;
            int i0[3], w0[3], w1[3], ext[3];
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
            // a halo particle whose cloud misses the owned cells on some axis
            // (most of them on the finer levels) has nothing to add here
            if (i0[0] + 1 < 0 || i0[0] >= ext[0] || i0[1] + 1 < 0 || i0[1] >= ext[1] || i0[2] + 1 < 0 ||
                i0[2] >= ext[2])
                continue;
            unsigned int *tlo = lo + tile_off, *thi = hi + tile_off;
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
                        const unsigned long long wgt = wyz * (unsigned long long)(cx ? w1[0] : w0[0]);
                        if (wgt == 0ull) continue;
                        const int cell = (iz * own + iy) * own + ix;
                        const unsigned int wl = (unsigned int)wgt, wh = (unsigned int)(wgt >> 32);
                        const unsigned int old = atomicAdd(&tlo[cell], wl);
                        const unsigned int add_hi = wh + ((old + wl < old) ? 1u : 0u);
                        if (add_hi) {
                            const unsigned int oldh = atomicAdd(&thi[cell], add_hi);
                            if (oldh + add_hi < oldh) set_status(P.status, ST_CAPACITY);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();

    // epilogue: each owned cell converted and written once
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const DepLevel &L = P.lev[l];
        const int s = l == 0 ? S0 : S1;
        constexpr int own0 = S0 >= 0 ? (BI >> S0) : (BI << (-S0));
        constexpr int own1 = S1 >= 0 ? (BI >> S1) : (BI << (-S1));
        const int own = l == 0 ? own0 : own1;
        const int ox = s >= 0 ? (c0x >> s) : (c0x << (-s));
        const int oy = s >= 0 ? (c0y >> s) : (c0y << (-s));
        const int oz = s >= 0 ? (c0z >> s) : (c0z << (-s));
        const int exl = s >= 0 ? (ex >> s) : (ex << (-s));
        const int eyl = s >= 0 ? (ey >> s) : (ey << (-s));
        const int ezl = s >= 0 ? (ez >> s) : (ez << (-s));
        const int tile_off = l == 0 ? 0 : own0 * own0 * own0;
        const unsigned int *tlo = lo + tile_off, *thi = hi + tile_off;
        if (L.out_f32 && own % 4 == 0 && exl % 4 == 0 && ox % 4 == 0 && L.n % 4 == 0 && tile_off % 4 == 0 &&
            P.tile_total % 4 == 0) {
            // four cells of a row per thread: 16-byte shared loads of both
            // words and one 16-byte store of the FP32 values
            const int q = exl >> 2, groups = q * eyl * ezl;
            for (int gi = threadIdx.x; gi < groups; gi += blockDim.x) {
                const int r = gi / q, ix = (gi - r * q) << 2;
                const int iy = r % eyl, iz = r / eyl;
                const int cell = (iz * own + iy) * own + ix;
                const uint4 l4 = *reinterpret_cast<const uint4 *>(&tlo[cell]);
                const uint4 h4 = *reinterpret_cast<const uint4 *>(&thi[cell]);
                const int64_t g = ((int64_t)(oz + iz) * L.n + (oy + iy)) * L.n + (ox + ix);
                float4 f;
                f.x = u64_delta_to_f32(((uint64_t)h4.x << 32) | l4.x, L.mean_int, L.scale);
                f.y = u64_delta_to_f32(((uint64_t)h4.y << 32) | l4.y, L.mean_int, L.scale);
                f.z = u64_delta_to_f32(((uint64_t)h4.z << 32) | l4.z, L.mean_int, L.scale);
                f.w = u64_delta_to_f32(((uint64_t)h4.w << 32) | l4.w, L.mean_int, L.scale);
                *reinterpret_cast<float4 *>(&L.out_f32[g]) = f;
            }
            continue;
        }
        const int cells = exl * eyl * ezl;
        for (int i = threadIdx.x; i < cells; i += blockDim.x) {
            const int ix = i % exl, iy = (i / exl) % eyl, iz = i / (exl * eyl);
            const int cell = (iz * own + iy) * own + ix;
            const uint64_t v = ((uint64_t)thi[cell] << 32) | (uint64_t)tlo[cell];
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
    P.count = p->count; P.start = p->start; P.cellid = ctx->cellid;
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
    P.tile_total = tile;
    const size_t smem = (size_t)tile * 8;
    const int64_t blocks = (int64_t)P.nbx * P.nbx * P.nbx;
    ProfScope prof(ctx, P_DEPOSIT, 0);
    const int s0 = P.lev[0].shift, s1 = P.nl > 1 ? P.lev[1].shift : s0;
    cudaError_t e = cudaErrorInvalidValue;
#define CUBE2_DEPOSIT_CASE(NL_, A_, B_, BI_)                                                           \
    if (P.nl == NL_ && s0 == A_ && s1 == B_) {                                                         \
        static bool attr = false;                                                                      \
        if (!attr) {                                                                                   \
            cudaFuncSetAttribute(deposit_kernel<NL_, A_, B_, BI_>,                                     \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);             \
            attr = true;                                                                               \
        }                                                                                              \
        deposit_kernel<NL_, A_, B_, BI_><<<(unsigned)blocks, DEP_THREADS, smem, ctx->stream>>>(P);     \
        e = cudaGetLastError();                                                                        \
    }
    CUBE2_DEPOSIT_CASE(1, 1, 1, 8)
    CUBE2_DEPOSIT_CASE(1, 0, 0, 8)
    CUBE2_DEPOSIT_CASE(1, -1, -1, 8)
    CUBE2_DEPOSIT_CASE(1, -2, -2, 4)
    CUBE2_DEPOSIT_CASE(2, 1, 0, 8)
    CUBE2_DEPOSIT_CASE(2, 1, -1, 8)
    CUBE2_DEPOSIT_CASE(2, 1, -2, 4)
    CUBE2_DEPOSIT_CASE(2, 0, -1, 8)
    CUBE2_DEPOSIT_CASE(2, 0, -2, 4)
    CUBE2_DEPOSIT_CASE(2, -1, -2, 4)
#undef CUBE2_DEPOSIT_CASE
    ctx->launches++;
    return e;
}

}  // namespace cube2
