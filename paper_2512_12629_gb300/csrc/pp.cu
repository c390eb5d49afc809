// Short-range particle-particle force (paper Sec. 2.2.3 and Eq. PP):
//   F_i += V_p / (4 pi) (R(r, b_pp) - R(r, b_range)) (x_j - x_i) / r,   0 < r < b_range,
// with R(r, b) of Eq. (refforce).  The IOS order is the cell list (Sec. 2.3): the
// IOS cell is at least b_range wide, so the 27 cells around a particle's cell
// hold all its partners.  The three cells of one (dz, dy) row are adjacent in
// memory, so the 27 cells are walked as 9 contiguous particle ranges (two where
// the row wraps around the box).
//
// Arithmetic is carried out in IOS-cell units.  A particle's in-cell offset
// off/2^16 is exact in FP32 (prep kernel, once per force evaluation) and so is
// (cell step + offset) and the separation of two such values: the pair term is
// bitwise antisymmetric.  Each ordered pair is evaluated from both sides (gather
// form, no atomics, deterministic).
//
// One thread per target, in particle (= cell) order.  Where
// all 32 targets of a warp sit in one cell (the clustered regime) they share
// their 27 neighbour cells: the warp stages 32 sources at a time in a per-warp
// shared-memory tile, each lane tests all 32 into an in-range bit mask and
// evaluates only the set bits.  Warps spanning several cells walk each lane's
// own ranges.  Per-particle sums are compensated: plain FP32 partials per tile
// (or per row of cells) are added to the running total with Kahan's scheme.
// The path a warp takes depends only on the cell counts and every sum has a
// fixed order, so results are bitwise reproducible.
#include "common.cuh"

namespace cube2 {
namespace {

struct PPParams {
    const float4 *pos;          // [N] (off_x, off_y, off_z)/2^16, .w = cell id bits
    const int32_t *count, *start;
    float *acc0, *acc1, *acc2;
    float *vel0, *vel1, *vel2;
    unsigned long long *stats;  // [2]: in-range ordered pairs, candidates
    int64_t N;
    int n_ios, accumulate;
    float inv_bpp, inv_bcut, bcut2;   // IOS-cell units
    float coef;                       // V_p / (4 pi s_ios^2)
    float kick;                       // 0: no kick; else v += kick * acc after the sum
    int *status;
};

// R(r, b) of Eq. (refforce) times b^2, as a function of u = r / b < 1.
__device__ __forceinline__ float ref_force_scaled(float u) {
    if (u < 0.5f) {
        // 64/5 u - 256/5 u^3 + 32 u^4 + 1536/35 u^5 - 192/5 u^6
        return u * (64.0f / 5.0f + u * u * (-256.0f / 5.0f + u * (32.0f + u * (1536.0f / 35.0f - 192.0f / 5.0f * u))));
    }
    // 3/(35 u^2) - 32/5 + 256/5 u - 96 u^2 + 256/5 u^3 + 32 u^4 - 1536/35 u^5 + 64/5 u^6
    const float poly = -32.0f / 5.0f + u * (256.0f / 5.0f + u * (-96.0f + u * (256.0f / 5.0f + u * (32.0f + u * (-1536.0f / 35.0f + 64.0f / 5.0f * u)))));
    return 3.0f / (35.0f * u * u) + poly;
}

// R_PP(r) / r for 0 < r < b_cut (Eq. PP), IOS-cell units.  Where r >= b_pp the
// first term is 1/r^2 and the difference is written as m(u)/r^2 with
// u = r/b_cut: for u >= 1/2 the outer-shell branch of Eq. (refforce) gives
// r^2 (1/r^2 - R) = v^5 (192/5 - 416/5 v + 2048/35 v^2 - 64/5 v^3), v = 1 - u
// (an exact polynomial shift, free of cancellation near the cutoff); below
// u = 1/2 the inner branch gives 1 - 64/5 u^3 + 256/5 u^5 - 32 u^6
// - 1536/35 u^7 + 192/5 u^8.
__device__ __forceinline__ float pp_over_r(float r2, float inv_bpp, float inv_bcut) {
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float u = r * inv_bcut;
    const float v = 1.0f - u;
    const float v2 = v * v;
    const float m_out = v2 * v2 * v * (192.0f / 5.0f + v * (-416.0f / 5.0f + v * (2048.0f / 35.0f - 64.0f / 5.0f * v)));
    const float u2 = u * u;
    const float m_in = 1.0f + u2 * u * (-64.0f / 5.0f + u2 * (256.0f / 5.0f + u * (-32.0f + u * (-1536.0f / 35.0f + 192.0f / 5.0f * u))));
    float val = (u >= 0.5f ? m_out : m_in) * rinv * rinv;
    if (r * inv_bpp < 1.0f)   // closer than b_pp: both terms are softened (rare)
        val = ref_force_scaled(r * inv_bpp) * inv_bpp * inv_bpp - ref_force_scaled(r * inv_bcut) * inv_bcut * inv_bcut;
    return val * rinv;
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__device__ __forceinline__ void finish(const PPParams &P, int64_t i, float a0, float a1, float a2) {
    if (P.accumulate) {
        a0 += P.acc0[i];
        a1 += P.acc1[i];
        a2 += P.acc2[i];
    }
    P.acc0[i] = a0;
    P.acc1[i] = a1;
    P.acc2[i] = a2;
    if (P.kick != 0.0f) {
        const float v0 = P.vel0[i] + P.kick * a0;
        const float v1 = P.vel1[i] + P.kick * a1;
        const float v2 = P.vel2[i] + P.kick * a2;
        P.vel0[i] = v0;
        P.vel1[i] = v1;
        P.vel2[i] = v2;
        if (!isfinite(v0) || !isfinite(v1) || !isfinite(v2)) set_status(P.status, ST_NONFINITE);
    } else if (!isfinite(a0) || !isfinite(a1) || !isfinite(a2)) {
        set_status(P.status, ST_NONFINITE);
    }
}

__device__ __forceinline__ void add_stats(unsigned long long *stats, unsigned long long pairs,
                                          unsigned long long cands) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        cands += __shfl_xor_sync(0xffffffffu, cands, o);
    }
    if ((threadIdx.x & 31) == 0 && (pairs | cands)) {
        atomicAdd(&stats[0], pairs);
        atomicAdd(&stats[1], cands);
    }
}


// The particles of the three cells (x-1, x, x+1) of row r as at most two
// contiguous ranges; dx of particle j in range k is base[k] + (j >= b1[k]) + (j >= b2[k]).
struct RowRanges {
    int beg[2], end[2], b1[2], b2[2], base[2];
    int nseg;
    __device__ __forceinline__ RowRanges(const PPParams &P, int64_t r, int cx, int n) {
        const int BIG = 0x7fffffff;
        if (cx > 0 && cx < n - 1) {
            nseg = 1;
            beg[0] = __ldg(&P.start[r + cx - 1]);
            b1[0] = __ldg(&P.start[r + cx]);
            b2[0] = __ldg(&P.start[r + cx + 1]);
            end[0] = b2[0] + __ldg(&P.count[r + cx + 1]);
            base[0] = -1;
        } else if (cx == 0) {
            nseg = 2;
            beg[0] = __ldg(&P.start[r]);
            b1[0] = __ldg(&P.start[r + 1]);
            b2[0] = BIG;
            end[0] = b1[0] + __ldg(&P.count[r + 1]);
            base[0] = 0;
            beg[1] = __ldg(&P.start[r + n - 1]);
            end[1] = beg[1] + __ldg(&P.count[r + n - 1]);
            b1[1] = b2[1] = BIG;
            base[1] = -1;
        } else {
            nseg = 2;
            beg[0] = __ldg(&P.start[r + n - 2]);
            b1[0] = __ldg(&P.start[r + n - 1]);
            b2[0] = BIG;
            end[0] = b1[0] + __ldg(&P.count[r + n - 1]);
            base[0] = -1;
            beg[1] = __ldg(&P.start[r]);
            end[1] = beg[1] + __ldg(&P.count[r]);
            b1[1] = b2[1] = BIG;
            base[1] = 1;
        }
    }
    __device__ __forceinline__ int size() const { return (end[0] - beg[0]) + (nseg > 1 ? end[1] - beg[1] : 0); }
};

constexpr int PP_WARPS_CTA = 8;
constexpr int PP_CTA = PP_WARPS_CTA * 32;

// Float offsets (and the cell id bits) for the PP kernel.
__global__ void __launch_bounds__(PP_CTA) prep_positions_kernel(const uint16_t *off0, const uint16_t *off1,
                                                                const uint16_t *off2, const int32_t *cellid,
                                                                float4 *pos, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = 1.0f / FIX;
    pos[i] = make_float4((float)off0[i] * s, (float)off1[i] * s, (float)off2[i] * s, __int_as_float(cellid[i]));
}

// Compensated sum of three components: terms are added plainly into a block
// partial (a tile or a row of candidates), and each block partial is added to
// the running total with Kahan compensation.
struct Sum3 {
    float x = 0.f, y = 0.f, z = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    __device__ __forceinline__ void add_block(float bx, float by, float bz) {
        kahan_add(x, cx, bx);
        kahan_add(y, cy, by);
        kahan_add(z, cz, bz);
    }
};

__global__ void __launch_bounds__(PP_CTA) pp_kernel(PPParams P) {
    __shared__ float tx[PP_WARPS_CTA][32], ty[PP_WARPS_CTA][32], tz[PP_WARPS_CTA][32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *sx = tx[wib], *sy = ty[wib], *sz = tz[wib];
    const bool has = i < P.N;
    const int n = P.n_ios;
    const float4 me0 = has ? P.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int c = has ? __float_as_int(me0.w) : -1;
    const int c0 = __shfl_sync(0xffffffffu, c, 0);
    if (!has) c = c0;
    const bool uniform = __all_sync(0xffffffffu, c == c0);
    const int cx = c % n, cy = (c / n) % n, cz = c / (n * n);
    Sum3 a;
    unsigned long long pairs = 0, cands = 0;
    if (uniform) {
        // the warp's targets share their 27 neighbour cells: stage 32 sources at a
        // time (3x3x3-cell frame, padded with far-away points), test all 32 into a
        // mask, evaluate the set bits
        const float mx = me0.x + 1.0f, my = me0.y + 1.0f, mz = me0.z + 1.0f;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy) {
                const int64_t r = ((int64_t)wrap(cz + dz, n) * n + wrap(cy + dy, n)) * n;
                const RowRanges rr(P, r, cx, n);
                if (has) cands += rr.size();
                for (int sgi = 0; sgi < rr.nseg; ++sgi) {
                    const int beg = sgi ? rr.beg[1] : rr.beg[0], end = sgi ? rr.end[1] : rr.end[0];
                    const int b1 = sgi ? rr.b1[1] : rr.b1[0], b2 = sgi ? rr.b2[1] : rr.b2[0];
                    const int base = (sgi ? rr.base[1] : rr.base[0]) + 1;
                    for (int t0 = beg; t0 < end; t0 += 32) {
                        const int j = t0 + lane;
                        if (j < end) {
                            const float4 q = __ldg(&P.pos[j]);
                            sx[lane] = q.x + (float)(base + (j >= b1) + (j >= b2));
                            sy[lane] = q.y + (float)(dy + 1);
                            sz[lane] = q.z + (float)(dz + 1);
                        } else {
                            sx[lane] = 1.0e18f;
                            sy[lane] = 1.0e18f;
                            sz[lane] = 1.0e18f;
                        }
                        __syncwarp();
                        unsigned mask = 0u;
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            const float rx = sx[k] - mx, ry = sy[k] - my, rz = sz[k] - mz;
                            const float r2 = rx * rx + ry * ry + rz * rz;
                            mask |= (r2 < P.bcut2 && r2 > 0.0f) ? (1u << k) : 0u;
                        }
                        if (!has) mask = 0u;
                        pairs += __popc(mask);
                        float px = 0.f, py = 0.f, pz = 0.f;
                        while (mask) {
                            const int k = __ffs(mask) - 1;
                            mask &= mask - 1u;
                            const float rx = sx[k] - mx, ry = sy[k] - my, rz = sz[k] - mz;
                            const float g = P.coef * pp_over_r(rx * rx + ry * ry + rz * rz, P.inv_bpp, P.inv_bcut);
                            px += g * rx;
                            py += g * ry;
                            pz += g * rz;
                        }
                        a.add_block(px, py, pz);
                        __syncwarp();
                    }
                }
            }
    } else if (has) {
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy) {
                const int64_t r = ((int64_t)wrap(cz + dz, n) * n + wrap(cy + dy, n)) * n;
                const RowRanges rr(P, r, cx, n);
                cands += rr.size();
                const float fdy = (float)dy, fdz = (float)dz;
                float px = 0.f, py = 0.f, pz = 0.f;
                for (int sgi = 0; sgi < rr.nseg; ++sgi) {
                    for (int j = rr.beg[sgi]; j < rr.end[sgi]; ++j) {
                        const float4 q = __ldg(&P.pos[j]);
                        const float fdx = (float)(rr.base[sgi] + (j >= rr.b1[sgi]) + (j >= rr.b2[sgi]));
                        const float rx = (fdx + q.x) - me0.x;
                        const float ry = (fdy + q.y) - me0.y;
                        const float rz = (fdz + q.z) - me0.z;
                        const float r2 = rx * rx + ry * ry + rz * rz;
                        if (r2 < P.bcut2 && r2 > 0.0f) {
                            const float g = P.coef * pp_over_r(r2, P.inv_bpp, P.inv_bcut);
                            px += g * rx;
                            py += g * ry;
                            pz += g * rz;
                            ++pairs;
                        }
                    }
                }
                a.add_block(px, py, pz);
            }
    }
    if (has) finish(P, i, a.x - a.cx, a.y - a.cy, a.z - a.cz);
    add_stats(P.stats, pairs, cands);
}

}  // namespace

cudaError_t launch_pp(cube2_ctx *ctx, const cube2_particles *p, int accumulate, float kick) {
    PPParams P{};
    P.pos = ctx->pos4;
    P.count = p->count; P.start = p->start;
    P.acc0 = p->acc[0]; P.acc1 = p->acc[1]; P.acc2 = p->acc[2];
    P.vel0 = p->vel[0]; P.vel1 = p->vel[1]; P.vel2 = p->vel[2];
    P.stats = ctx->pp_stats;
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.accumulate = accumulate;
    const double s = ctx->s_ios;
    P.inv_bpp = (float)(s / ctx->cfg.b_pp);
    P.inv_bcut = (float)(s / ctx->b_range);
    P.bcut2 = (float)((ctx->b_range / s) * (ctx->b_range / s));
    const double vp = ctx->cfg.box * ctx->cfg.box * ctx->cfg.box / (double)ctx->N;
    P.coef = (float)(vp / (4.0 * 3.14159265358979323846) / (s * s));
    P.kick = kick;
    P.status = ctx->dev_status;
    if (ctx->N == 0) return cudaSuccess;
    const int nblocks = (int)((ctx->N + PP_CTA - 1) / PP_CTA);
    {
        ProfScope prof(ctx, P_PREP, 0);
        prep_positions_kernel<<<(unsigned)nblocks, PP_CTA, 0, ctx->stream>>>(p->off[0], p->off[1], p->off[2],
                                                                           ctx->cellid, ctx->pos4, ctx->N);
    }
    {
        ProfScope prof(ctx, P_PP, 0);
        pp_kernel<<<(unsigned)nblocks, PP_CTA, 0, ctx->stream>>>(P);
    }
    ctx->launches += 2;
    return cudaGetLastError();
}

}  // namespace cube2
