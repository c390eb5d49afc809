// Short-range particle-particle force (paper Sec. 2.2.3 and Eq. PP):
//   F_i += V_p / (4 pi) (R(r, b_pp) - R(r, b_range)) (x_j - x_i) / r,   0 < r < b_range,
// with R(r, b) of Eq. (refforce).  The IOS order is the cell list (Sec. 2.3): the
// IOS cell is at least b_range wide, so the 27 cells around a particle's cell
// hold all its partners.  Separations are formed exactly in fixed point,
// (dc 2^16 + off_j - off_i), so the pair term is bitwise antisymmetric; each
// ordered pair is evaluated from both sides (gather form, no atomics) and
// summed in FP32 with Kahan compensation.
#include "common.cuh"

namespace cube2 {
namespace {

struct PPParams {
    const uint16_t *off0, *off1, *off2;
    const int32_t *count, *start, *cellid;
    float *acc0, *acc1, *acc2;
    float *vel0, *vel1, *vel2;
    int64_t N;
    int n_ios, accumulate;
    float unit;           // s_ios / 2^16 [Mpc/h per fixed-point unit]
    float inv_bpp, inv_bcut, bcut2;
    float coef;           // V_p / (4 pi)
    float kick;           // 0: no kick; else v += kick * acc after the sum
    int *status;
};

// R(r, b) of Eq. (refforce) as u^-2 P(u) / b^2 with u = r / b, for u < 1;
// callers handle u >= 1 (where R = 1/r^2).
__device__ __forceinline__ float ref_force_inside(float u, float inv_b) {
    float p;
    if (u < 0.5f) {
        // 64/5 u - 256/5 u^3 + 32 u^4 + 1536/35 u^5 - 192/5 u^6
        p = u * (64.0f / 5.0f + u * u * (-256.0f / 5.0f + u * (32.0f + u * (1536.0f / 35.0f - 192.0f / 5.0f * u))));
    } else {
        // 3/(35 u^2) - 32/5 + 256/5 u - 96 u^2 + 256/5 u^3 + 32 u^4 - 1536/35 u^5 + 64/5 u^6
        const float poly = -32.0f / 5.0f + u * (256.0f / 5.0f + u * (-96.0f + u * (256.0f / 5.0f + u * (32.0f + u * (-1536.0f / 35.0f + 64.0f / 5.0f * u)))));
        p = 3.0f / (35.0f * u * u) + poly;
    }
    return p * inv_b * inv_b;
}

// R_PP(r) = R(r, b_pp) - R(r, b_cut) for 0 < r < b_cut (Eq. PP).  Where
// r >= b_pp the first term is 1/r^2 and the difference is written as m(u)/r^2
// with u = r/b_cut: on b_cut/2 <= r the outer-shell branch of Eq. (refforce)
// gives r^2 (1/r^2 - R) = v^5 (192/5 - 416/5 v + 2048/35 v^2 - 64/5 v^3),
// v = 1 - u (exact polynomial shift, no cancellation near the cutoff); below
// b_cut/2 the inner branch gives 1 - 64/5 u^3 + 256/5 u^5 - 32 u^6
// - 1536/35 u^7 + 192/5 u^8.
__device__ __forceinline__ float pp_reference(float r, float rinv, float inv_bpp, float inv_bcut) {
    if (r * inv_bpp >= 1.0f) {
        const float u = r * inv_bcut;
        float m;
        if (u >= 0.5f) {
            const float v = 1.0f - u;
            const float v2 = v * v;
            m = v2 * v2 * v * (192.0f / 5.0f + v * (-416.0f / 5.0f + v * (2048.0f / 35.0f - 64.0f / 5.0f * v)));
        } else {
            const float u2 = u * u;
            m = 1.0f + u2 * u * (-64.0f / 5.0f + u2 * (256.0f / 5.0f + u * (-32.0f + u * (-1536.0f / 35.0f + 192.0f / 5.0f * u))));
        }
        return m * rinv * rinv;
    }
    return ref_force_inside(r * inv_bpp, inv_bpp) - ref_force_inside(r * inv_bcut, inv_bcut);
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__global__ void __launch_bounds__(256) pp_kernel(PPParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int n = P.n_ios;
    const int c = P.cellid[i];
    const int cx = c % n, cy = (c / n) % n, cz = c / (n * n);
    const int ox = P.off0[i], oy = P.off1[i], oz = P.off2[i];
    float fx = 0.f, fy = 0.f, fz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
    for (int dz = -1; dz <= 1; ++dz) {
        const int zc = wrap(cz + dz, n);
        for (int dy = -1; dy <= 1; ++dy) {
            const int yc = wrap(cy + dy, n);
            for (int dx = -1; dx <= 1; ++dx) {
                const int xc = wrap(cx + dx, n);
                const int64_t nc = ((int64_t)zc * n + yc) * n + xc;
                const int s = __ldg(&P.start[nc]);
                const int e = s + __ldg(&P.count[nc]);
                for (int j = s; j < e; ++j) {
                    const float rx = (float)(dx * FIX + (int)__ldg(&P.off0[j]) - ox) * P.unit;
                    const float ry = (float)(dy * FIX + (int)__ldg(&P.off1[j]) - oy) * P.unit;
                    const float rz = (float)(dz * FIX + (int)__ldg(&P.off2[j]) - oz) * P.unit;
                    const float r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 >= P.bcut2 || r2 == 0.0f) continue;   // also skips j == i
                    const float rinv = rsqrtf(r2);
                    const float r = r2 * rinv;
                    const float g = P.coef * pp_reference(r, rinv, P.inv_bpp, P.inv_bcut) * rinv;
                    kahan_add(fx, kx, g * rx);
                    kahan_add(fy, ky, g * ry);
                    kahan_add(fz, kz, g * rz);
                }
            }
        }
    }
    float a0 = fx, a1 = fy, a2 = fz;
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

}  // namespace

cudaError_t launch_pp(cube2_ctx *ctx, const cube2_particles *p, int accumulate, float kick) {
    PPParams P{};
    P.off0 = p->off[0]; P.off1 = p->off[1]; P.off2 = p->off[2];
    P.count = p->count; P.start = p->start; P.cellid = ctx->cellid;
    P.acc0 = p->acc[0]; P.acc1 = p->acc[1]; P.acc2 = p->acc[2];
    P.vel0 = p->vel[0]; P.vel1 = p->vel[1]; P.vel2 = p->vel[2];
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.accumulate = accumulate;
    P.unit = (float)(ctx->s_ios / FIX);
    P.inv_bpp = (float)(1.0 / ctx->cfg.b_pp);
    P.inv_bcut = (float)(1.0 / ctx->b_range);
    P.bcut2 = (float)(ctx->b_range * ctx->b_range);
    const double vp = ctx->cfg.box * ctx->cfg.box * ctx->cfg.box / (double)ctx->N;
    P.coef = (float)(vp / (4.0 * 3.14159265358979323846));
    P.kick = kick;
    P.status = ctx->dev_status;
    const int64_t blocks = (ctx->N + 255) / 256;
    if (blocks == 0) return cudaSuccess;
    ProfScope prof(ctx, P_PP, 0);
    pp_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(P);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace cube2
