// Optimised Green's function of one PM level, Eq. (Gk) of the paper (Sec. 2.1.2),
// and the FFT twiddle tables.  FP64 arithmetic on the GPU, FP32 result.
//
// For a mode k = 2 pi m / n (m_d in (-n/2, n/2]) the kernel forms
//   d_d   = 4/3 sin k_d - 1/6 sin 2k_d                     (Eq. diff, D = i d)
//   W^2   = prod_d sinc^(2p)((k_d + 2 pi n_d)/2)            (p = 2 CIC, 3 TSC)
//   dS2   = S^2(|k_n|, b_soft) - S^2(|k_n|, b_trunc)        (Eqs. Rk, Sk)
//           times 1 - sinc(|k_n| L_iso) when the level is isolated (Eq. isok)
//   G     = -sum_n W^2 (d.k_n) dS2/|k_n|^2 / (|d|^2 [sum_n W^2]^2)
// over the images |n_d| <= alias, and stores G / n^3 (the inverse FFT is
// unnormalised) in the symmetry-reduced layout of green_index.  G = 0 where
// |d| = 0.  The alias sum of W^2 factorises per
// axis; the numerator does not and is summed image by image.
#include "common.cuh"

namespace cube2 {
namespace {

constexpr int MAX_ALIAS = 4;

// S(k, b) of Eq. (Sk) with x = k b / 2.  Below x = 1/2 the closed form
// cancels badly, so the Taylor series of 2 - 2cos x - x sin x divided by
// x^4/12 is used there: 12 * sum_{j>=2} (-1)^j (2j-2) x^(2j-4) / (2j)!.
__device__ double profile_transform(double k, double b) {
    if (b < 0) return 0.0;                       // b = infinity
    const double x = 0.5 * k * b;
    if (x < 0.5) {
        const double x2 = x * x;
        double term = 1.0 / 24.0;                // j = 2: (2j-2)/(2j)! = 2/24
        double sum = 0.0;
        double p = 1.0;                          // x^(2j-4)
        for (int j = 2; j <= 13; ++j) {
            // term = 1/(2j)!
            const double c = ((j & 1) ? -1.0 : 1.0) * (2.0 * j - 2.0) * term;
            sum += c * p;
            p *= x2;
            term /= (2.0 * j + 1.0) * (2.0 * j + 2.0);
        }
        return 12.0 * sum;
    }
    double s, c;
    sincos(x, &s, &c);
    const double x2 = x * x;
    return 12.0 / (x2 * x2) * (2.0 - 2.0 * c - x * s);
}

// 1 - sin(x)/x of Eq. (isok); below x = 0.01 its Taylor series (the
// difference cancels there).
__device__ double one_minus_sinc(double x) {
    if (x < 1e-2) {
        const double x2 = x * x;
        return x2 / 6.0 - x2 * x2 / 120.0;
    }
    return 1.0 - sin(x) / x;
}

__device__ double fd_weight(int m, int n) {
    // 4/3 sin(2 pi m/n) - 1/6 sin(4 pi m/n); sinpi gives exact zeros at k in {0, pi}
    const double t = 2.0 * (double)m / (double)n;
    return 4.0 / 3.0 * sinpi(t) - 1.0 / 6.0 * sinpi(2.0 * t);
}

// One entry of the reduced table per thread: entry idx holds the sorted
// triple (a, b, c) of non-negative modes, evaluated as m = (a, b, c).
__global__ void green_kernel(float *__restrict__ G, int n, double b_soft, double b_trunc, double iso,
                             int alias, int order, double norm) {
    const int64_t total = green_table_len(n);
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    // c: largest with c(c+1)(c+2)/6 <= idx; b: largest with b(b+1)/2 <= rest
    int c = (int)cbrt(6.0 * (double)idx);
    while ((int64_t)c * (c + 1) * (c + 2) / 6 > idx) --c;
    while ((int64_t)(c + 1) * (c + 2) * (c + 3) / 6 <= idx) ++c;
    const int64_t rest = idx - (int64_t)c * (c + 1) * (c + 2) / 6;
    int b = (int)((sqrt(8.0 * (double)rest + 1.0) - 1.0) * 0.5);
    while ((int64_t)b * (b + 1) / 2 > rest) --b;
    while ((int64_t)(b + 1) * (b + 2) / 2 <= rest) ++b;
    const int a = (int)(rest - (int64_t)b * (b + 1) / 2);
    const int m[3] = {a, b, c};
    double d[3], d2 = 0.0;
    for (int ax = 0; ax < 3; ++ax) { d[ax] = fd_weight(m[ax], n); d2 += d[ax] * d[ax]; }
    if (d2 == 0.0) { G[idx] = 0.0f; return; }
    const double two_pi = 6.283185307179586476925286766559;
    const double pi = 3.141592653589793238462643383279;
    // per-axis image wavenumbers and squared assignment factors sinc^(2p)(k_n/2)
    double kn[3][2 * MAX_ALIAS + 1], w2[3][2 * MAX_ALIAS + 1];
    double den = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        const double frac = (double)m[ax] / (double)n;
        const double s = sinpi(frac);
        double sum = 0.0;
        for (int i = -alias; i <= alias; ++i) {
            const double u = frac + i;           // k_n / (2 pi)
            kn[ax][i + alias] = two_pi * u;
            double w;
            if (u == 0.0) w = 1.0;
            else {
                const double sc = s / (pi * u), sc2 = sc * sc;
                w = order == 3 ? sc2 * sc2 * sc2 : sc2 * sc2;   // W^2 = sinc^(2 order)
            }
            w2[ax][i + alias] = w;
            sum += w;
        }
        den *= sum;
    }
    double num = 0.0;
    for (int iz = 0; iz <= 2 * alias; ++iz) {
        for (int iy = 0; iy <= 2 * alias; ++iy) {
            const double wyz = w2[1][iy] * w2[2][iz];
            for (int ix = 0; ix <= 2 * alias; ++ix) {
                const double k0 = kn[0][ix], k1 = kn[1][iy], k2 = kn[2][iz];
                const double kk = k0 * k0 + k1 * k1 + k2 * k2;
                if (kk == 0.0) continue;
                const double kabs = sqrt(kk);
                const double s1 = profile_transform(kabs, b_soft);
                const double s2 = profile_transform(kabs, b_trunc);
                double ds2 = s1 * s1 - s2 * s2;
                if (iso > 0.0) ds2 *= one_minus_sinc(kabs * iso);
                num -= w2[0][ix] * wyz * (d[0] * k0 + d[1] * k1 + d[2] * k2) * ds2 / kk;
            }
        }
    }
    G[idx] = (float)(num / (d2 * den * den) * norm);
}

// Full half spectrum [kz][ky][kx <= n/2] from the reduced table.
__global__ void green_expand_kernel(const float *__restrict__ G, float *__restrict__ out, int n) {
    const int nh = n / 2 + 1;
    const int64_t total = (int64_t)n * n * nh;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int kx = (int)(idx % nh), ky = (int)((idx / nh) % n), kz = (int)(idx / ((int64_t)nh * n));
    out[idx] = G[green_index(kx, ky, kz, n)];
}

// [kz <= n/2][ky <= n/2][kx < kxp] from the reduced table (zero past kx = n/2).
__global__ void green_fold_kernel(const float *__restrict__ G, float *__restrict__ out, int n, int kxp) {
    const int h = n / 2 + 1;
    const int64_t total = (int64_t)h * h * kxp;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int kx = (int)(idx % kxp), ky = (int)((idx / kxp) % h), kz = (int)(idx / ((int64_t)kxp * h));
    out[idx] = kx <= n / 2 ? G[green_index(kx, ky, kz, n)] : 0.0f;
}

__global__ void twiddle_kernel(float2 *tw, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_float2((float)c, (float)s);
}

}  // namespace

cudaError_t launch_init_twiddles(cube2_ctx *ctx, Level &L) {
    twiddle_kernel<<<(L.n + 255) / 256, 256, 0, ctx->stream>>>(L.tw, L.n);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_green_expand(cube2_ctx *ctx, const Level &L, float *out) {
    const int64_t total = (int64_t)L.n * L.n * (L.n / 2 + 1);
    green_expand_kernel<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(L.green, out, L.n);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_green_fold(cube2_ctx *ctx, const Level &L) {
    if (!L.green2) return cudaSuccess;
    const int64_t h = L.n / 2 + 1, total = h * h * L.kxp;
    green_fold_kernel<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(L.green, L.green2, L.n, L.kxp);
    ctx->launches++;
    return cudaGetLastError();
}

cudaError_t launch_green(cube2_ctx *ctx, Level &L, int alias, int order) {
    if (alias > MAX_ALIAS) alias = MAX_ALIAS;
    const int64_t total = green_table_len(L.n);
    const double norm = 1.0 / ((double)L.n * (double)L.n * (double)L.n);
    const int threads = 128;
    const int64_t blocks = (total + threads - 1) / threads;
    ProfScope prof(ctx, P_GREEN, L.index);
    green_kernel<<<(unsigned)blocks, threads, 0, ctx->stream>>>(L.green, L.n, L.b_soft, L.b_trunc, L.iso, alias,
                                                                 order, norm);
    ctx->launches++;
    return cudaGetLastError();
}

}  // namespace cube2
