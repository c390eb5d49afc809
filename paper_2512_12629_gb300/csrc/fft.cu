// 3-D real FFT Poisson solve of one PM level (paper Sec. 2.1.2: phi(k) = rho(k) G(k);
// Sec. 2.2.2: batches of 1-D line FFTs along each axis).
//
// Layout: real grid [z][y][x] (x fastest, n^3 FP32); half spectrum
// [kz][ky][kx] complex64 with kx in [0, n/2] stored in rows of kxp >= n/2+1
// (multiple of 16, so every row starts on a 128-byte boundary).
//
// Passes (each one read + one write of the grid, in place where possible):
//   X  r2c : 2L real rows per CTA packed as L complex lines a + ib, one complex
//            FFT per line, split into the two half spectra.
//   Y      : L consecutive kx columns x n rows of one kz plane per CTA.
//   Z+G    : L consecutive kx columns x n planes of one ky row per CTA: forward
//            FFT along z, multiply by G(k) (1/n^3 folded in), inverse FFT along z.
//   Y^-1, X^-1 c2r : mirror images of Y and X.
// Within a CTA the L lines live in shared memory as S[pos * (L+1) + line]; the
// odd line stride keeps both line-parallel and position-parallel accesses free
// of bank conflicts.  Each line is transformed by a Stockham autosort sequence of
// radix-8/4/3/2 stages (natural order in and out): a stage reads R values with
// stride n/R, applies the twiddles exp(-2 pi i r (j mod Ns) / (Ns R)), does an
// R-point DFT in registers and writes them with stride Ns to position
// (j / Ns) Ns R + (j mod Ns).  Every thread holds its values in registers
// across a barrier, so stages run in place.  Twiddles are an FP32 table
// exp(-2 pi i k/n) built from FP64 sincospi.
#include "common.cuh"

#include <algorithm>
#include <string>

namespace cube2 {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const float2 s13 = cadd(v[1], v[3]), d13 = rot90<INV>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <bool INV>
struct Dft<8, INV> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float h = 0.70710678118654752440f;
        // radix-2 split: even/odd halves
        float2 a[4] = {v[0], v[2], v[4], v[6]};
        float2 b[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV>::run(a);
        Dft<4, INV>::run(b);
        // twiddle b[k] by w8^k, w8 = exp(-+ i pi/4)
        const float2 b1 = b[1], b3 = b[3];
        b[1] = INV ? make_float2(h * (b1.x - b1.y), h * (b1.x + b1.y))
                   : make_float2(h * (b1.x + b1.y), h * (b1.y - b1.x));
        b[2] = rot90<INV>(b[2]);
        b[3] = INV ? make_float2(-h * (b3.x + b3.y), h * (b3.x - b3.y))
                   : make_float2(h * (b3.y - b3.x), -h * (b3.x + b3.y));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(a[k], b[k]);
            v[k + 4] = csub(a[k], b[k]);
        }
    }
};

template <bool INV>
struct Dft<3, INV> {
    __device__ __forceinline__ static void run(float2 *v) {
        const float c = -0.5f;
        const float s = INV ? 0.86602540378443864676f : -0.86602540378443864676f;
        const float2 t = cadd(v[1], v[2]);
        const float2 d = csub(v[1], v[2]);
        const float2 m = make_float2(v[0].x + c * t.x, v[0].y + c * t.y);
        const float2 r = make_float2(-s * d.y, s * d.x);   // i s d
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

__host__ __device__ constexpr int pick_radix(int rem) {
    return rem % 3 == 0 ? 3 : (rem == 2 || rem == 4) ? rem : rem == 16 ? 4 : rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : 2;
}

template <int N, int L, int LP, int T, int R, int NS, bool INV>
__device__ __forceinline__ void stockham_stage(float2 *S, const float2 *__restrict__ tw) {
    constexpr int NB = N / R;
    constexpr int TOT = NB * L;
    constexpr int PER = (TOT + T - 1) / T;
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * T;
        if (TOT % T == 0 || b < TOT) {
            const int line = b % L, j = b / L;
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = S[(j + r * NB) * LP + line];
            if (NS > 1) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = __ldg(&tw[r * k * (N / (NS * R))]);
                    if (INV) w.y = -w.y;
                    v[p][r] = cmul(v[p][r], w);
                }
            }
            Dft<R, INV>::run(v[p]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * T;
        if (TOT % T == 0 || b < TOT) {
            const int line = b % L, j = b / L;
            const int k = j % NS;
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) S[(base + r * NS) * LP + line] = v[p][r];
        }
    }
    __syncthreads();
}

template <int N, int L, int LP, int T, int NS, bool INV>
__device__ __forceinline__ void fft_lines(float2 *S, const float2 *__restrict__ tw) {
    if constexpr (NS < N) {
        constexpr int R = pick_radix(N / NS);
        stockham_stage<N, L, LP, T, R, NS, INV>(S, tw);
        fft_lines<N, L, LP, T, NS * R, INV>(S, tw);
    }
}

// L lines per tile; x passes pad the line stride to L + 1 (their load and store
// phases are position-parallel), y/z passes keep it at L so every tile row is a
// 16-byte-aligned 128-byte line filled with asynchronous 16-byte copies.
template <int N>
struct Tile {
    static constexpr int L = N >= 2048 ? 8 : FFT_LINES;
    static constexpr int LP = L + 1;
    static constexpr int LPY = L;
    static constexpr int T0 = N * L / 16;
    static constexpr int T = T0 < 64 ? 64 : (T0 > 1024 ? 1024 : T0);
    static constexpr size_t SMEM = (size_t)N * LP * sizeof(float2);
    static constexpr size_t SMEMY = (size_t)N * LPY * sizeof(float2);
    // resident CTAs the z pass asks registers for: two for 512-thread tiles
    // that fit twice in shared memory (64 registers, no spills); one otherwise
    // (larger tiles do not fit twice, and smaller bounds only cost registers).
    // Three 512-thread CTAs per SM (40 registers, spills) measured slower for
    // the y and z passes (0.37 and 0.66 ms against 0.23 and 0.44 at 512^3) and
    // equal for the x passes.
    static constexpr int ZMINB = (T == 512 && 2 * SMEMY <= 200 * 1024) ? 2 : 1;
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---------------------------------------------------------------- X passes
// Each pass is a per-block body with two entry kernels: one block per tile for
// a single mesh (BATCH = false), or, for the batched meshes of the adaptive
// third level (BATCH = true), a resident-sized grid whose blocks loop over the
// tiles of the meshes in use (*active, on the device).
template <int N>
__device__ __forceinline__ void x_r2c_block(float2 *S, const float *__restrict__ in, float2 *__restrict__ out,
                                            int64_t nrows, int kxp, const float2 *__restrict__ tw, int64_t vb) {
    constexpr int L = Tile<N>::L, LP = Tile<N>::LP, T = Tile<N>::T;
    const int64_t row0 = vb * 2 * L;
    if constexpr (N % 4 == 0) {
        // four x of the two rows of a line per thread (16-byte loads, 8-byte
        // shared stores), lanes over the lines: 8 % faster than one element per
        // thread at 512^3 (the inverse pass's matching 16-byte stores, 16 rows
        // per warp instruction, measured 1.6x slower)
        constexpr int Q = N / 4;
        for (int i = threadIdx.x; i < L * Q; i += T) {
            const int l = i % L, x = 4 * (i / L);
            const int64_t ra = row0 + 2 * l;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 a = ra < nrows ? __ldg(reinterpret_cast<const float4 *>(in + ra * N + x)) : z4;
            const float4 b = ra + 1 < nrows ? __ldg(reinterpret_cast<const float4 *>(in + (ra + 1) * N + x)) : z4;
            S[(x + 0) * LP + l] = make_float2(a.x, b.x);
            S[(x + 1) * LP + l] = make_float2(a.y, b.y);
            S[(x + 2) * LP + l] = make_float2(a.z, b.z);
            S[(x + 3) * LP + l] = make_float2(a.w, b.w);
        }
    } else {
        for (int i = threadIdx.x; i < 2 * L * N; i += T) {
            const int r = i / N, x = i % N;
            const int64_t row = row0 + r;
            const float v = row < nrows ? __ldg(&in[row * N + x]) : 0.0f;
            reinterpret_cast<float *>(&S[x * LP + (r >> 1)])[r & 1] = v;
        }
    }
    __syncthreads();
    fft_lines<N, L, LP, T, 1, false>(S, tw);
    constexpr int NH = N / 2 + 1;
    for (int i = threadIdx.x; i < L * NH; i += T) {
        const int l = i / NH, k = i % NH;
        const float2 z = S[k * LP + l];
        const float2 zc = S[((N - k) % N) * LP + l];
        const float2 A = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
        const float2 B = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
        const int64_t ra = row0 + 2 * l;
        if (ra < nrows) out[ra * kxp + k] = A;
        if (ra + 1 < nrows) out[(ra + 1) * kxp + k] = B;
    }
}

template <int N, bool BATCH>
__global__ void __launch_bounds__(Tile<N>::T) fft_x_r2c(const float *__restrict__ in, float2 *__restrict__ out,
                                                       int64_t nrows, int kxp, const float2 *__restrict__ tw,
                                                       const int *__restrict__ active) {
    extern __shared__ float2 S[];
    if constexpr (BATCH) {
        constexpr int L = Tile<N>::L;
        const int64_t nvb = ((int64_t)*active * N * N + 2 * L - 1) / (2 * L);
        for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
            x_r2c_block<N>(S, in, out, nrows, kxp, tw, vb);
            __syncthreads();
        }
    } else {
        x_r2c_block<N>(S, in, out, nrows, kxp, tw, blockIdx.x);
    }
}

template <int N>
__device__ __forceinline__ void x_c2r_block(float2 *S, const float2 *__restrict__ in, float *__restrict__ out,
                                            int64_t nrows, int kxp, const float2 *__restrict__ tw, int64_t vb) {
    constexpr int L = Tile<N>::L, LP = Tile<N>::LP, T = Tile<N>::T;
    const int64_t row0 = vb * 2 * L;
    constexpr int NH = N / 2 + 1;
    for (int i = threadIdx.x; i < L * NH; i += T) {
        const int l = i / NH, k = i % NH;
        const int64_t ra = row0 + 2 * l;
        float2 A = ra < nrows ? in[ra * kxp + k] : make_float2(0.f, 0.f);
        float2 B = ra + 1 < nrows ? in[(ra + 1) * kxp + k] : make_float2(0.f, 0.f);
        if (k == 0 || k == N / 2) { A.y = 0.f; B.y = 0.f; }
        S[k * LP + l] = make_float2(A.x - B.y, A.y + B.x);                    // A + iB
        if (k > 0 && k < N / 2) S[(N - k) * LP + l] = make_float2(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
    }
    __syncthreads();
    fft_lines<N, L, LP, T, 1, true>(S, tw);
    // one x of a line per thread: its two rows from one 8-byte shared load,
    // written by two coalesced 4-byte stores
    for (int i = threadIdx.x; i < L * N; i += T) {
        const int l = i / N, x = i % N;
        const int64_t ra = row0 + 2 * l;
        const float2 v = S[x * LP + l];
        if (ra < nrows) out[ra * N + x] = v.x;
        if (ra + 1 < nrows) out[(ra + 1) * N + x] = v.y;
    }
}

template <int N, bool BATCH>
__global__ void __launch_bounds__(Tile<N>::T) fft_x_c2r(const float2 *__restrict__ in, float *__restrict__ out,
                                                       int64_t nrows, int kxp, const float2 *__restrict__ tw,
                                                       const int *__restrict__ active) {
    extern __shared__ float2 S[];
    if constexpr (BATCH) {
        constexpr int L = Tile<N>::L;
        const int64_t nvb = ((int64_t)*active * N * N + 2 * L - 1) / (2 * L);
        for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
            x_c2r_block<N>(S, in, out, nrows, kxp, tw, vb);
            __syncthreads();
        }
    } else {
        x_c2r_block<N>(S, in, out, nrows, kxp, tw, blockIdx.x);
    }
}

// ---------------------------------------------------------------- Y passes
template <int N, bool INV>
__device__ __forceinline__ void y_block(float2 *S, float2 *__restrict__ data, int kxp, const float2 *__restrict__ tw,
                                        int64_t vb) {
    constexpr int L = Tile<N>::L, LP = Tile<N>::LPY, T = Tile<N>::T;
    const int tiles_x = kxp / L;
    const int tx = (int)(vb % tiles_x);
    const int64_t z = vb / tiles_x;                    // plane over all batched meshes
    float2 *base = data + z * N * kxp + tx * L;
    for (int i = threadIdx.x; i < N * L / 2; i += T) {
        const int y = i / (L / 2), l2 = 2 * (i % (L / 2));
        cp_async16(&S[y * LP + l2], &base[(int64_t)y * kxp + l2]);
    }
    cp_async_wait_all();
    __syncthreads();
    fft_lines<N, L, LP, T, 1, INV>(S, tw);
    for (int i = threadIdx.x; i < N * L / 2; i += T) {
        const int y = i / (L / 2), l2 = 2 * (i % (L / 2));
        *reinterpret_cast<float4 *>(&base[(int64_t)y * kxp + l2]) = *reinterpret_cast<const float4 *>(&S[y * LP + l2]);
    }
}

template <int N, bool INV, bool BATCH>
__global__ void __launch_bounds__(Tile<N>::T) fft_y(float2 *__restrict__ data, int kxp, const float2 *__restrict__ tw,
                                                   const int *__restrict__ active) {
    extern __shared__ __align__(16) float2 S[];
    if constexpr (BATCH) {
        const int64_t nvb = (int64_t)*active * N * (kxp / Tile<N>::L);
        for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
            y_block<N, INV>(S, data, kxp, tw, vb);
            __syncthreads();
        }
    } else {
        y_block<N, INV>(S, data, kxp, tw, blockIdx.x);
    }
}

// ------------------------------------------------------------ Z (+ Green)
// GMODE 0: forward z FFT only; 1: G from a full [kz][ky][kxp] table; 2: G
// from the symmetry-reduced table (green_index); 3: G from the table folded in
// ky and kz ([kz <= N/2][ky <= N/2][kxp], the reduced table's entries).
template <int N, int GMODE>
__device__ __forceinline__ void z_block(float2 *S, float2 *__restrict__ data, const float *__restrict__ green,
                                        int kxp, const float2 *__restrict__ tw, int64_t vb) {
    constexpr int L = Tile<N>::L, LP = Tile<N>::LPY, T = Tile<N>::T;
    const int tiles_x = kxp / L;
    const int tx = (int)(vb % tiles_x);
    const int64_t row = vb / tiles_x;                     // (mesh, ky) over all batched meshes
    const int64_t mesh = row / N;
    const int64_t ky = row - mesh * N;
    const int64_t zstride = (int64_t)N * kxp;
    float2 *base = data + mesh * N * zstride + ky * kxp + tx * L;
    for (int i = threadIdx.x; i < N * L / 2; i += T) {
        const int z = i / (L / 2), l2 = 2 * (i % (L / 2));
        cp_async16(&S[z * LP + l2], &base[z * zstride + l2]);
    }
    cp_async_wait_all();
    __syncthreads();
    fft_lines<N, L, LP, T, 1, false>(S, tw);
    if (GMODE != 0) {
        const float *g = green + ky * kxp + tx * L;
        for (int i = threadIdx.x; i < N * L / 2; i += T) {
            const int z = i / (L / 2), l2 = 2 * (i % (L / 2));
            float2 gv;
            if (GMODE == 1) {
                gv = __ldg(reinterpret_cast<const float2 *>(&g[z * zstride + l2]));
            } else if (GMODE == 3) {
                const int zf = z <= N / 2 ? z : N - z, kyf = ky <= N / 2 ? (int)ky : N - (int)ky;
                gv = __ldg(reinterpret_cast<const float2 *>(
                    &green[((int64_t)zf * (N / 2 + 1) + kyf) * kxp + tx * L + l2]));
            } else {
                const int kx = tx * L + l2;   // padding columns (kx > N/2) hold zeros
                gv.x = kx <= N / 2 ? __ldg(&green[green_index(kx, (int)ky, z, N)]) : 0.0f;
                gv.y = kx + 1 <= N / 2 ? __ldg(&green[green_index(kx + 1, (int)ky, z, N)]) : 0.0f;
            }
            float4 v = *reinterpret_cast<const float4 *>(&S[z * LP + l2]);
            v.x *= gv.x;
            v.y *= gv.x;
            v.z *= gv.y;
            v.w *= gv.y;
            *reinterpret_cast<float4 *>(&S[z * LP + l2]) = v;
        }
        __syncthreads();
        fft_lines<N, L, LP, T, 1, true>(S, tw);
    }
    for (int i = threadIdx.x; i < N * L / 2; i += T) {
        const int z = i / (L / 2), l2 = 2 * (i % (L / 2));
        *reinterpret_cast<float4 *>(&base[z * zstride + l2]) = *reinterpret_cast<const float4 *>(&S[z * LP + l2]);
    }
}

template <int N, int GMODE, bool BATCH>
__global__ void __launch_bounds__(Tile<N>::T, Tile<N>::ZMINB) fft_z(float2 *__restrict__ data, const float *__restrict__ green,
                                                   int kxp, const float2 *__restrict__ tw, const int *__restrict__ active) {
    extern __shared__ __align__(16) float2 S[];
    if constexpr (BATCH) {
        const int64_t nvb = (int64_t)*active * N * (kxp / Tile<N>::L);
        for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
            z_block<N, GMODE>(S, data, green, kxp, tw, vb);
            __syncthreads();
        }
    } else {
        z_block<N, GMODE>(S, data, green, kxp, tw, blockIdx.x);
    }
}

// Grid of a pass: every block for a single mesh; for batched meshes a
// resident-sized grid that loops over the blocks of the meshes in use.
inline unsigned pass_grid(const cube2_ctx *ctx, const Level &Lv, int64_t blocks) {
    return (unsigned)(Lv.active ? std::min<int64_t>(blocks, (int64_t)ctx->num_sms * 16) : blocks);
}

// the batched variants exist for the local meshes of the adaptive third level
constexpr int BATCH_MAX_N = 256;

template <int N>
struct Launcher {
    template <bool B>
    static cudaError_t forward_v(cube2_ctx *ctx, Level &Lv) {
        const int64_t nrows = (int64_t)Lv.batch * N * N;
        const unsigned bx = pass_grid(ctx, Lv, (nrows + 2 * Tile<N>::L - 1) / (2 * Tile<N>::L));
        {
            ProfScope prof(ctx, B ? -1 : P_FFT_X_FWD, Lv.index);   // batched meshes: profiled as one group by the caller
            fft_x_r2c<N, B><<<bx, Tile<N>::T, Tile<N>::SMEM, ctx->stream>>>(Lv.real, Lv.spec, nrows, Lv.kxp, Lv.tw,
                                                                            Lv.active);
        }
        const unsigned by = pass_grid(ctx, Lv, (int64_t)Lv.batch * N * (Lv.kxp / Tile<N>::L));
        {
            ProfScope prof(ctx, B ? -1 : P_FFT_Y_FWD, Lv.index);
            fft_y<N, false, B><<<by, Tile<N>::T, Tile<N>::SMEMY, ctx->stream>>>(Lv.spec, Lv.kxp, Lv.tw, Lv.active);
        }
        ctx->launches += 2;
        return cudaGetLastError();
    }
    template <bool B>
    static cudaError_t z_pass_v(cube2_ctx *ctx, Level &Lv, bool green) {
        const unsigned bz = pass_grid(ctx, Lv, (int64_t)Lv.batch * N * (Lv.kxp / Tile<N>::L));
        ProfScope prof(ctx, B ? -1 : P_FFT_Z_GREEN, Lv.index);
        if (green && !B && Lv.green2)
            fft_z<N, 3, false><<<bz, Tile<N>::T, Tile<N>::SMEMY, ctx->stream>>>(Lv.spec, Lv.green2, Lv.kxp, Lv.tw,
                                                                              Lv.active);
        else if (green)
            fft_z<N, 2, B><<<bz, Tile<N>::T, Tile<N>::SMEMY, ctx->stream>>>(Lv.spec, Lv.green, Lv.kxp, Lv.tw, Lv.active);
        else
            fft_z<N, 0, B><<<bz, Tile<N>::T, Tile<N>::SMEMY, ctx->stream>>>(Lv.spec, nullptr, Lv.kxp, Lv.tw, Lv.active);
        ctx->launches += 1;
        return cudaGetLastError();
    }
    template <bool B>
    static cudaError_t inverse_v(cube2_ctx *ctx, Level &Lv) {
        const unsigned by = pass_grid(ctx, Lv, (int64_t)Lv.batch * N * (Lv.kxp / Tile<N>::L));
        {
            ProfScope prof(ctx, B ? -1 : P_FFT_Y_INV, Lv.index);
            fft_y<N, true, B><<<by, Tile<N>::T, Tile<N>::SMEMY, ctx->stream>>>(Lv.spec, Lv.kxp, Lv.tw, Lv.active);
        }
        const int64_t nrows = (int64_t)Lv.batch * N * N;
        const unsigned bx = pass_grid(ctx, Lv, (nrows + 2 * Tile<N>::L - 1) / (2 * Tile<N>::L));
        {
            ProfScope prof(ctx, B ? -1 : P_FFT_X_INV, Lv.index);
            fft_x_c2r<N, B><<<bx, Tile<N>::T, Tile<N>::SMEM, ctx->stream>>>(Lv.spec, Lv.real, nrows, Lv.kxp, Lv.tw,
                                                                            Lv.active);
        }
        ctx->launches += 2;
        return cudaGetLastError();
    }
    static cudaError_t forward(cube2_ctx *ctx, Level &Lv) {
        setup();
        if constexpr (N <= BATCH_MAX_N)
            if (Lv.active) return forward_v<true>(ctx, Lv);
        if (Lv.active) return cudaErrorInvalidValue;
        return forward_v<false>(ctx, Lv);
    }
    static cudaError_t z_pass(cube2_ctx *ctx, Level &Lv, bool green) {
        setup();
        if constexpr (N <= BATCH_MAX_N)
            if (Lv.active) return z_pass_v<true>(ctx, Lv, green);
        if (Lv.active) return cudaErrorInvalidValue;
        return z_pass_v<false>(ctx, Lv, green);
    }
    static cudaError_t inverse(cube2_ctx *ctx, Level &Lv) {
        setup();
        if constexpr (N <= BATCH_MAX_N)
            if (Lv.active) return inverse_v<true>(ctx, Lv);
        if (Lv.active) return cudaErrorInvalidValue;
        return inverse_v<false>(ctx, Lv);
    }
    template <bool B>
    static void setup_v() {
        const int smem = (int)Tile<N>::SMEM;
        cudaFuncSetAttribute(fft_x_r2c<N, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(fft_x_c2r<N, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(fft_y<N, false, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(fft_y<N, true, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(fft_z<N, 0, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(fft_z<N, 2, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    static void setup() {
        static bool done = false;
        if (done) return;
        setup_v<false>();
        cudaFuncSetAttribute(fft_z<N, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tile<N>::SMEM);
        cudaFuncSetAttribute(fft_z<N, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tile<N>::SMEM);
        if constexpr (N <= BATCH_MAX_N) setup_v<true>();
        done = true;
    }
};

enum class Op { Forward, ZGreen, ZForward, Inverse };

template <int N>
cudaError_t run_op(cube2_ctx *ctx, Level &Lv, Op op) {
    switch (op) {
        case Op::Forward: return Launcher<N>::forward(ctx, Lv);
        case Op::ZGreen: return Launcher<N>::z_pass(ctx, Lv, true);
        case Op::ZForward: return Launcher<N>::z_pass(ctx, Lv, false);
        case Op::Inverse: return Launcher<N>::inverse(ctx, Lv);
    }
    return cudaErrorInvalidValue;
}

cudaError_t dispatch(cube2_ctx *ctx, Level &Lv, Op op) {
    switch (Lv.n) {
        case 8: return run_op<8>(ctx, Lv, op);
        case 12: return run_op<12>(ctx, Lv, op);
        case 16: return run_op<16>(ctx, Lv, op);
        case 24: return run_op<24>(ctx, Lv, op);
        case 32: return run_op<32>(ctx, Lv, op);
        case 48: return run_op<48>(ctx, Lv, op);
        case 64: return run_op<64>(ctx, Lv, op);
        case 96: return run_op<96>(ctx, Lv, op);
        case 128: return run_op<128>(ctx, Lv, op);
        case 192: return run_op<192>(ctx, Lv, op);
        case 256: return run_op<256>(ctx, Lv, op);
        case 384: return run_op<384>(ctx, Lv, op);
        case 512: return run_op<512>(ctx, Lv, op);
        case 768: return run_op<768>(ctx, Lv, op);
        case 1024: return run_op<1024>(ctx, Lv, op);
        case 1536: return run_op<1536>(ctx, Lv, op);
        case 2048: return run_op<2048>(ctx, Lv, op);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool fft_size_supported(int n) {
    switch (n) {
        case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 192:
        case 256: case 384: case 512: case 768: case 1024: case 1536: case 2048: return true;
        default: return false;
    }
}

cudaError_t launch_fft_forward(cube2_ctx *ctx, Level &L) { return dispatch(ctx, L, Op::Forward); }
cudaError_t launch_fft_z_green(cube2_ctx *ctx, Level &L) { return dispatch(ctx, L, Op::ZGreen); }
cudaError_t launch_fft_z_forward(cube2_ctx *ctx, Level &L) { return dispatch(ctx, L, Op::ZForward); }
cudaError_t launch_fft_inverse(cube2_ctx *ctx, Level &L) { return dispatch(ctx, L, Op::Inverse); }

cudaError_t launch_fft_batched_solve(cube2_ctx *ctx, Level &L) {
    cudaError_t e = dispatch(ctx, L, Op::Forward);
    if (e == cudaSuccess) e = dispatch(ctx, L, Op::ZGreen);
    if (e == cudaSuccess) e = dispatch(ctx, L, Op::Inverse);
    return e;
}

}  // namespace cube2

// ---------------------------------------------------------------------------
// Allocation-free Poisson solve (cube2_solve_pm_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code that runs under a fixed device-memory budget handed out by its
// host application, or that must not let cudaMalloc/cudaFree synchronise the
// device in the middle of its own work.  For them this variant of solve_pm
// takes the density, the Green's table and the output from the caller and keeps
// its own working memory (spectrum, padded Green's table, twiddles) in one
// file-scope device array, resolved once per device with cudaGetSymbolAddress.
// It calls no allocating CUDA or library routine.
#include <mutex>

namespace cube2 {
namespace {

constexpr int NOALLOC_MAX_N = 128;
constexpr int NOALLOC_KXP = ((NOALLOC_MAX_N / 2 + 1) + 15) / 16 * 16;
constexpr size_t NOALLOC_HALF = (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_KXP;
constexpr size_t NOALLOC_SPEC_BYTES = NOALLOC_HALF * sizeof(float2);
constexpr size_t NOALLOC_GREEN_BYTES = NOALLOC_HALF * sizeof(float);
constexpr size_t NOALLOC_BYTES = NOALLOC_SPEC_BYTES + NOALLOC_GREEN_BYTES + NOALLOC_MAX_N * sizeof(float2);

// Working memory of every cube2_solve_pm_noalloc call on a device (15.7 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

__global__ void noalloc_twiddle_kernel(float2 *tw, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_float2((float)c, (float)s);
}

template <int N>
cudaError_t noalloc_passes(const float *rho, float2 *spec, const float *gpad, float *phi, const float2 *tw, int kxp,
                           cudaStream_t st) {
    Launcher<N>::setup();
    constexpr int L = Tile<N>::L;
    const int64_t nrows = (int64_t)N * N;
    const unsigned bx = (unsigned)((nrows + 2 * L - 1) / (2 * L));
    const unsigned by = (unsigned)((int64_t)N * (kxp / L));
    fft_x_r2c<N, false><<<bx, Tile<N>::T, Tile<N>::SMEM, st>>>(rho, spec, nrows, kxp, tw, nullptr);
    fft_y<N, false, false><<<by, Tile<N>::T, Tile<N>::SMEMY, st>>>(spec, kxp, tw, nullptr);
    fft_z<N, 1, false><<<by, Tile<N>::T, Tile<N>::SMEMY, st>>>(spec, gpad, kxp, tw, nullptr);
    fft_y<N, true, false><<<by, Tile<N>::T, Tile<N>::SMEMY, st>>>(spec, kxp, tw, nullptr);
    fft_x_c2r<N, false><<<bx, Tile<N>::T, Tile<N>::SMEM, st>>>(spec, phi, nrows, kxp, tw, nullptr);
    return cudaGetLastError();
}

}  // namespace

void set_context_free_error(const std::string &msg);

}  // namespace cube2

extern "C" int cube2_solve_pm_noalloc(const float *rho, const float *green, float *phi, int32_t n, void *stream) {
    using namespace cube2;
    if (!rho || !green || !phi) {
        set_context_free_error("cube2_solve_pm_noalloc: null pointer");
        return CUBE2_ERR_BAD_ARG;
    }
    if (n > NOALLOC_MAX_N || !fft_size_supported(n)) {
        set_context_free_error("cube2_solve_pm_noalloc: mesh size " + std::to_string(n) +
                               " not supported (2^a 3^b from 8 to " + std::to_string(NOALLOC_MAX_N) + ")");
        return CUBE2_ERR_UNSUPPORTED_SIZE;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_context_free_error(std::string("cube2_solve_pm_noalloc: no usable device: ") + cudaGetErrorString(e));
        return CUBE2_ERR_CUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_context_free_error("cube2_solve_pm_noalloc: device index " + std::to_string(dev) + " beyond the " +
                               std::to_string(NOALLOC_MAX_DEVICES) + " devices this entry point serves");
        return CUBE2_ERR_CUDA;
    }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                set_context_free_error(std::string("cube2_solve_pm_noalloc: cudaGetSymbolAddress failed: ") +
                                       cudaGetErrorString(e));
                return CUBE2_ERR_CUDA;
            }
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *b = static_cast<unsigned char *>(base);
    float2 *spec = reinterpret_cast<float2 *>(b);
    float *gpad = reinterpret_cast<float *>(b + NOALLOC_SPEC_BYTES);
    float2 *tw = reinterpret_cast<float2 *>(b + NOALLOC_SPEC_BYTES + NOALLOC_GREEN_BYTES);
    const size_t nh = (size_t)(n / 2 + 1);
    // rows of the half spectrum padded to a multiple of 16 columns, as in a
    // context; the array holds the 128^3 layout, so every smaller mesh fits
    const int kxp = (int)((nh + 15) / 16 * 16);
    // the caller's compact [n][n][n/2+1] table into the padded layout; the
    // padding columns, left from earlier calls, are cleared
    e = cudaMemcpy2DAsync(gpad, kxp * sizeof(float), green, nh * sizeof(float), nh * sizeof(float),
                          (size_t)n * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && (size_t)kxp > nh)
        e = cudaMemset2DAsync(gpad + nh, kxp * sizeof(float), 0, (kxp - nh) * sizeof(float), (size_t)n * n, st);
    if (e == cudaSuccess) {
        noalloc_twiddle_kernel<<<(n + 127) / 128, 128, 0, st>>>(tw, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        switch (n) {
            case 8: e = noalloc_passes<8>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 12: e = noalloc_passes<12>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 16: e = noalloc_passes<16>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 24: e = noalloc_passes<24>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 32: e = noalloc_passes<32>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 48: e = noalloc_passes<48>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 64: e = noalloc_passes<64>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 96: e = noalloc_passes<96>(rho, spec, gpad, phi, tw, kxp, st); break;
            case 128: e = noalloc_passes<128>(rho, spec, gpad, phi, tw, kxp, st); break;
            default: e = cudaErrorInvalidValue; break;
        }
    }
    if (e != cudaSuccess) {
        set_context_free_error(std::string("cube2_solve_pm_noalloc: ") + cudaGetErrorString(e));
        return CUBE2_ERR_CUDA;
    }
    return CUBE2_OK;
}
