// FP32 pipe probe: the denominator of the PP kernel's roofline.  The PP force
// is plain FP32 arithmetic (no dense contraction), so its ceiling is the FMA
// rate of the SMs; this kernel measures that rate on the device at hand
// instead of deriving it from unit counts.  Each thread runs eight
// independent chains of dependent FMAs (enough independent work to cover the
// FMA latency at full occupancy); nothing is read from or written to memory
// inside the loop.
#include "common.cuh"

namespace cube2 {
namespace {

constexpr int PROBE_CHAINS = 8;

__global__ void fma_probe_kernel(float *out, int iters, float b, float c) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    // never true for the arguments the library passes; keeps the chains live
    if (s == 1234567.0f) out[0] = s;
}

}  // namespace
}  // namespace cube2

extern "C" int cube2_fma_probe(float *out, int blocks, int threads, int iters, void *stream) {
    if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || threads % 32 || iters <= 0) return CUBE2_ERR_BAD_ARG;
    cube2::fma_probe_kernel<<<(unsigned)blocks, (unsigned)threads, 0, (cudaStream_t)stream>>>(out, iters, 0.999999f,
                                                                                            1e-7f);
    return cudaGetLastError() == cudaSuccess ? CUBE2_OK : CUBE2_ERR_CUDA;
}
