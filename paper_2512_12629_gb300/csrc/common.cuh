// Internal declarations shared by the CUDA translation units of libcube2gb.
// The public C ABI is include/cube2.h; nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cube2.h"

namespace cube2 {

constexpr int FIX_BITS = 16;              // IOS fixed point: 2^16 sub-cells per cell
constexpr int FIX = 1 << FIX_BITS;
constexpr int FFT_LINES = 16;             // lines (columns) per FFT tile
constexpr int DEPOSIT_BRICK = 8;          // IOS cells per CTA brick edge

// Sticky device status bits (first error wins when mapped to a code).
enum StatusBits : int {
    ST_CAPACITY = 1,
    ST_NONFINITE = 2,
    ST_DISPLACEMENT = 4,
    ST_TIMEOUT = 8,
};

// Kernel classes for the optional CUDA-event profile (cube2_profile).
enum ProfClass : int {
    P_DEPOSIT = 0, P_FFT_X_FWD, P_FFT_Y_FWD, P_FFT_Z_GREEN, P_FFT_Y_INV, P_FFT_X_INV,
    P_INTERP, P_PP, P_KICK, P_KICK_DRIFT, P_SCAN, P_SCATTER, P_SORT, P_GATHER, P_CELLID, P_GREEN,
    P_PP_ORDER, P_PREP, P_SORT_BIG,
    P_VJP_GATHER, P_VJP_SOURCE, P_PP_VJP, P_ADJ_KDK,   // adjoint: PM gathers, cotangent source, PP product, reverse KDK
    P_PM3_MAP, P_PM3_DEPOSIT, P_PM3_FFT, P_PM3_GATHER, // adaptive third level: refinement map, local deposit,
                                                       // batched local solves, gather
    P_NCLASS
};

struct Level {
    int index = 0;           // level number (coarsest = 0)
    int n = 0;               // mesh cells per dimension
    int kxp = 0;             // padded width of the half spectrum (>= n/2+1, multiple of 16)
    int shift = 0;           // n_ios / n = 2^shift
    double H = 0;            // cell size [Mpc/h]
    double b_soft = 0;       // softening, this level's cells
    double b_trunc = -1;     // truncation, this level's cells (< 0: infinity)
    double iso = 0;          // isolation length, this level's cells (0: periodic)
    float *real = nullptr;   // [n^3]  density, then potential
    float2 *spec = nullptr;  // [n][n][kxp] half spectrum scratch
    float *green = nullptr;  // symmetry-reduced Green's table (1/n^3 folded in), see green_index
    // the same entries folded in ky and kz only, [n/2+1 (kz)][n/2+1 (ky)][kxp]
    // (zero past kx = n/2): read by the z pass with plain indices (n <= 1024)
    float *green2 = nullptr;
    int64_t green_len = 0;   // entries of the reduced table
    float2 *tw = nullptr;    // [n] twiddles exp(-2 pi i k / n)
    uint64_t mean_int = 0;   // M = floor(N 2^48 / n^3)
    float dens_scale = 0;    // RN32(n^3/N 2^-48)
    bool has_green = false, has_density = false, has_potential = false;
    // batched meshes (the adaptive third level): real/spec hold `batch` meshes
    // back to back; FFT blocks of mesh index >= *active (device) return at once
    int batch = 1;
    const int *active = nullptr;
};

// Adaptive third PM level (Sec. 2.1.1 Eq. PM3, Sec. 2.2.3): local periodic
// meshes over the subtiles whose densest IOS cell is dense enough.
struct PM3 {
    bool on = false;
    int T = 0;               // subtile edge [IOS cells]
    int ns = 0;              // subtiles per dimension (n_ios / T)
    int64_t n_sub = 0;       // ns^3
    int r = 0;               // refinement: H_3 = H_finest / r
    int B = 0;               // buffer [local cells] on each side of the subtile
    int m = 0;               // local mesh cells per dimension
    int q_shift = 0;         // local cell = 2^(16 - q_shift) fixed-point units
    int rho_min = 0;         // refine when max count over the subtile's IOS cells >= rho_min
    int max_tiles = 0;       // capacity of local meshes per force evaluation
    double H = 0;            // local cell [Mpc/h]
    double b3 = 0;           // softening b_3 = beta_3 H_3 [Mpc/h]; PP range of refined subtiles
    float dens_scale = 0;    // RN32(V_p / H_3^3 2^-48)
    Level lev;               // batched meshes: real/spec [max_tiles] meshes, Green's table, twiddles
    int32_t *rho_max = nullptr;          // [n_sub] densest IOS cell per subtile
    int32_t *slot = nullptr;             // [n_sub] local mesh of each subtile, -1 = not refined
    int32_t *list = nullptr;             // [max_tiles] subtile of each local mesh
    int *count = nullptr;                // [2] meshes in use, subtiles asking for refinement
};

}  // namespace cube2

struct cube2_ctx {
    cube2_config cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t aux_stream = nullptr;   // host-buffer step: early downloads
    cudaEvent_t aux_event = nullptr;     // ... after the re-bin
    int device = 0;
    int nl = 0;
    cube2::Level lev[CUBE2_MAX_LEVELS];
    int64_t N = 0;
    int n_ios = 0;
    int64_t n_cells = 0;     // n_ios^3
    double s_ios = 0;        // IOS cell [Mpc/h]
    double b_range = 0;      // PP range [Mpc/h] (softening of the finest level)
    // particle scratch (all [N] unless noted)
    int32_t *cellid = nullptr;
    uint16_t *toff = nullptr;      // [3][N]
    float *tvel = nullptr;         // [3][N]
    int32_t *tcell = nullptr;
    int32_t *tslot = nullptr;
    int32_t *perm = nullptr;
    int32_t *ncount = nullptr;     // [n_cells] histogram of the new cells
    int32_t *nstart = nullptr;     // [n_cells] its exclusive scan
    int32_t *perm2 = nullptr;      // [N] merge scratch of the segmented sort
    int32_t *big = nullptr;        // [n_cells] cells too large for the per-thread sort
    int *big_n = nullptr;          // [2] their numbers (up to 1024 particles, more)
    float4 *pos4 = nullptr;        // [N] in-cell offsets as floats (+ cell id bits), PP order
    int32_t *pp_perm = nullptr;    // [N] particle index of each PP slot (sub-cell order in dense cells)
    unsigned long long *pp_stats = nullptr;  // [4] in-range ordered pairs, candidates; the same of per-lane walks
    int num_sms = 152;
    int32_t *scan_tmp = nullptr;   // block sums of the multi-level scan
    int64_t scan_tmp_len = 0;
    int *dev_status = nullptr;     // sticky device status word
    int *host_status = nullptr;    // pinned mirror
    std::string err;
    int64_t launches = 0;
    // optional per-kernel-class CUDA-event profile
    bool prof = false;
    int prof_overflow = 0;
    cudaEvent_t *ev = nullptr;     // pool of 2 * prof_cap events
    int prof_cap = 0, prof_used = 0;
    int *prof_cls = nullptr;       // [prof_cap] class * CUBE2_MAX_LEVELS + level
    // force vector-Jacobian product scratch (cube2_adjoint_init)
    float *vjp_mu = nullptr;       // [3][n_max^3] CIC deposit of the cotangent
    float *vjp_t = nullptr;        // [3][N] a force product
    float *vjp_u = nullptr;        // [12][N] reverse-step scratch
    double *vjp_sq = nullptr;      // [1] loss accumulator
    cube2::PM3 pm3;                // adaptive third level (cfg.pm3_tile > 0)
    float *vel32 = nullptr;        // [3][N] FP32 working momenta of a step (cfg.vel_fp16 = 1 only)
    // shared-stream width of the PP kernel (warps spanning at most pp_wmax + 1 cells)
    int pp_wmax = 16;
    // PP work counters (cube2_pp_count): off unless asked for
    bool pp_count = false;
    // ensemble recording: launch_pp prepares the PP inputs and leaves the PP
    // kernel to the ensemble's persistent kernel, saving its parameters here
    bool defer_pp = false;
    alignas(16) unsigned char pp_deferred[320];
};

namespace cube2 {

int set_error(cube2_ctx *ctx, int code, const std::string &msg);

// Bracket a launch group with profile events (no-ops unless profiling is on).
int prof_begin(cube2_ctx *ctx, int cls, int level);
void prof_end(cube2_ctx *ctx, int slot);
struct ProfScope {
    cube2_ctx *c;
    int slot;
    ProfScope(cube2_ctx *ctx, int cls, int level = 0) : c(ctx), slot(prof_begin(ctx, cls, level)) {}
    ~ProfScope() { prof_end(c, slot); }
};
int cuda_error(cube2_ctx *ctx, cudaError_t e, const char *what);

// Launch wrappers implemented in the kernel translation units.  Each returns
// the cudaError_t of its last launch and bumps ctx->launches.
cudaError_t launch_init_twiddles(cube2_ctx *ctx, Level &L);
cudaError_t launch_green(cube2_ctx *ctx, Level &L, int alias, int order);
cudaError_t launch_green_expand(cube2_ctx *ctx, const Level &L, float *out);
cudaError_t launch_green_fold(cube2_ctx *ctx, const Level &L);   // full [n][n][n/2+1] copy

// Eq. (Gk) is even in every k_d and symmetric under permutations of the axes
// (cubic mesh, symmetric image sums), so the table is stored once per sorted
// triple 0 <= a <= b <= c <= n/2 of |m_x|, |m_y|, |m_z| (m_d the signed mode):
// entry c(c+1)(c+2)/6 + b(b+1)/2 + a, (n/2+1)(n/2+2)(n/2+3)/6 entries.
__host__ __device__ inline int64_t green_table_len(int n) {
    const int64_t m = n / 2 + 1;
    return m * (m + 1) * (m + 2) / 6;
}
__device__ __forceinline__ int green_index(int kx, int ky, int kz, int n) {
    int a = kx, b = ky <= n / 2 ? ky : n - ky, c = kz <= n / 2 ? kz : n - kz;
    int t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    return c * (c + 1) * (c + 2) / 6 + b * (b + 1) / 2 + a;
}
cudaError_t launch_tsc_deposit(cube2_ctx *ctx, Level &L, const cube2_particles *p);
cudaError_t launch_deposit(cube2_ctx *ctx, int level, const cube2_particles *p, uint64_t *out_u64);
cudaError_t launch_fft_forward(cube2_ctx *ctx, Level &L);          // real -> spec (x, y passes)
cudaError_t launch_fft_z_green(cube2_ctx *ctx, Level &L);          // z fwd * G * z inv
cudaError_t launch_fft_z_forward(cube2_ctx *ctx, Level &L);        // z fwd only (diagnostic)
cudaError_t launch_fft_inverse(cube2_ctx *ctx, Level &L);          // spec -> real (y, x passes)
cudaError_t launch_cellid(cube2_ctx *ctx, const cube2_particles *p);
cudaError_t launch_interp(cube2_ctx *ctx, int level, const cube2_particles *p, int accumulate);
cudaError_t launch_pp(cube2_ctx *ctx, const cube2_particles *p, int accumulate, float kick);
cudaError_t launch_fft_batched_solve(cube2_ctx *ctx, Level &L);     // forward, z * G * z^-1, inverse
cudaError_t launch_pm3(cube2_ctx *ctx, const cube2_particles *p);    // map, local deposit + solve, gather (acc +=)
cudaError_t launch_pm3_map(cube2_ctx *ctx, const cube2_particles *p);  // refinement map only
cudaError_t launch_vel_encode(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3]);
size_t pp_params_bytes();
size_t pp_queue_bytes();
cudaError_t launch_pp_persistent_step(cudaStream_t st, const void *boxes, const int32_t *item_box,
                                      const int32_t *base, int n_items, unsigned *cost, int32_t *order, void *queue,
                                      const int *publish_host, int epoch, unsigned long long timeout_ns, int grid);
cudaError_t launch_vel_decode(cube2_ctx *ctx, const cube2_particles *p, float *const v[3]);
cudaError_t launch_kick(cube2_ctx *ctx, const cube2_particles *p, float kick);
cudaError_t launch_kick_drift(cube2_ctx *ctx, const cube2_particles *p, float kick, float drift_fix);
cudaError_t launch_scan(cube2_ctx *ctx, const int32_t *in, int32_t *out, int64_t n);
cudaError_t launch_rebin(cube2_ctx *ctx, const cube2_particles *p);
cudaError_t launch_place(cube2_ctx *ctx, const double *const pos[3], const float *const mom[3]);
int64_t scan_scratch_len(int64_t n);
// force vector-Jacobian product
cudaError_t launch_vjp_gather_e(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *const v[3],
                                float *const w[3]);
cudaError_t launch_vjp_gather_psi(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *const v[3],
                                  float *const w[3]);
cudaError_t launch_vjp_source(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *const v[3]);
cudaError_t launch_pp_vjp(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3], float *const w[3]);
cudaError_t launch_density_mse_vjp(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *target,
                                   float *const w[3], double *sq);
cudaError_t launch_density_vjp(cube2_ctx *ctx, Level &L, const cube2_particles *p, const float *g, float *const w[3]);
cudaError_t launch_kdk_adjoint_scatter(cube2_ctx *ctx, const int32_t *perm, float *const xbar[3],
                                       float *const pbar[3], const float *t, float k2);
cudaError_t launch_kdk_adjoint_drift(cube2_ctx *ctx, float *const xbar[3], float *const pbar[3], float drift);
cudaError_t launch_axpy3(cube2_ctx *ctx, float *const y[3], const float *t, float a);

}  // namespace cube2

// Device helpers ------------------------------------------------------------
namespace cube2 {

__device__ __forceinline__ void set_status(int *status, int bit) { atomicOr(status, bit); }

__device__ __forceinline__ int wrap(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

}  // namespace cube2
