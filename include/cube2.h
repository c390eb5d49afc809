/*
 * cube2.h -- C ABI of the GB300 (sm_103a) multi-level PM + PP gravity step.
 *
 * Method: CUBE2 (Yu et al., Sci. China PMA 2026), Sec. 2.1 (force
 * decomposition, optimised Green's function), Sec. 2.2 (kick/drift) and
 * Sec. 2.3 (Information Optimized Storage, IOS).  Every operation below runs
 * in hand-written CUDA kernels; nothing falls back to the CPU or to cuFFT.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Periodic comoving box of side L [Mpc/h] (Sec. 2, periodic boundary
 *   conditions).  Time variable is the scale factor a; H_0 = 1 units.
 * - IOS (Sec. 2.3): the box is cut into n_ios^3 cells (linear id
 *   c = (cz*n_ios + cy)*n_ios + cx, x fastest).  Particles are stored sorted by
 *   cell; particle p of cell c has uint16 in-cell offsets off[d][p] in units
 *   of 2^-16 cell, i.e. fixed-point coordinate X_d = c_d*2^16 + off_d.
 *   count[c] is the number of particles in cell c and start[c] its exclusive
 *   prefix sum, so the particles of c are [start[c], start[c]+count[c]).
 *   The IOS order doubles as the PP cell list.
 * - PM levels are numbered coarsest first.  Level l has an n_mesh[l]^3 mesh
 *   whose cell H_l = L/n_mesh[l] relates to the IOS cell by a power of two
 *   (n_ios/n_mesh[l] in {1/4, 1/2, 1, 2}); its softening is
 *   b_l = beta[l]*H_l and its truncation is b_{l-1} (infinity for l = 0),
 *   Eq. (force_decomp) and Eqs. (PM1)-(PM3).  The PP range is b_{last}
 *   (must not exceed the IOS cell), the PP softening b_pp, Eq. (PP).
 * - Force: acc = F = -grad u with lap u = delta (mean density one), in
 *   Mpc/h units; the PP pair term is V_p R_PP(r)/(4 pi) with V_p = L^3/N.
 * - Velocities are canonical momenta p = a^2 dx/dt.  dp/da = 1.5 Omega_m F /
 *   (a^2 E(a)),  dx/da = p / (a^3 E(a)),  E = sqrt(Omega_m a^-3 + Omega_L).
 *
 * Memory and streams
 * ------------------
 * All particle arrays are DEVICE pointers owned by the caller (for instance
 * torch tensors); the library never frees them.  cube2_init_mesh allocates
 * every buffer the context needs (meshes, Green's tables, FFT spectrum,
 * re-binning scratch) once; no later call allocates.  Every call enqueues
 * work on the stream given to cube2_init_mesh and returns without waiting,
 * except where stated.
 *
 * Errors
 * ------
 * Every call returns CUBE2_OK (0) or a negative CUBE2_ERR_* code and records
 * a message readable with cube2_last_error.  Argument errors are detected on
 * the host before any launch.  Errors found by kernels (uint64 deposit
 * overflow, non-finite forces, an IOS displacement that cannot be encoded)
 * set a sticky device status word; cube2_check synchronises the stream and
 * returns it.  After a device error the particle state is unspecified.
 */
#ifndef CUBE2_H
#define CUBE2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CUBE2_OK                    0
#define CUBE2_ERR_BAD_ARG          -1  /* null pointer, bad level, size mismatch   */
#define CUBE2_ERR_CUDA             -2  /* a CUDA runtime call failed               */
#define CUBE2_ERR_CAPACITY         -3  /* a uint64 deposit cell overflowed          */
#define CUBE2_ERR_TIMEOUT          -4  /* a bounded device wait ran out            */
#define CUBE2_ERR_NONFINITE        -5  /* NaN/Inf in a force or velocity           */
#define CUBE2_ERR_UNSUPPORTED_SIZE -6  /* mesh not 2^a 3^b, ratio not a power of 2 */
#define CUBE2_ERR_STATE            -7  /* call order violated (no table/density)   */
#define CUBE2_ERR_DISPLACEMENT     -8  /* drift moved a particle by >= n_ios/2     */

#define CUBE2_MAX_LEVELS 2

typedef struct cube2_ctx cube2_ctx;

/* Problem definition (host struct, copied by cube2_init_mesh). */
typedef struct {
    double  box;                       /* L [Mpc/h]                               */
    int32_t n_ios;                     /* IOS cells per dimension (>= 4)           */
    int32_t n_levels;                  /* number of PM levels, 1 or 2              */
    int32_t n_mesh[CUBE2_MAX_LEVELS];  /* mesh cells per dimension, coarsest first */
    double  beta[CUBE2_MAX_LEVELS];    /* softening in own mesh cells              */
    double  b_pp;                      /* PP softening [Mpc/h]                      */
    double  omega_m, omega_l;          /* flat LCDM density parameters             */
    int64_t n_particles;               /* particle count N (fixes V_p = L^3/N)     */
    int32_t alias_max;                 /* images per axis in Eq. (Gk); 2 in paper  */
    int32_t assign_order;              /* mass assignment: 2 (or 0) = CIC, exact
                                        * integer deposit; 3 = TSC (Eq. filter,
                                        * the paper's), FP32 accumulation      */
    double  iso_length;                /* 0 = periodic.  > 0: isolated boundary
                                        * conditions (Appendix A): the coarsest
                                        * level's reference force is truncated
                                        * at r = iso_length [Mpc/h] by Eq. isok,
                                        * R(k) times 1 - sinc(|k| iso_length) in
                                        * every alias image; at most box/2, so a
                                        * pair closer than iso_length - b_coarse
                                        * feels no periodic image             */
    /* Adaptive third PM level (Sec. 2.1.1 Eq. PM3, Sec. 2.2.3), CIC only.
     * pm3_tile = 0 switches it off (the fields below are then ignored).  The
     * box is cut into subtiles of pm3_tile^3 IOS cells (pm3_tile divides
     * n_ios); a subtile whose densest IOS cell holds >= pm3_rho_min particles
     * gets a local periodic mesh of spacing H_3 = H_finest / pm3_refine over
     * the subtile plus a buffer of B = ceil(b_finest / H_3) + 4 cells on each
     * side (m = the smallest 2^a 3^b >= pm3_tile s_ios / H_3 + 2 B cells, which
     * must be a supported mesh size of at most 256), softening b_3 = pm3_beta H_3 and the
     * kernel R(r, b_3) - R(r, b_finest); its own particles get that force and
     * a PP range of b_3 instead of b_finest.  pm3_refine: a power of two with
     * H_3 <= s_ios; b_pp < b_3 < b_finest.  At most pm3_max_tiles subtiles are
     * refined per force evaluation (the first in subtile order, x fastest);
     * the rest keep the two-level method.  The capacity actually allocated is
     * min(pm3_max_tiles, subtiles, 65535) (cube2_pm3_info reports it).        */
    int32_t pm3_tile;
    int32_t pm3_refine;
    double  pm3_beta;
    int32_t pm3_rho_min;
    int32_t pm3_max_tiles;
    /* 1: the particle sets this context steps store their velocities as FP16
     * with a per-IOS-cell FP32 scale (cube2_particles.vel16 / vscale, the
     * compressed velocity storage of Sec. 2.3); the context then holds one
     * FP32 working copy of them (12 bytes per particle) for the step.  0: FP32
     * velocities (cube2_particles.vel).                                       */
    int32_t vel_fp16;
} cube2_config;

/* Level index of the adaptive third level in cube2_set_green / cube2_get_green. */
#define CUBE2_LEVEL_PM3 2

/* Particle set in IOS form; every pointer is a device pointer (see above). */
typedef struct {
    int64_t   n;          /* number of particles, must equal cfg.n_particles      */
    uint16_t *off[3];     /* [3][n] in-cell offsets, SoA, sorted by IOS cell      */
    int32_t  *count;      /* [n_ios^3] particles per IOS cell                      */
    int32_t  *start;      /* [n_ios^3] exclusive prefix sum of count               */
    float    *vel[3];     /* [3][n] canonical momenta (FP32)                       */
    float    *acc[3];     /* [3][n] force F = -grad u (FP32, output of force calls) */
    /* FP16 velocity storage (contexts with cfg.vel_fp16 = 1; NULL otherwise,
     * and vel is then unused): the momentum of particle p is
     * v_d = half(vel16[d][p]) * vscale[c], c its IOS cell, with
     * vscale[c] = max over the cell's particles and d of |v_d| (FP32) and
     * vel16 = RN_half(RN32(v_d / vscale[c])) (0 where vscale[c] = 0).
     * vel16: [3][n] IEEE binary16 bit patterns; vscale: [n_ios^3] FP32.     */
    uint16_t *vel16[3];
    float    *vscale;
} cube2_particles;

/* Validate cfg, allocate the context and all device buffers, and build the
 * FFT twiddle tables.  stream is a cudaStream_t (NULL = legacy default).
 * The context is bound to the device current at this call.  Returns
 * CUBE2_ERR_UNSUPPORTED_SIZE for meshes outside 2^a 3^b in [8, 2048] or level
 * ratios that are not powers of two, CUBE2_ERR_BAD_ARG for other bad fields,
 * CUBE2_ERR_CUDA if an allocation fails (nothing is leaked). */
int cube2_init_mesh(cube2_ctx **ctx, const cube2_config *cfg, void *stream);

/* Eq. (Gk) with Eqs. (Rk), (Sk), (diff) and the assignment's W(k) =
 * prod sinc^p(k_d/2) (p = 2 CIC, 3 TSC), alias sum over |n_d| <= alias_max, evaluated in FP64 on the GPU for level
 * `level` with the inverse-FFT factor 1/n^3 folded in, G = 0 where |D(k)| = 0.
 * G is even in each k_d and symmetric under axis permutations, so it is
 * computed and stored once per sorted triple 0 <= a <= b <= c <= n/2 of
 * |m_x|, |m_y|, |m_z| (entry c(c+1)(c+2)/6 + b(b+1)/2 + a, FP32,
 * (n/2+1)(n/2+2)(n/2+3)/6 entries: 11 MB at n = 512, 0.7 GB at n = 2048);
 * cube2_get_green expands it.  For n <= 1024 the context also keeps the same
 * entries folded in k_y and k_z only ([n/2+1][n/2+1][n/2+1 padded to a
 * multiple of 16], 72 MB at n = 512), built here from the reduced table, which
 * the z pass reads with plain indices; larger meshes look up the reduced
 * table directly.
 * With cfg.iso_length > 0 the coarsest level's images are weighted by
 * 1 - sinc(|k_n| iso_length) (Eq. isok, isolated boundary conditions).
 * cache_path (optional, may be NULL) names a file: if it holds a table for
 * the same (n, b_soft, b_trunc, alias, order, iso) in the reduced layout it is read instead of computed,
 * otherwise the computed table is written there (Sec. 2.1.2: tables may be
 * stored as files).  Synchronises the stream when a file is used. */
int cube2_set_green(cube2_ctx *ctx, int level, const char *cache_path);

/* The adaptive third level (cfg.pm3_tile > 0) is part of cube2_force and
 * cube2_kdk_step once its table is built: cube2_set_green(ctx,
 * CUBE2_LEVEL_PM3, path) evaluates Eq. (Gk) for the local m^3 mesh with
 * softening pm3_beta and truncation b_finest / H_3 (local cells).  Each force
 * evaluation then builds the refinement map from the counts, deposits the
 * refined subtiles' local boxes (exact integer CIC, FP32 density
 * V_p / H_3^3 sum W), solves all local meshes in one batch of FFT passes,
 * adds -H_3 (D * phi) gathered at each refined subtile's own particles to acc
 * and runs PP with the per-target range.  cube2_pp_force alone uses the map
 * of the counts it is given as well.  The adjoint entry points reject a
 * context with the third level (CUBE2_ERR_STATE).
 *
 * cube2_pm3_info: out = {pm3_tile, subtiles per dimension, refinement r,
 * buffer B, mesh m, H_3 [Mpc/h], b_3 [Mpc/h], local mesh capacity} (host only;
 * CUBE2_ERR_STATE when the third level is off).
 * cube2_pm3_stats: synchronises; out = {local meshes in use, subtiles that
 * asked for refinement} of the last force or PP call.
 * cube2_pm3_map: out (device int32 [subtiles^3], x fastest) = the local mesh
 * index of each subtile in the last force or PP call, -1 where unrefined. */
int cube2_pm3_info(cube2_ctx *ctx, double out[8]);
int cube2_pm3_stats(cube2_ctx *ctx, int64_t out[2]);
int cube2_pm3_map(cube2_ctx *ctx, int32_t *out);

/* CIC mass assignment (Eq. filter, CIC reading) of the particles onto level
 * `level` (or every level in one particle pass when level = -1).  Integer
 * fixed point: 1-D weights are exact integers at scale 2^16 of the mesh cell,
 * the 3-D weight their product, accumulated as uint64 in shared-memory tiles
 * (exact, so the result does not depend on order).  The internal FP32 grid is
 * RN32(acc - M) * RN32(n^3/N * 2^-48) with M = floor(N 2^48 / n^3): the
 * overdensity in mean-one units.  A uint64 wrap sets CUBE2_ERR_CAPACITY. */
int cube2_deposit(cube2_ctx *ctx, int level, const cube2_particles *p);

/* Test access: the exact uint64 accumulator of `level` for particles p,
 * written to out ([n][n][n] uint64, device, x fastest).  Same kernel as
 * cube2_deposit with an integer epilogue. */
int cube2_deposit_u64(cube2_ctx *ctx, int level, const cube2_particles *p, uint64_t *out);

/* Poisson solve of level `level` (Sec. 2.1.2): forward 3-D r2c FFT of the
 * deposited grid (batched radix line passes along x, y, z), multiplication
 * by G on the last forward pass, inverse 3-D c2r FFT.  Leaves phi (mesh
 * units, lap phi = rho) in the level's real grid.  Needs cube2_set_green and
 * cube2_deposit for that level first (else CUBE2_ERR_STATE). */
int cube2_solve_pm(cube2_ctx *ctx, int level);

/* Force interpolation (Sec. 2.1.2): E = D * phi with the 4-point difference
 * of Eq. (diff) evaluated on the fly, gathered with the deposit's CIC
 * weights, scaled to F = -H_l E.  level = -1 sums every level in one
 * particle pass.  accumulate = 0 overwrites acc, 1 adds to it. */
int cube2_interp_force(cube2_ctx *ctx, int level, const cube2_particles *p, int accumulate);

/* PP force (Sec. 2.2.3, Eq. PP): for all pairs closer than the PP range,
 * F_i += V_p (R(r,b_pp) - R(r,b_range))/(4 pi) (x_j - x_i)/r, separations
 * formed exactly in fixed point over the 27 neighbouring IOS cells, FP32
 * sums with Kahan compensation.  accumulate as above. */
int cube2_pp_force(cube2_ctx *ctx, const cube2_particles *p, int accumulate);

/* Full force: deposit every level, solve every level, interpolate, PP.
 * Writes acc = F.  Requires every level's Green's table. */
int cube2_force(cube2_ctx *ctx, const cube2_particles *p);

/* One kick-drift-kick step a0 -> a1 (Secs. 2.2.3, 2.3, 3.2): requires acc
 * to hold F at the current positions (from cube2_force or the previous step).
 * p += 1.5 Om K(a0,ah) acc; X += rint(p Dr(a0,a1) 2^16/s_ios) mod n_ios 2^16
 * (round half even); stable re-bin by new cell (ties keep the old order),
 * rewriting off, count, start, vel in place; acc = F(new positions);
 * p += 1.5 Om K(ah,a1) acc, with ah = (a0+a1)/2 and K, Dr Gauss-Legendre
 * integrals of 1/(a^2 E) and 1/(a^3 E). */
int cube2_kdk_step(cube2_ctx *ctx, cube2_particles *p, double a0, double a1);

/* The same step for a particle set held in HOST memory (pinned for speed):
 * copies host -> dev (off, count, vel, acc; host->start is not read: the
 * device forms it from count, of which it is the exclusive prefix sum in the
 * IOS layout), runs cube2_kdk_step on dev, copies dev -> host (off, count,
 * start, vel, acc), then synchronises.  Offsets, counts and starts
 * are final after the re-bin; their download runs on a second stream of the
 * context while the forces are computed. */
int cube2_kdk_step_host(cube2_ctx *ctx, cube2_particles *dev, cube2_particles *host,
                        double a0, double a1);

/* Information Optimized Storage from arbitrary positions (Sec. 2.3: a particle
 * is its cell, given by its place in the cell-sorted order and the per-cell
 * counts, plus uint16 offsets inside the cell).  pos: three device FP64 [N]
 * arrays of comoving positions [Mpc/h], any real values (wrapped into the
 * periodic box); mom: three device FP32 [N] momentum arrays, or NULL for
 * zero momenta.  X_d = rint(x_d / s_ios * 2^16) mod n_ios 2^16 (FP64, round
 * half to even), cell = floor(X/2^16), offset = X mod 2^16; particles are
 * stably sorted by cell (ties keep the input order).  Writes p->off, p->vel,
 * p->count, p->start (p->acc untouched) and, when perm is not NULL, perm[j] =
 * the input index of IOS slot j (device int32 [N]).  Non-finite or enormous
 * positions set CUBE2_ERR_NONFINITE in the sticky status (cube2_check).  The
 * entry of a differentiable run: gradients in IOS order map back through perm. */
int cube2_ios_from_positions(cube2_ctx *ctx, const double *const pos[3], const float *const mom[3],
                             cube2_particles *p, int32_t *perm);

/* Test/diagnostic copies of internal grids into caller device buffers:
 * density after cube2_deposit, potential after cube2_solve_pm ([n][n][n]
 * FP32), Green's table (expanded from the reduced layout to [n][n][n/2+1]
 * FP32, including the 1/n^3 factor). */
int cube2_get_density(cube2_ctx *ctx, int level, float *out);
int cube2_get_potential(cube2_ctx *ctx, int level, float *out);
int cube2_get_green(cube2_ctx *ctx, int level, float *out);

/* Forward r2c FFT of the deposited grid only, written to out as interleaved
 * complex FP32 [n][n][n/2+1] (unnormalised, numpy.fft.rfftn convention). */
int cube2_debug_forward_fft(cube2_ctx *ctx, int level, float *out);

/* Allocation-free Poisson solve, without a context.  The paper has no
 * counterpart: it is for callers that cannot allocate device memory where
 * they need a solve (a fixed device-memory budget owned by the host
 * application, or code that must not let cudaMalloc/cudaFree synchronise the
 * device).  rho: device FP32 [n][n][n] overdensity (as cube2_get_density
 * gives); green: device FP32 [n][n][n/2+1] table with 1/n^3 folded in (as
 * cube2_get_green gives); phi: device FP32 [n][n][n] output, all on the
 * current device.  The same FFT passes as cube2_solve_pm, with the Green's
 * table read from the caller's full half-spectrum layout instead of the
 * context's symmetry-reduced one: the same result up to FP32 rounding.
 * Working memory is one file-scope device array of 15.7 MB that every GPU
 * loading the library holds until exit; n must be a supported size no larger
 * than 128 (else CUBE2_ERR_UNSUPPORTED_SIZE, message in
 * cube2_last_error(NULL)).  The first call on a device looks up that array's
 * address (cudaGetSymbolAddress) with the device current and keeps it for the
 * life of the process; make that first call before any stream capture, and
 * do not call this entry point on a device after cudaDeviceReset.  All calls
 * share the array and keep the last call's contents, so calls that overlap
 * on the GPU (different streams or threads without ordering) race.  No
 * allocation takes place. */
int cube2_solve_pm_noalloc(const float *rho, const float *green, float *phi, int32_t n, void *stream);

/* FP32 pipe probe (the ceiling of the PP force, Sec. 2.2.3 / Eq. PP, which is
 * plain FP32 arithmetic): launches blocks x threads threads (threads a
 * multiple of 32, at most 1024), each running 8 independent chains of 16 * iters
 * dependent FMAs, on `stream` (a cudaStream_t).  The work is
 * 2 * 8 * 16 * iters * blocks * threads FP32 operations; the caller times the
 * launch (CUDA events) to obtain the device's FMA rate.  out: one device
 * float, never written in practice (it keeps the chains from being removed).
 * Returns CUBE2_ERR_BAD_ARG for bad sizes, CUBE2_ERR_CUDA if the launch fails. */
int cube2_fma_probe(float *out, int blocks, int threads, int iters, void *stream);

/* FP16 velocity codec (contexts with cfg.vel_fp16 = 1).  cube2_vel_encode:
 * p->vel16 and p->vscale from FP32 momenta v[3] (device [N] each, in p's
 * particle order; counts and starts of p give the cells).
 * cube2_vel_decode: v[3] (device FP32 [N] each) = half(vel16) * vscale.
 * In a step the kick decodes, the re-bin gathers FP32 momenta into the
 * context's working copy, the second kick updates it and the step ends by
 * encoding it into p->vel16 / p->vscale.  cube2_kdk_step_host,
 * cube2_ios_from_positions and the adjoint take FP32 velocities only
 * (CUBE2_ERR_BAD_ARG / CUBE2_ERR_STATE for a vel_fp16 context). */
int cube2_vel_encode(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3]);
int cube2_vel_decode(cube2_ctx *ctx, const cube2_particles *p, float *const v[3]);

/* Host helper: out = {K(a0,ah), Dr(a0,a1), K(ah,a1)} for cfg's cosmology. */
int cube2_kdk_factors(const cube2_config *cfg, double a0, double a1, double out[3]);

/* Synchronise the context stream, then return the sticky device status
 * (CUBE2_OK or the first kernel-detected CUBE2_ERR_*), clearing it. */
int cube2_check(cube2_ctx *ctx);

/* Message of the last error recorded on ctx ("" if none); NULL ctx gives
 * the message of the last failed cube2_init_mesh or cube2_solve_pm_noalloc
 * on the calling thread. */
const char *cube2_last_error(cube2_ctx *ctx);

/* Optional per-kernel-class timing with CUDA events on the context stream.
 * cube2_profile(ctx, cap) discards earlier records and, for cap > 0, records
 * a start/stop event pair around each launch group of the later calls (up to
 * cap groups; cap = 0 switches profiling off).  cube2_profile_read
 * synchronises, writes the summed milliseconds and group counts per
 * (class, level) into ms[class * CUBE2_MAX_LEVELS + level] and
 * counts[...] (arrays of CUBE2_PROFILE_CLASSES * CUBE2_MAX_LEVELS), clears the
 * records, and returns CUBE2_ERR_CAPACITY if the pool overflowed.  Class
 * names: cube2_profile_class_name. */
#define CUBE2_PROFILE_CLASSES 27
int cube2_profile(cube2_ctx *ctx, int cap);
int cube2_profile_read(cube2_ctx *ctx, double *ms, int64_t *counts);
const char *cube2_profile_class_name(int cls);

/* PP work counters.  cube2_pp_count(ctx, 1) switches counting on for the
 * context's later PP evaluations (force, pp_force, steps; not the ensemble's
 * persistent kernel), 0 off (the default: the counters cost PP time).
 * cube2_pp_stats: the counts accumulated while counting was on, since the
 * last call: out[0] = ordered pairs closer than the PP range that were
 * evaluated, out[1] = candidate pairs tested (per target: the shared source
 * stream of its warp where the warp has one, else the particles of its 27
 * cells).  Synchronises the stream and resets the counters. */
int cube2_pp_count(cube2_ctx *ctx, int on);
int cube2_pp_stats(cube2_ctx *ctx, int64_t out[2]);

/* The same counters split by path: out[0..1] = (pairs, candidates) of all
 * targets as above, out[2..3] = those of the targets whose warp walked its
 * own 27 cells per lane (no shared stream).  Synchronises and resets. */
int cube2_pp_stats_paths(cube2_ctx *ctx, int64_t out[4]);

/* Number of kernel launches this context has issued (for launch accounting). */
int64_t cube2_launch_count(cube2_ctx *ctx);

/* Free every buffer the context owns.  Synchronises its stream first. */
void cube2_destroy(cube2_ctx *ctx);

/* ---- Adjoint: vector-Jacobian product of the force -----------------------
 * The force of Secs. 2.1-2.2 (every PM level plus PP) as a function of the
 * particle positions x (Mpc/h), with the IOS quantisation of Sec. 2.3 taken
 * as the identity (the CIC weights and their gradients are those of the
 * stored positions).  For a cotangent v the product is
 * w_i = d<v, F(x)>/dx_i: per PM level, -sum_c grad W(u_i,c) (E(c).v_i) +
 * sum_c grad W(u_i,c) psi(c) with psi = G * (n^3/N) sum_d D_d * mu_d and mu_d
 * the CIC deposit of v_d (G even, D_d odd); for PP,
 * sum_j (g I + g'/r d d^T)(v_j - v_i), g = V_p R_PP(r)/(4 pi r). */

/* Allocate the adjoint's scratch (three FP32 meshes of the largest level,
 * 15 FP32 values per particle).  The one allocating call after
 * cube2_init_mesh; idempotent. */
int cube2_adjoint_init(cube2_ctx *ctx);

/* w[d] (device FP32 [N], overwritten) = the product for cotangent v[d]
 * (device FP32 [N]), both in the particle order of p.  Needs
 * cube2_adjoint_init and every level's Green's table (CUBE2_ERR_STATE).
 * Overwrites the levels' density/potential grids.  The cotangent deposit
 * uses float atomics: results agree with the FP64 product to FP32 accuracy
 * but their last bits may differ between runs. */
int cube2_force_vjp(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3], float *const w[3]);

/* out (device int32 [N]) = the particle map of the last cube2_kdk_step's
 * re-bin: out[new index] = index before the re-bin (the adjoint of a step
 * needs it to carry adjoints back to the earlier order). */
int cube2_kdk_permutation(cube2_ctx *ctx, int32_t *out);

/* Loss of a final density against a target and its gradient in the
 * positions: L = (1/n^3) sum_c (delta(c) - target(c))^2 on level `level`,
 * delta the FP32 overdensity cube2_deposit computes, target device FP32
 * [n][n][n]; w[d] (device FP32 [N], overwritten) = dL/dx_i (Mpc/h^-1) =
 * (n^3/(N H)) sum_c grad_u W(u_i, c) 2 (delta - target)(c)/n^3.  *loss on the
 * host; synchronises.  Needs cube2_adjoint_init.  Overwrites the level's
 * density grid. */
int cube2_density_mse_vjp(cube2_ctx *ctx, int level, const cube2_particles *p, const float *target,
                          float *const w[3], double *loss);

/* Position gradient of <g, delta> for a cotangent g on the density of level
 * `level` (device FP32 [n][n][n], the layout of cube2_get_density): w[d]
 * (device FP32 [N], overwritten) = d<g, delta>/dx_i = (n^3/(N H)) sum_c
 * g(c) grad_u W(u_i, c), with delta the CIC overdensity cube2_deposit
 * computes (Sec. 2.1.2 assignment; IOS quantisation taken as the identity).
 * The entry of a backward pass through the final density: the cotangent
 * arrives as it is, with no loss of its own.  Overwrites the level's grid. */
int cube2_density_vjp(cube2_ctx *ctx, int level, const cube2_particles *p, const float *g, float *const w[3]);

/* Reverse of one cube2_kdk_step(a0, a1) (Sec. 2.2: kick K(a0, ah), drift
 * Dr(a0, a1), force, kick K(ah, a1); drift rounding taken as the identity).
 * pre / post: the particle states before and after the step (positions,
 * counts and starts are read); perm: its cube2_kdk_permutation.  On entry
 * xbar, pbar (device FP32 [N] each) hold dL/dx and dL/dv after the step in
 * post's order; on return they hold them before the step in pre's order:
 * xbar += k2 F'(post)^T pbar; back through the re-bin; pbar += Dr xbar;
 * xbar += k1 F'(pre)^T pbar, with k = 1.5 Omega_m K and the force products of
 * cube2_force_vjp.  Needs cube2_adjoint_init. */
int cube2_kdk_adjoint_step(cube2_ctx *ctx, const cube2_particles *pre, const cube2_particles *post,
                           const int32_t *perm, float *const xbar[3], float *const pbar[3], double a0, double a1);

/* Reverse of n_steps consecutive cube2_kdk_step calls over the schedule
 * a[0..n_steps]: states[0..n_steps] the checkpoints (before the first step,
 * after each step), perms[k] the re-bin map of step k.  xbar, pbar: as in
 * cube2_kdk_adjoint_step, in the last state's order on entry and the first
 * state's on return.  Same result as cube2_kdk_adjoint_step applied from the
 * last step back, with one force product per step instead of two: the
 * product that ends the reverse of step k+1 (at state k+1, with the pbar the
 * reverse of step k starts from) is the one step k needs first. */
int cube2_kdk_adjoint(cube2_ctx *ctx, const cube2_particles *const *states, const int32_t *const *perms, int n_steps,
                      const double *a, float *const xbar[3], float *const pbar[3]);

/* ---- Ensembles of independent boxes -------------------------------------
 * Many small simulations on one GPU, and their split over GPUs.  Placement
 * follows the load balancing of paper Sec. 2.2.3 (Fig. balance): tasks in
 * decreasing cost order, each to the least loaded worker. */

/* Longest-processing-time-first placement: sort the n costs (finite, >= 0)
 * in decreasing order (ties keep index order) and give each, in that order,
 * to the bin with the smallest load so far (lowest index on ties).  Writes
 * bin_of[i] in [0, bins).  Host only; CUBE2_ERR_BAD_ARG on bad input. */
int cube2_lpt_partition(const double *cost, int n, int bins, int *bin_of);

/* Work estimate of one KDK step of a box with configuration cfg (arbitrary
 * units): FFT n^3 log2(n^3) over every PM level plus 64 per particle
 * (cfg->n_particles).  Host only, no device needed. */
int cube2_config_cost(const cube2_config *cfg, double *cost);

typedef struct cube2_ensemble cube2_ensemble;

/* Record n_steps KDK steps of each of n_boxes boxes into one CUDA graph.
 * ctxs[b] / parts[b]: a distinct context and its particle set, on one device,
 * with current forces (cube2_force, or a previous step) and profiling off.
 * a: [n_boxes][n_steps + 1] row-major scale factors, increasing per box.
 * Boxes go to min(n_streams, n_boxes) concurrent graph branches by
 * cube2_lpt_partition of cube2_config_cost (1 <= n_streams <= 64); a branch runs
 * its boxes one after another, largest first.  Synchronises every box's
 * stream, then records; no kernel runs until cube2_ensemble_launch.  On
 * failure nothing is kept and *out is NULL. */
int cube2_ensemble_create(cube2_ensemble **out, cube2_ctx *const *ctxs, cube2_particles *const *parts,
                          int n_boxes, const double *a, int n_steps, int n_streams);

/* Options of an ensemble recording.
 *   n_streams       concurrent graph branches (1..64); boxes are placed on them
 *                   by cube2_lpt_partition of cube2_config_cost
 *   persistent_pp   0: every box's steps are its own launches on its branch
 *                   (one join at the end).  1: step by step, each box's step
 *                   up to its PP inputs on its branch, then ONE persistent PP
 *                   kernel (with the second kick) over every box: its CTAs take
 *                   (box, block of 128 targets) items from a device queue,
 *                   ordered each step by a cost estimate (the particles in the
 *                   targets' IOS cells; largest first, the load balancing of
 *                   Sec. 2.2.3).  The host publishes each step's queue by a
 *                   stream-ordered write of the step's epoch from pinned
 *                   memory; the kernel waits for it at most timeout_ms
 *                   (%globaltimer) and otherwise records CUBE2_ERR_TIMEOUT
 *                   (cube2_ensemble_check) and returns.  Boxes with the third
 *                   level or FP16 velocities are refused (CUBE2_ERR_STATE).
 *   pp_ctas_per_sm  persistent grid: CTAs per SM (1..16)
 *   pp_wmax         PP shared-stream width for every box (0: each context's own, 16)
 *   timeout_ms      bound of the persistent kernel's wait (> 0)                  */
typedef struct {
    int32_t n_streams;
    int32_t persistent_pp;
    int32_t pp_ctas_per_sm;
    int32_t pp_wmax;
    double  timeout_ms;
} cube2_ensemble_opts;

/* cube2_ensemble_create with options (cube2_ensemble_create is this with
 * persistent_pp = 0, pp_wmax = 0). */
int cube2_ensemble_create_ex(cube2_ensemble **out, cube2_ctx *const *ctxs, cube2_particles *const *parts,
                             int n_boxes, const double *a, int n_steps, const cube2_ensemble_opts *opts);

/* Synchronise `stream` and return CUBE2_ERR_TIMEOUT (clearing it) if a
 * persistent PP kernel of the last launches gave up waiting for its queue;
 * the boxes' states are then unspecified.  CUBE2_OK otherwise. */
int cube2_ensemble_check(cube2_ensemble *ens, void *stream);

/* Host control of the persistent kernel's queue publication: on = 0 makes the
 * later launches write no valid epoch (the host withholds the work counts), so
 * that each persistent kernel's bounded wait runs out; on = 1 restores it.
 * This is how a lost host publication is detected without any GPU fault. */
int cube2_ensemble_publish(cube2_ensemble *ens, int on);

/* Autotuner of the runtime knobs: starting from *best (persistent_pp and
 * timeout_ms kept), a coordinate search over pp_ctas_per_sm in {4, 8, 16}
 * (persistent only), pp_wmax in {8, 16, 24} and n_streams in {8, 16, 32}; each
 * candidate is recorded and timed with CUDA events on `stream` (the fastest of
 * `trials` launches after one warm-up launch), every launch starting from the
 * boxes' states at the call (snapshotted in scratch that this call allocates
 * and frees; states restored at the end).  Writes the fastest options to *best
 * and their milliseconds per launch to *best_ms. */
int cube2_ensemble_autotune(cube2_ctx *const *ctxs, cube2_particles *const *parts, int n_boxes, const double *a,
                            int n_steps, int trials, void *stream, cube2_ensemble_opts *best, double *best_ms);

/* Run the recorded steps once on `stream` (a cudaStream_t; NULL = default
 * stream).  Each launch advances every box by its n_steps from whatever state
 * its particle arrays hold.  Synchronise `stream` before reading results or
 * calling cube2_check on a box. */
int cube2_ensemble_launch(cube2_ensemble *ens, void *stream);

/* out[0] = kernel nodes in the graph, out[1] = particle-steps per launch. */
int cube2_ensemble_info(const cube2_ensemble *ens, int64_t out[2]);

/* Wait for the graph's last launch on its streams and free it. */
void cube2_ensemble_destroy(cube2_ensemble *ens);

#ifdef __cplusplus
}
#endif
#endif /* CUBE2_H */
