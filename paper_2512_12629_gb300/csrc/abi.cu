// C ABI entry points of libcube2gb (declared in include/cube2.h): argument
// validation, buffer ownership, stream ordering and the host-side scalars of
// the kick-drift-kick step.  All particle and mesh arithmetic runs in the
// kernels of deposit.cu, fft.cu, green.cu, interp.cu, pp.cu and kdk.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"

#include <algorithm>

namespace cube2 {
bool fft_size_supported(int n);

int set_error(cube2_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int prof_begin(cube2_ctx *ctx, int cls, int level) {
    if (!ctx->prof || cls < 0) return -1;
    if (ctx->prof_used >= ctx->prof_cap) { ctx->prof_overflow = 1; return -1; }
    const int slot = ctx->prof_used++;
    ctx->prof_cls[slot] = cls * CUBE2_MAX_LEVELS + level;
    cudaEventRecord(ctx->ev[2 * slot], ctx->stream);
    return slot;
}

void prof_end(cube2_ctx *ctx, int slot) {
    if (slot >= 0) cudaEventRecord(ctx->ev[2 * slot + 1], ctx->stream);
}

namespace {
thread_local std::string g_init_error;
}

void set_context_free_error(const std::string &msg) { g_init_error = msg; }

int cuda_error(cube2_ctx *ctx, cudaError_t e, const char *what) {
    return set_error(ctx, CUBE2_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

double integrate(double a0, double a1, double om, double ol, int power) {
    static std::vector<double> gx, gw;
    if (gx.empty()) gauss_legendre(48, gx, gw);
    const double mid = 0.5 * (a0 + a1), half = 0.5 * (a1 - a0);
    double s = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
        const double a = mid + half * gx[i];
        const double e = sqrt(om / (a * a * a) + ol);
        s += gw[i] / (pow(a, power) * e);
    }
    return half * s;
}

int ilog2_ratio(int big, int small) {
    if (small <= 0 || big % small) return -100;
    int q = big / small, s = 0;
    while ((1 << s) < q) ++s;
    return (1 << s) == q ? s : -100;
}

int level_shift(int n_ios, int n) {
    if (n_ios >= n) return ilog2_ratio(n_ios, n);
    const int s = ilog2_ratio(n, n_ios);
    return s == -100 ? -100 : -s;
}

void prof_free(cube2_ctx *c) {
    if (c->ev) {
        for (int i = 0; i < 2 * c->prof_cap; ++i) cudaEventDestroy(c->ev[i]);
        delete[] c->ev;
        delete[] c->prof_cls;
    }
    c->ev = nullptr;
    c->prof_cls = nullptr;
    c->prof_cap = c->prof_used = 0;
    c->prof = false;
}

void free_ctx(cube2_ctx *c) {
    if (!c) return;
    prof_free(c);
    for (int l = 0; l < CUBE2_MAX_LEVELS; ++l) {
        cudaFree(c->lev[l].real);
        cudaFree(c->lev[l].spec);
        cudaFree(c->lev[l].green);
        cudaFree(c->lev[l].green2);
        cudaFree(c->lev[l].tw);
    }
    cudaFree(c->cellid);
    cudaFree(c->toff);
    cudaFree(c->tvel);
    cudaFree(c->tcell);
    cudaFree(c->tslot);
    cudaFree(c->perm);
    cudaFree(c->scan_tmp);
    cudaFree(c->ncount);
    cudaFree(c->nstart);
    cudaFree(c->perm2);
    cudaFree(c->big);
    cudaFree(c->big_n);
    cudaFree(c->pos4);
    cudaFree(c->pp_perm);
    cudaFree(c->vjp_mu);
    cudaFree(c->vjp_t);
    cudaFree(c->vjp_u);
    cudaFree(c->vjp_sq);
    cudaFree(c->pp_stats);
    cudaFree(c->pm3.lev.real);
    cudaFree(c->pm3.lev.spec);
    cudaFree(c->pm3.lev.green);
    cudaFree(c->pm3.lev.tw);
    cudaFree(c->pm3.rho_max);
    cudaFree(c->pm3.slot);
    cudaFree(c->pm3.list);
    cudaFree(c->pm3.count);
    cudaFree(c->vel32);
    cudaFree(c->dev_status);
    cudaFreeHost(c->host_status);
    if (c->aux_event) cudaEventDestroy(c->aux_event);
    if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
    delete c;
}

bool particles_ok(cube2_ctx *ctx, const cube2_particles *p, bool need_vel, bool need_acc) {
    if (!p) return false;
    if (p->n != ctx->N) return false;
    if (ctx->N == 0) return p->count && p->start;
    for (int d = 0; d < 3; ++d) {
        if (!p->off[d]) return false;
        // a vel_fp16 context steps FP16 velocities with their per-cell scale
        if (need_vel && (ctx->vel32 ? !p->vel16[d] : !p->vel[d])) return false;
        if (need_acc && !p->acc[d]) return false;
    }
    if (need_vel && ctx->vel32 && !p->vscale) return false;
    return p->count && p->start;
}

int level_ok(cube2_ctx *ctx, int level, bool allow_all) {
    if (allow_all && level == -1) return CUBE2_OK;
    if (level < 0 || level >= ctx->nl) return set_error(ctx, CUBE2_ERR_BAD_ARG, "level out of range");
    return CUBE2_OK;
}

// Geometry of the adaptive third level from the config (after the global
// levels are set up).  Returns "" when valid, else 'U' (unsupported size) or
// 'B' (bad argument) followed by the message.
std::string pm3_geometry(cube2_ctx *c) {
    const cube2_config *cfg = &c->cfg;
    PM3 &M = c->pm3;
    const Level &F = c->lev[c->nl - 1];
    if (c->cfg.assign_order != 2) return "Bthe adaptive third level uses CIC assignment";
    if (c->n_ios % cfg->pm3_tile) return "Bpm3_tile must divide n_ios";
    const int r = cfg->pm3_refine;
    if (r < 1 || (r & (r - 1))) return "Bpm3_refine must be a power of two";
    int lr = 0;
    while ((1 << lr) < r) ++lr;
    // H_finest / s_ios = n_ios / n_finest = 2^F.shift, so H_3 / s_ios = 2^-(lr - F.shift)
    const int q_shift = lr - F.shift;
    if (q_shift < 0 || q_shift > 12) return "Bthe third level's cell must be at most the IOS cell (and >= 2^-12 of it)";
    if (cfg->pm3_rho_min < 1 || cfg->pm3_max_tiles < 1) return "Bpm3_rho_min and pm3_max_tiles must be positive";
    M.T = cfg->pm3_tile;
    M.ns = c->n_ios / M.T;
    M.n_sub = (int64_t)M.ns * M.ns * M.ns;
    M.r = r;
    M.q_shift = q_shift;
    M.rho_min = cfg->pm3_rho_min;
    // more slots than subtiles would never be filled; the slot is a grid dimension
    M.max_tiles = (int)std::min<int64_t>(std::min<int64_t>(cfg->pm3_max_tiles, M.n_sub), 65535);
    M.H = F.H / r;
    M.b3 = cfg->pm3_beta * M.H;
    if (!(M.b3 < c->b_range) || !(M.b3 > cfg->b_pp)) return "Bthe third level's softening must lie between b_pp and the PP range";
    M.B = (int)ceil(c->b_range / M.H - 1e-12) + 4;
    const int64_t need = ((int64_t)M.T << q_shift) + 2 * M.B;
    int64_t best = -1;
    for (int64_t a = 1; a <= (int64_t)1 << 20; a *= 2)
        for (int64_t v = a; v <= (int64_t)1 << 22; v *= 3)
            if (v >= need && (best < 0 || v < best)) best = v;
    if (best < 0 || best > 256 || !fft_size_supported((int)best))
        return "Uthe third level's local mesh size is not supported (batched local meshes go up to 256)";
    M.m = (int)best;
    if (M.m * M.H > cfg->box * (1.0 + 1e-12)) return "Bthe third level's local box exceeds the simulation box";
    const int64_t m3 = (int64_t)M.m * M.m * M.m;
    if ((int64_t)M.max_tiles * m3 > ((int64_t)1 << 31) * 8) return "Bpm3_max_tiles x local mesh too large";
    Level &L = M.lev;
    L.index = 0;
    L.n = M.m;
    L.kxp = ((L.n / 2 + 1) + 15) / 16 * 16;
    L.H = M.H;
    L.b_soft = cfg->pm3_beta;
    L.b_trunc = c->b_range / M.H;
    L.iso = 0.0;
    L.batch = M.max_tiles;
    const double vp = cfg->box * cfg->box * cfg->box / (double)(c->N > 0 ? c->N : 1);
    M.dens_scale = (float)(vp / (M.H * M.H * M.H) * ldexp(1.0, -48));
    M.on = true;
    return "";
}

}  // namespace
}  // namespace cube2

using namespace cube2;

extern "C" {

int cube2_init_mesh(cube2_ctx **out, const cube2_config *cfg, void *stream) {
    g_init_error.clear();
    auto fail = [](int code, const std::string &m) { g_init_error = m; return code; };
    if (!out || !cfg) return fail(CUBE2_ERR_BAD_ARG, "null ctx or config");
    *out = nullptr;
    if (!(cfg->box > 0) || cfg->n_ios < 4 || cfg->n_levels < 1 || cfg->n_levels > CUBE2_MAX_LEVELS ||
        cfg->n_particles < 0 || cfg->n_particles > 2147483647LL || !(cfg->b_pp > 0) ||
        !(cfg->omega_m > 0) || cfg->omega_l < 0 || cfg->alias_max < 0 || cfg->alias_max > 4 ||
        (cfg->assign_order != 0 && cfg->assign_order != 2 && cfg->assign_order != 3) ||
        !(cfg->iso_length >= 0) || cfg->iso_length > 0.5 * cfg->box)
        return fail(CUBE2_ERR_BAD_ARG, "invalid config field");
    if ((int64_t)cfg->n_ios * cfg->n_ios * cfg->n_ios > 2147483647LL)
        return fail(CUBE2_ERR_UNSUPPORTED_SIZE, "n_ios^3 exceeds int32 cell ids");
    for (int l = 0; l < cfg->n_levels; ++l) {
        const int n = cfg->n_mesh[l];
        if (!fft_size_supported(n)) return fail(CUBE2_ERR_UNSUPPORTED_SIZE, "mesh size not supported (2^a 3^b, 8..2048)");
        const int s = level_shift(cfg->n_ios, n);
        if (s < -2 || s > 1) return fail(CUBE2_ERR_UNSUPPORTED_SIZE, "n_ios / n_mesh must be 1/4, 1/2, 1 or 2");
        if (!(cfg->beta[l] > 0)) return fail(CUBE2_ERR_BAD_ARG, "beta must be positive");
        if (l > 0 && cfg->n_mesh[l] <= cfg->n_mesh[l - 1]) return fail(CUBE2_ERR_BAD_ARG, "levels must be coarsest first");
    }
    cube2_ctx *c = new cube2_ctx();
    c->cfg = *cfg;
    if (c->cfg.assign_order == 0) c->cfg.assign_order = 2;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    c->nl = cfg->n_levels;
    c->N = cfg->n_particles;
    c->n_ios = cfg->n_ios;
    c->n_cells = (int64_t)cfg->n_ios * cfg->n_ios * cfg->n_ios;
    c->s_ios = cfg->box / cfg->n_ios;
    double prev_b = -1.0;  // softening of the coarser level [Mpc/h]
    for (int l = 0; l < c->nl; ++l) {
        Level &L = c->lev[l];
        L.index = l;
        L.n = cfg->n_mesh[l];
        L.kxp = ((L.n / 2 + 1) + 15) / 16 * 16;
        L.shift = level_shift(cfg->n_ios, L.n);
        L.H = cfg->box / L.n;
        L.b_soft = cfg->beta[l];
        L.b_trunc = prev_b < 0 ? -1.0 : prev_b / L.H;
        // only the coarsest level's force reaches past its own softening
        L.iso = (l == 0 && cfg->iso_length > 0) ? cfg->iso_length / L.H : 0.0;
        prev_b = cfg->beta[l] * L.H;
        const int64_t n3 = (int64_t)L.n * L.n * L.n;
        // M = floor(N 2^48 / n^3) in 128-bit integer arithmetic
        const unsigned __int128 num = (unsigned __int128)(uint64_t)c->N << 48;
        L.mean_int = (uint64_t)(num / (unsigned __int128)n3);
        L.dens_scale = c->N > 0 ? (float)((double)n3 / (double)c->N * ldexp(1.0, -48)) : 0.0f;
    }
    c->b_range = prev_b;
    if (c->b_range > c->s_ios * (1.0 + 1e-12)) {
        delete c;
        return fail(CUBE2_ERR_BAD_ARG, "PP range (finest softening) exceeds the IOS cell");
    }
    if (cfg->b_pp >= c->b_range) {
        delete c;
        return fail(CUBE2_ERR_BAD_ARG, "b_pp must be below the PP range");
    }
    if (cfg->pm3_tile > 0) {
        const std::string why = pm3_geometry(c);
        if (!why.empty()) {
            delete c;
            return fail(why[0] == 'U' ? CUBE2_ERR_UNSUPPORTED_SIZE : CUBE2_ERR_BAD_ARG, why.substr(1));
        }
    }
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
    };
    for (int l = 0; l < c->nl; ++l) {
        Level &L = c->lev[l];
        const size_t n3 = (size_t)L.n * L.n * L.n;
        const size_t nh = (size_t)L.n * L.n * L.kxp;
        alloc((void **)&L.real, n3 * sizeof(float));
        alloc((void **)&L.spec, nh * sizeof(float2));
        L.green_len = green_table_len(L.n);
        alloc((void **)&L.green, (size_t)L.green_len * sizeof(float));
        if (L.n <= 1024) {
            const size_t h = (size_t)(L.n / 2 + 1);
            alloc((void **)&L.green2, h * h * (size_t)L.kxp * sizeof(float));
        }
        alloc((void **)&L.tw, (size_t)L.n * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemsetAsync(L.spec, 0, nh * sizeof(float2), c->stream);
    }
    const size_t N = (size_t)c->N;
    alloc((void **)&c->cellid, N * 4);
    alloc((void **)&c->toff, N * 3 * 2);
    alloc((void **)&c->tvel, N * 3 * 4);
    alloc((void **)&c->tcell, N * 4);
    alloc((void **)&c->tslot, N * 4);
    alloc((void **)&c->perm, N * 4);
    alloc((void **)&c->ncount, (size_t)c->n_cells * 4);
    alloc((void **)&c->nstart, (size_t)c->n_cells * 4);
    alloc((void **)&c->perm2, N * 4);
    alloc((void **)&c->big, (size_t)c->n_cells * 4);
    alloc((void **)&c->big_n, 2 * sizeof(int));
    alloc((void **)&c->pos4, N * 16);
    alloc((void **)&c->pp_perm, N * 4);
    alloc((void **)&c->pp_stats, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->pp_stats, 0, 4 * sizeof(unsigned long long), c->stream);
    if (cfg->vel_fp16) alloc((void **)&c->vel32, N * 3 * 4);
    if (c->pm3.on) {
        PM3 &M = c->pm3;
        Level &L = M.lev;
        const size_t m3 = (size_t)L.n * L.n * L.n;
        const size_t nh = (size_t)L.n * L.n * L.kxp;
        alloc((void **)&L.real, (size_t)M.max_tiles * m3 * sizeof(float));
        alloc((void **)&L.spec, (size_t)M.max_tiles * nh * sizeof(float2));
        L.green_len = green_table_len(L.n);
        alloc((void **)&L.green, (size_t)L.green_len * sizeof(float));
        alloc((void **)&L.tw, (size_t)L.n * sizeof(float2));
        alloc((void **)&M.rho_max, (size_t)M.n_sub * 4);
        alloc((void **)&M.slot, (size_t)M.n_sub * 4);
        alloc((void **)&M.list, (size_t)M.max_tiles * 4);
        alloc((void **)&M.count, 2 * sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(L.spec, 0, (size_t)M.max_tiles * nh * sizeof(float2), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(M.count, 0, 2 * sizeof(int), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(M.slot, 0xff, (size_t)M.n_sub * 4, c->stream);
        L.active = M.count;
        if (e == cudaSuccess) e = launch_init_twiddles(c, L);
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    c->scan_tmp_len = scan_scratch_len(c->n_cells);
    alloc((void **)&c->scan_tmp, (size_t)c->scan_tmp_len * 4);
    alloc((void **)&c->dev_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev_status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->host_status, sizeof(int), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->aux_event, cudaEventDisableTiming);
    for (int l = 0; l < c->nl && e == cudaSuccess; ++l) e = launch_init_twiddles(c, c->lev[l]);
    if (e != cudaSuccess) {
        g_init_error = std::string("allocation/setup failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_ctx(c);
        return CUBE2_ERR_CUDA;
    }
    *out = c;
    return CUBE2_OK;
}

int cube2_set_green(cube2_ctx *ctx, int level, const char *cache_path) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    const bool pm3 = level == CUBE2_LEVEL_PM3 && ctx->pm3.on;
    int r = pm3 ? CUBE2_OK : level_ok(ctx, level, false);
    if (r) return r;
    Level &L = pm3 ? ctx->pm3.lev : ctx->lev[level];
    const size_t nh = (size_t)L.green_len;
    // cache header: magic, n, entries (reduced layout), alias, assignment order, b_soft, b_trunc, isolation length
    struct Header { char magic[8]; int32_t n, len, alias, order; double b_soft, b_trunc, iso; } hdr{};
    memcpy(hdr.magic, "CUBE2G04", 8);
    hdr.n = L.n;
    hdr.len = (int32_t)L.green_len;
    hdr.alias = ctx->cfg.alias_max;
    hdr.order = ctx->cfg.assign_order;
    hdr.b_soft = L.b_soft;
    hdr.b_trunc = L.b_trunc;
    hdr.iso = L.iso;
    if (cache_path && cache_path[0]) {
        FILE *f = fopen(cache_path, "rb");
        if (f) {
            Header h{};
            bool ok = fread(&h, sizeof h, 1, f) == 1 && memcmp(&h, &hdr, sizeof h) == 0;
            if (ok) {
                std::vector<float> buf(nh);
                ok = fread(buf.data(), sizeof(float), nh, f) == nh;
                fclose(f);
                if (ok) {
                    cudaError_t e = cudaMemcpyAsync(L.green, buf.data(), nh * 4, cudaMemcpyHostToDevice, ctx->stream);
                    if (e == cudaSuccess) e = launch_green_fold(ctx, L);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
                    if (e != cudaSuccess) return cuda_error(ctx, e, "green cache upload");
                    L.has_green = true;
                    return CUBE2_OK;
                }
            } else {
                fclose(f);
            }
        }
    }
    cudaError_t e = launch_green(ctx, L, ctx->cfg.alias_max, ctx->cfg.assign_order);
    if (e == cudaSuccess) e = launch_green_fold(ctx, L);
    if (e != cudaSuccess) return cuda_error(ctx, e, "green kernel");
    L.has_green = true;
    if (cache_path && cache_path[0]) {
        std::vector<float> buf(nh);
        e = cudaMemcpyAsync(buf.data(), L.green, nh * 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_error(ctx, e, "green cache download");
        FILE *f = fopen(cache_path, "wb");
        if (!f) return set_error(ctx, CUBE2_ERR_BAD_ARG, std::string("cannot write green cache ") + cache_path);
        const bool ok = fwrite(&hdr, sizeof hdr, 1, f) == 1 && fwrite(buf.data(), 4, nh, f) == nh;
        fclose(f);
        if (!ok) return set_error(ctx, CUBE2_ERR_BAD_ARG, "short write of green cache");
    }
    return CUBE2_OK;
}

// Deposit / interpolation of one level (level >= 0) or of all levels (-1),
// with the context's assignment (CIC: one exact-integer pass over all
// levels; TSC: per level).
static cudaError_t deposit_levels(cube2_ctx *ctx, int level, const cube2_particles *p) {
    if (ctx->cfg.assign_order != 3) return launch_deposit(ctx, level, p, nullptr);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < ctx->nl && e == cudaSuccess; ++l)
        if (level < 0 || l == level) e = launch_tsc_deposit(ctx, ctx->lev[l], p);
    return e;
}

static cudaError_t interp_levels(cube2_ctx *ctx, int level, const cube2_particles *p, int accumulate) {
    // CIC and TSC: the tiled gather over every level in one pass
    return launch_interp(ctx, level, p, accumulate);
}

int cube2_deposit(cube2_ctx *ctx, int level, const cube2_particles *p) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, true);
    if (r) return r;
    if (!particles_ok(ctx, p, false, false)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle arrays");
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = deposit_levels(ctx, level, p);
    if (e != cudaSuccess) return cuda_error(ctx, e, "deposit");
    for (int l = 0; l < ctx->nl; ++l)
        if (level < 0 || l == level) { ctx->lev[l].has_density = true; ctx->lev[l].has_potential = false; }
    return CUBE2_OK;
}

int cube2_deposit_u64(cube2_ctx *ctx, int level, const cube2_particles *p, uint64_t *out) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, false);
    if (r) return r;
    if (!out || !particles_ok(ctx, p, false, false)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad arguments");
    if (ctx->cfg.assign_order == 3)
        return set_error(ctx, CUBE2_ERR_UNSUPPORTED_SIZE, "the exact integer accumulator exists for CIC only");
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = launch_deposit(ctx, level, p, out);
    if (e != cudaSuccess) return cuda_error(ctx, e, "deposit_u64");
    return CUBE2_OK;
}

int cube2_solve_pm(cube2_ctx *ctx, int level) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, false);
    if (r) return r;
    Level &L = ctx->lev[level];
    if (!L.has_green || !L.has_density) return set_error(ctx, CUBE2_ERR_STATE, "solve_pm needs set_green and deposit");
    cudaError_t e = launch_fft_forward(ctx, L);
    if (e == cudaSuccess) e = launch_fft_z_green(ctx, L);
    if (e == cudaSuccess) e = launch_fft_inverse(ctx, L);
    if (e != cudaSuccess) return cuda_error(ctx, e, "solve_pm");
    L.has_density = false;
    L.has_potential = true;
    return CUBE2_OK;
}

int cube2_interp_force(cube2_ctx *ctx, int level, const cube2_particles *p, int accumulate) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, true);
    if (r) return r;
    if (!particles_ok(ctx, p, false, true)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle arrays");
    for (int l = 0; l < ctx->nl; ++l)
        if ((level < 0 || l == level) && !ctx->lev[l].has_potential)
            return set_error(ctx, CUBE2_ERR_STATE, "interp_force needs solve_pm");
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = interp_levels(ctx, level, p, accumulate);
    if (e != cudaSuccess) return cuda_error(ctx, e, "interp_force");
    return CUBE2_OK;
}

int cube2_pp_force(cube2_ctx *ctx, const cube2_particles *p, int accumulate) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (!particles_ok(ctx, p, false, true)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle arrays");
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess && ctx->pm3.on) e = launch_pm3_map(ctx, p);
    if (e == cudaSuccess) e = launch_pp(ctx, p, accumulate, 0.0f);
    if (e != cudaSuccess) return cuda_error(ctx, e, "pp_force");
    return CUBE2_OK;
}

// deposit + solve (all levels) + interp + PP (+ optional fused kick); cellid must be valid.
static int force_core(cube2_ctx *ctx, const cube2_particles *p, float kick) {
    for (int l = 0; l < ctx->nl; ++l)
        if (!ctx->lev[l].has_green) return set_error(ctx, CUBE2_ERR_STATE, "force needs every level's Green's table");
    if (ctx->pm3.on && !ctx->pm3.lev.has_green)
        return set_error(ctx, CUBE2_ERR_STATE, "force needs the third level's Green's table (CUBE2_LEVEL_PM3)");
    cudaError_t e = deposit_levels(ctx, -1, p);
    for (int l = 0; l < ctx->nl && e == cudaSuccess; ++l) {
        e = launch_fft_forward(ctx, ctx->lev[l]);
        if (e == cudaSuccess) e = launch_fft_z_green(ctx, ctx->lev[l]);
        if (e == cudaSuccess) e = launch_fft_inverse(ctx, ctx->lev[l]);
        ctx->lev[l].has_density = false;
        ctx->lev[l].has_potential = true;
    }
    if (e == cudaSuccess) e = interp_levels(ctx, -1, p, 0);
    if (e == cudaSuccess && ctx->pm3.on) e = launch_pm3(ctx, p);
    if (e == cudaSuccess) e = launch_pp(ctx, p, 1, kick);
    if (e != cudaSuccess) return cuda_error(ctx, e, "force");
    return CUBE2_OK;
}

int cube2_force(cube2_ctx *ctx, const cube2_particles *p) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (!particles_ok(ctx, p, false, true)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle arrays");
    cudaError_t e = launch_cellid(ctx, p);
    if (e != cudaSuccess) return cuda_error(ctx, e, "cellid");
    return force_core(ctx, p, 0.0f);
}

int cube2_kdk_factors(const cube2_config *cfg, double a0, double a1, double out[3]) {
    if (!cfg || !out || !(a0 > 0) || !(a1 > a0)) return CUBE2_ERR_BAD_ARG;
    const double ah = 0.5 * (a0 + a1);
    out[0] = integrate(a0, ah, cfg->omega_m, cfg->omega_l, 2);
    out[1] = integrate(a0, a1, cfg->omega_m, cfg->omega_l, 3);
    out[2] = integrate(ah, a1, cfg->omega_m, cfg->omega_l, 2);
    return CUBE2_OK;
}

// One KDK step; if after_rebin is given it is recorded on the context stream
// once the particle positions, counts and starts hold their final values.
static int kdk_step_core(cube2_ctx *ctx, cube2_particles *p, double a0, double a1, cudaEvent_t after_rebin) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (!particles_ok(ctx, p, true, true)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle arrays");
    double f[3];
    if (cube2_kdk_factors(&ctx->cfg, a0, a1, f)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "need 0 < a0 < a1");
    const double c = 1.5 * ctx->cfg.omega_m;
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = launch_kick_drift(ctx, p, (float)(c * f[0]), (float)(f[1] * FIX / ctx->s_ios));
    if (e == cudaSuccess) e = launch_rebin(ctx, p);
    if (e == cudaSuccess && after_rebin) e = cudaEventRecord(after_rebin, ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "kick/drift/rebin");
    const int r = force_core(ctx, p, (float)(c * f[2]));
    if (r != CUBE2_OK || !ctx->vel32) return r;
    // FP16 storage: encode the working momenta of the new order
    const float *const w[3] = {ctx->vel32, ctx->vel32 + ctx->N, ctx->vel32 + 2 * ctx->N};
    e = launch_vel_encode(ctx, p, w);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "velocity encode");
}

int cube2_kdk_step(cube2_ctx *ctx, cube2_particles *p, double a0, double a1) {
    return kdk_step_core(ctx, p, a0, a1, nullptr);
}

int cube2_ios_from_positions(cube2_ctx *ctx, const double *const pos[3], const float *const mom[3],
                             cube2_particles *p, int32_t *perm) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (ctx->vel32) return set_error(ctx, CUBE2_ERR_BAD_ARG, "placement writes FP32 velocities (vel_fp16 context)");
    if (!particles_ok(ctx, p, true, false)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle arrays");
    if (ctx->N > 0 && (!pos || !pos[0] || !pos[1] || !pos[2]))
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "null position arrays");
    if (ctx->N > 0 && mom && (!mom[0] || !mom[1] || !mom[2]))
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "momenta must be three arrays or null");
    cudaError_t e = launch_place(ctx, pos, mom);
    if (e == cudaSuccess) e = launch_rebin(ctx, p);
    if (e == cudaSuccess && perm && ctx->N > 0)
        e = cudaMemcpyAsync(perm, ctx->perm, sizeof(int32_t) * (size_t)ctx->N, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "ios_from_positions");
    return CUBE2_OK;
}

int cube2_adjoint_init(cube2_ctx *ctx) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (ctx->vel32) return set_error(ctx, CUBE2_ERR_STATE, "the adjoint takes FP32 velocities (vel_fp16 context)");
    if (ctx->pm3.on) return set_error(ctx, CUBE2_ERR_STATE, "the adjoint does not cover the adaptive third level");
    if (ctx->vjp_mu) return CUBE2_OK;
    int64_t m = 0;
    for (int l = 0; l < ctx->nl; ++l) m = std::max(m, (int64_t)ctx->lev[l].n * ctx->lev[l].n * ctx->lev[l].n);
    const size_t N = (size_t)std::max<int64_t>(ctx->N, 1);
    cudaError_t e = cudaMalloc((void **)&ctx->vjp_mu, sizeof(float) * 3 * (size_t)m);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->vjp_t, sizeof(float) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->vjp_u, sizeof(float) * 12 * N);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->vjp_sq, sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(ctx->vjp_mu);
        cudaFree(ctx->vjp_t);
        cudaFree(ctx->vjp_u);
        cudaFree(ctx->vjp_sq);
        ctx->vjp_mu = nullptr;
        ctx->vjp_t = ctx->vjp_u = nullptr;
        ctx->vjp_sq = nullptr;
        return cuda_error(ctx, e, "adjoint scratch");
    }
    return CUBE2_OK;
}

// w = d<v, F>/dx (overwritten); cellid must be valid for p.
static cudaError_t force_vjp_core(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3],
                                  float *const w[3]) {
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < 3 && e == cudaSuccess; ++d)
        if (ctx->N > 0) e = cudaMemsetAsync(w[d], 0, sizeof(float) * (size_t)ctx->N, ctx->stream);
    for (int l = 0; l < ctx->nl && e == cudaSuccess; ++l) {
        Level &L = ctx->lev[l];
        e = launch_deposit(ctx, l, p, nullptr);                        // rho
        if (e == cudaSuccess) e = launch_fft_forward(ctx, L);           // phi = G * rho
        if (e == cudaSuccess) e = launch_fft_z_green(ctx, L);
        if (e == cudaSuccess) e = launch_fft_inverse(ctx, L);
        if (e == cudaSuccess) e = launch_vjp_gather_e(ctx, L, p, v, w);  // -sum grad W (E . v)
        if (e == cudaSuccess) e = launch_vjp_source(ctx, L, p, v);      // s = (n^3/N) sum_d D_d * mu_d
        if (e == cudaSuccess) e = launch_fft_forward(ctx, L);           // psi = G * s
        if (e == cudaSuccess) e = launch_fft_z_green(ctx, L);
        if (e == cudaSuccess) e = launch_fft_inverse(ctx, L);
        if (e == cudaSuccess) e = launch_vjp_gather_psi(ctx, L, p, v, w);  // + sum grad W psi
        L.has_density = false;
        L.has_potential = false;
    }
    if (e == cudaSuccess) e = launch_pp_vjp(ctx, p, v, w);
    return e;
}

static int adjoint_ready(cube2_ctx *ctx) {
    if (ctx->cfg.assign_order == 3)
        return set_error(ctx, CUBE2_ERR_UNSUPPORTED_SIZE, "the adjoint is built for the CIC assignment");
    if (!ctx->vjp_mu) return set_error(ctx, CUBE2_ERR_STATE, "call cube2_adjoint_init first");
    for (int l = 0; l < ctx->nl; ++l)
        if (!ctx->lev[l].has_green) return set_error(ctx, CUBE2_ERR_STATE, "the product needs every level's Green's table");
    return CUBE2_OK;
}

int cube2_force_vjp(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3], float *const w[3]) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (!particles_ok(ctx, p, false, false) || !v || !w)
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle or cotangent arrays");
    for (int d = 0; d < 3; ++d)
        if (ctx->N > 0 && (!v[d] || !w[d])) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null cotangent array");
    int r = adjoint_ready(ctx);
    if (r) return r;
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = force_vjp_core(ctx, p, v, w);
    if (e != cudaSuccess) return cuda_error(ctx, e, "force_vjp");
    return CUBE2_OK;
}

int cube2_kdk_permutation(cube2_ctx *ctx, int32_t *out) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (!out && ctx->N > 0) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null out");
    if (ctx->N == 0) return CUBE2_OK;
    const cudaError_t e = cudaMemcpyAsync(out, ctx->perm, sizeof(int32_t) * (size_t)ctx->N, cudaMemcpyDeviceToDevice,
                                          ctx->stream);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "permutation copy");
}

int cube2_density_mse_vjp(cube2_ctx *ctx, int level, const cube2_particles *p, const float *target, float *const w[3],
                          double *loss) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, false);
    if (r) return r;
    if (!particles_ok(ctx, p, false, false) || !target || !w || !loss)
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle, target or output arrays");
    for (int d = 0; d < 3; ++d)
        if (ctx->N > 0 && !w[d]) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null output array");
    if (ctx->cfg.assign_order == 3)
        return set_error(ctx, CUBE2_ERR_UNSUPPORTED_SIZE, "the adjoint is built for the CIC assignment");
    if (!ctx->vjp_mu) return set_error(ctx, CUBE2_ERR_STATE, "call cube2_adjoint_init first");
    Level &L = ctx->lev[level];
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = launch_deposit(ctx, level, p, nullptr);
    for (int d = 0; d < 3 && e == cudaSuccess; ++d)
        if (ctx->N > 0) e = cudaMemsetAsync(w[d], 0, sizeof(float) * (size_t)ctx->N, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->vjp_sq, 0, sizeof(double), ctx->stream);
    if (e == cudaSuccess) e = launch_density_mse_vjp(ctx, L, p, target, w, ctx->vjp_sq);
    double sq = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sq, ctx->vjp_sq, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "density_mse_vjp");
    L.has_density = false;
    L.has_potential = false;
    *loss = sq / ((double)L.n * L.n * L.n);
    return CUBE2_OK;
}

int cube2_density_vjp(cube2_ctx *ctx, int level, const cube2_particles *p, const float *g, float *const w[3]) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, false);
    if (r) return r;
    if (!particles_ok(ctx, p, false, false) || !g || !w)
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle, cotangent or output arrays");
    for (int d = 0; d < 3; ++d)
        if (ctx->N > 0 && !w[d]) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null output array");
    if (ctx->cfg.assign_order == 3)
        return set_error(ctx, CUBE2_ERR_UNSUPPORTED_SIZE, "the adjoint is built for the CIC assignment");
    Level &L = ctx->lev[level];
    cudaError_t e = launch_cellid(ctx, p);
    for (int d = 0; d < 3 && e == cudaSuccess; ++d)
        if (ctx->N > 0) e = cudaMemsetAsync(w[d], 0, sizeof(float) * (size_t)ctx->N, ctx->stream);
    if (e == cudaSuccess) e = launch_density_vjp(ctx, L, p, g, w);
    if (e != cudaSuccess) return cuda_error(ctx, e, "density_vjp");
    L.has_density = false;
    L.has_potential = false;
    return CUBE2_OK;
}

int cube2_kdk_adjoint_step(cube2_ctx *ctx, const cube2_particles *pre, const cube2_particles *post,
                           const int32_t *perm, float *const xbar[3], float *const pbar[3], double a0, double a1) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (!particles_ok(ctx, pre, false, false) || !particles_ok(ctx, post, false, false) || !xbar || !pbar ||
        (ctx->N > 0 && !perm))
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad checkpoint, permutation or adjoint arrays");
    for (int d = 0; d < 3; ++d)
        if (ctx->N > 0 && (!xbar[d] || !pbar[d])) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null adjoint array");
    int r = adjoint_ready(ctx);
    if (r) return r;
    double f[3];
    if (cube2_kdk_factors(&ctx->cfg, a0, a1, f)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "need 0 < a0 < a1");
    const double c = 1.5 * ctx->cfg.omega_m;
    const size_t N = (size_t)ctx->N;
    float *const t[3] = {ctx->vjp_t, ctx->vjp_t + N, ctx->vjp_t + 2 * N};
    const float *const pb[3] = {pbar[0], pbar[1], pbar[2]};
    // second kick: p_out = p_mid + k2 F(x_new)  ->  xbar += k2 F^T pbar   (post-step order)
    cudaError_t e = launch_cellid(ctx, post);
    if (e == cudaSuccess) e = force_vjp_core(ctx, post, pb, t);
    // re-bin: back to the pre-step order
    if (e == cudaSuccess) e = launch_kdk_adjoint_scatter(ctx, perm, xbar, pbar, ctx->vjp_t, (float)(c * f[2]));
    // drift: x_new = x + Dr p_mid  ->  pbar += Dr xbar
    if (e == cudaSuccess) e = launch_kdk_adjoint_drift(ctx, xbar, pbar, (float)f[1]);
    // first kick: p_mid = p + k1 F(x)  ->  xbar += k1 F^T pbar
    if (e == cudaSuccess) e = launch_cellid(ctx, pre);
    if (e == cudaSuccess) e = force_vjp_core(ctx, pre, pb, t);
    if (e == cudaSuccess) e = launch_axpy3(ctx, xbar, ctx->vjp_t, (float)(c * f[0]));
    if (e != cudaSuccess) return cuda_error(ctx, e, "kdk_adjoint_step");
    return CUBE2_OK;
}

int cube2_kdk_adjoint(cube2_ctx *ctx, const cube2_particles *const *states, const int32_t *const *perms, int n_steps,
                      const double *a, float *const xbar[3], float *const pbar[3]) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    if (!states || !perms || !a || n_steps < 1 || !xbar || !pbar)
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad states, maps, schedule or adjoint arrays");
    for (int k = 0; k <= n_steps; ++k)
        if (!particles_ok(ctx, states[k], false, false)) return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad state");
    for (int k = 0; k < n_steps; ++k) {
        if (ctx->N > 0 && !perms[k]) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null re-bin map");
        if (!(a[k] > 0) || !(a[k + 1] > a[k])) return set_error(ctx, CUBE2_ERR_BAD_ARG, "need 0 < a0 < a1 < ...");
    }
    for (int d = 0; d < 3; ++d)
        if (ctx->N > 0 && (!xbar[d] || !pbar[d])) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null adjoint array");
    int r = adjoint_ready(ctx);
    if (r) return r;
    const double c = 1.5 * ctx->cfg.omega_m;
    const size_t N = (size_t)ctx->N;
    float *const t[3] = {ctx->vjp_t, ctx->vjp_t + N, ctx->vjp_t + 2 * N};
    const float *const pb[3] = {pbar[0], pbar[1], pbar[2]};
    // t = F'(x_n)^T pbar at the last state; afterwards each step's first-kick
    // product (at its pre state, with the pbar the next reverse step starts
    // from) is the previous step's second-kick product
    cudaError_t e = launch_cellid(ctx, states[n_steps]);
    if (e == cudaSuccess) e = force_vjp_core(ctx, states[n_steps], pb, t);
    for (int k = n_steps - 1; k >= 0 && e == cudaSuccess; --k) {
        double f[3];
        cube2_kdk_factors(&ctx->cfg, a[k], a[k + 1], f);
        e = launch_kdk_adjoint_scatter(ctx, perms[k], xbar, pbar, ctx->vjp_t, (float)(c * f[2]));
        if (e == cudaSuccess) e = launch_kdk_adjoint_drift(ctx, xbar, pbar, (float)f[1]);
        if (e == cudaSuccess) e = launch_cellid(ctx, states[k]);
        if (e == cudaSuccess) e = force_vjp_core(ctx, states[k], pb, t);
        if (e == cudaSuccess) e = launch_axpy3(ctx, xbar, ctx->vjp_t, (float)(c * f[0]));
    }
    if (e != cudaSuccess) return cuda_error(ctx, e, "kdk_adjoint");
    return CUBE2_OK;
}

int cube2_kdk_step_host(cube2_ctx *ctx, cube2_particles *dev, cube2_particles *host, double a0, double a1) {
    if (!ctx || !host) return CUBE2_ERR_BAD_ARG;
    if (ctx->vel32) return set_error(ctx, CUBE2_ERR_BAD_ARG, "the host-buffer step takes FP32 velocities");
    if (!particles_ok(ctx, dev, true, true) || !particles_ok(ctx, host, true, true))
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle arrays");
    const size_t N = (size_t)ctx->N, C = (size_t)ctx->n_cells;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes, cudaMemcpyKind k, cudaStream_t s) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, k, s);
    };
    for (int d = 0; d < 3; ++d) {
        cp(dev->off[d], host->off[d], N * 2, cudaMemcpyHostToDevice, ctx->stream);
        cp(dev->vel[d], host->vel[d], N * 4, cudaMemcpyHostToDevice, ctx->stream);
        cp(dev->acc[d], host->acc[d], N * 4, cudaMemcpyHostToDevice, ctx->stream);
    }
    cp(dev->count, host->count, C * 4, cudaMemcpyHostToDevice, ctx->stream);
    // start is the exclusive prefix sum of count (the IOS layout): formed on
    // the device instead of uploaded
    if (e == cudaSuccess) e = launch_scan(ctx, dev->count, dev->start, (int64_t)C);
    if (e != cudaSuccess) return cuda_error(ctx, e, "upload");
    int r = kdk_step_core(ctx, dev, a0, a1, ctx->aux_event);
    if (r) return r;
    // positions, counts and starts are final after the re-bin: download them
    // on the second stream while the forces are computed
    e = cudaStreamWaitEvent(ctx->aux_stream, ctx->aux_event, 0);
    for (int d = 0; d < 3; ++d) cp(host->off[d], dev->off[d], N * 2, cudaMemcpyDeviceToHost, ctx->aux_stream);
    cp(host->count, dev->count, C * 4, cudaMemcpyDeviceToHost, ctx->aux_stream);
    cp(host->start, dev->start, C * 4, cudaMemcpyDeviceToHost, ctx->aux_stream);
    for (int d = 0; d < 3; ++d) {
        cp(host->vel[d], dev->vel[d], N * 4, cudaMemcpyDeviceToHost, ctx->stream);
        cp(host->acc[d], dev->acc[d], N * 4, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->aux_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "download");
    return CUBE2_OK;
}

static int copy_grid(cube2_ctx *ctx, void *out, const void *src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "grid copy");
}

int cube2_get_density(cube2_ctx *ctx, int level, float *out) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, false);
    if (r) return r;
    if (!out) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null out");
    const Level &L = ctx->lev[level];
    if (!L.has_density) return set_error(ctx, CUBE2_ERR_STATE, "no density (deposit first)");
    return copy_grid(ctx, out, L.real, (size_t)L.n * L.n * L.n * 4);
}

int cube2_get_potential(cube2_ctx *ctx, int level, float *out) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, false);
    if (r) return r;
    if (!out) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null out");
    const Level &L = ctx->lev[level];
    if (!L.has_potential) return set_error(ctx, CUBE2_ERR_STATE, "no potential (solve_pm first)");
    return copy_grid(ctx, out, L.real, (size_t)L.n * L.n * L.n * 4);
}

int cube2_get_green(cube2_ctx *ctx, int level, float *out) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    const bool pm3 = level == CUBE2_LEVEL_PM3 && ctx->pm3.on;
    int r = pm3 ? CUBE2_OK : level_ok(ctx, level, false);
    if (r) return r;
    if (!out) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null out");
    const Level &L = pm3 ? ctx->pm3.lev : ctx->lev[level];
    if (!L.has_green) return set_error(ctx, CUBE2_ERR_STATE, "no Green's table");
    const cudaError_t e = launch_green_expand(ctx, L, out);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "green expand");
}

int cube2_debug_forward_fft(cube2_ctx *ctx, int level, float *out) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    int r = level_ok(ctx, level, false);
    if (r) return r;
    Level &L = ctx->lev[level];
    if (!out) return set_error(ctx, CUBE2_ERR_BAD_ARG, "null out");
    if (!L.has_density) return set_error(ctx, CUBE2_ERR_STATE, "no density (deposit first)");
    cudaError_t e = launch_fft_forward(ctx, L);
    if (e == cudaSuccess) e = launch_fft_z_forward(ctx, L);
    if (e != cudaSuccess) return cuda_error(ctx, e, "forward fft");
    const int nh = L.n / 2 + 1;
    e = cudaMemcpy2DAsync(out, nh * 8, L.spec, L.kxp * 8, nh * 8, (size_t)L.n * L.n, cudaMemcpyDeviceToDevice,
                          ctx->stream);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "spectrum copy");
}

int cube2_check(cube2_ctx *ctx) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    cudaError_t e = cudaMemcpyAsync(ctx->host_status, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "check");
    const int st = *ctx->host_status;
    if (!st) return CUBE2_OK;
    e = cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "check reset");
    if (st & ST_CAPACITY) return set_error(ctx, CUBE2_ERR_CAPACITY, "uint64 deposit accumulator overflowed");
    if (st & ST_NONFINITE) return set_error(ctx, CUBE2_ERR_NONFINITE, "non-finite force or momentum");
    if (st & ST_DISPLACEMENT) return set_error(ctx, CUBE2_ERR_DISPLACEMENT, "drift displacement too large");
    return set_error(ctx, CUBE2_ERR_TIMEOUT, "device wait timed out");
}

int cube2_profile(cube2_ctx *ctx, int capacity) {
    if (!ctx || capacity < 0) return CUBE2_ERR_BAD_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "profile sync");
    prof_free(ctx);
    ctx->prof_overflow = 0;
    if (capacity == 0) return CUBE2_OK;
    ctx->ev = new cudaEvent_t[2 * (size_t)capacity];
    ctx->prof_cls = new int[capacity];
    for (int i = 0; i < 2 * capacity; ++i) {
        e = cudaEventCreate(&ctx->ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->ev[j]);
            delete[] ctx->ev;
            delete[] ctx->prof_cls;
            ctx->ev = nullptr;
            ctx->prof_cls = nullptr;
            return cuda_error(ctx, e, "profile events");
        }
    }
    ctx->prof_cap = capacity;
    ctx->prof_used = 0;
    ctx->prof = true;
    return CUBE2_OK;
}

int cube2_profile_read(cube2_ctx *ctx, double *ms, int64_t *counts) {
    if (!ctx || !ms || !counts) return CUBE2_ERR_BAD_ARG;
    const int nslots = CUBE2_PROFILE_CLASSES * CUBE2_MAX_LEVELS;
    for (int i = 0; i < nslots; ++i) { ms[i] = 0.0; counts[i] = 0; }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "profile sync");
    for (int s = 0; s < ctx->prof_used; ++s) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ctx->ev[2 * s], ctx->ev[2 * s + 1]);
        if (e != cudaSuccess) return cuda_error(ctx, e, "profile elapsed");
        ms[ctx->prof_cls[s]] += t;
        counts[ctx->prof_cls[s]] += 1;
    }
    ctx->prof_used = 0;
    const int over = ctx->prof_overflow;
    ctx->prof_overflow = 0;
    return over ? set_error(ctx, CUBE2_ERR_CAPACITY, "profile event pool overflowed") : CUBE2_OK;
}

const char *cube2_profile_class_name(int cls) {
    static const char *names[CUBE2_PROFILE_CLASSES] = {
        "deposit", "fft_x_fwd", "fft_y_fwd", "fft_z_green", "fft_y_inv", "fft_x_inv", "interp", "pp",
        "kick", "kick_drift", "scan", "scatter", "sort", "gather", "cellid", "green", "pp_order", "prep",
        "sort_big", "vjp_gather", "vjp_source", "pp_vjp", "adj_kdk", "pm3_map", "pm3_deposit", "pm3_fft",
        "pm3_gather"};
    return (cls >= 0 && cls < CUBE2_PROFILE_CLASSES) ? names[cls] : "";
}

int cube2_pp_count(cube2_ctx *ctx, int on) {
    if (!ctx) return CUBE2_ERR_BAD_ARG;
    ctx->pp_count = on != 0;
    return CUBE2_OK;
}

int cube2_pp_stats_paths(cube2_ctx *ctx, int64_t out[4]) {
    if (!ctx || !out) return CUBE2_ERR_BAD_ARG;
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, ctx->pp_stats, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->pp_stats, 0, sizeof h, ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "pp stats");
    for (int k = 0; k < 4; ++k) out[k] = (int64_t)h[k];
    return CUBE2_OK;
}

int cube2_pp_stats(cube2_ctx *ctx, int64_t out[2]) {
    if (!ctx || !out) return CUBE2_ERR_BAD_ARG;
    int64_t all[4];
    const int rc = cube2_pp_stats_paths(ctx, all);
    if (rc != CUBE2_OK) return rc;
    out[0] = all[0];
    out[1] = all[1];
    return CUBE2_OK;
}

int cube2_vel_encode(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3]) {
    if (!ctx || !v) return CUBE2_ERR_BAD_ARG;
    if (!ctx->vel32) return set_error(ctx, CUBE2_ERR_STATE, "the context was not made with vel_fp16");
    if (!particles_ok(ctx, p, true, false) || (ctx->N > 0 && (!v[0] || !v[1] || !v[2])))
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle or velocity arrays");
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = launch_vel_encode(ctx, p, v);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "velocity encode");
}

int cube2_vel_decode(cube2_ctx *ctx, const cube2_particles *p, float *const v[3]) {
    if (!ctx || !v) return CUBE2_ERR_BAD_ARG;
    if (!ctx->vel32) return set_error(ctx, CUBE2_ERR_STATE, "the context was not made with vel_fp16");
    if (!particles_ok(ctx, p, true, false) || (ctx->N > 0 && (!v[0] || !v[1] || !v[2])))
        return set_error(ctx, CUBE2_ERR_BAD_ARG, "bad particle or velocity arrays");
    cudaError_t e = launch_cellid(ctx, p);
    if (e == cudaSuccess) e = launch_vel_decode(ctx, p, v);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "velocity decode");
}

int cube2_pm3_info(cube2_ctx *ctx, double out[8]) {
    if (!ctx || !out) return CUBE2_ERR_BAD_ARG;
    const PM3 &M = ctx->pm3;
    if (!M.on) return set_error(ctx, CUBE2_ERR_STATE, "the adaptive third level is off");
    const double v[8] = {(double)M.T, (double)M.ns, (double)M.r, (double)M.B, (double)M.m, M.H, M.b3,
                         (double)M.max_tiles};
    for (int i = 0; i < 8; ++i) out[i] = v[i];
    return CUBE2_OK;
}

int cube2_pm3_stats(cube2_ctx *ctx, int64_t out[2]) {
    if (!ctx || !out) return CUBE2_ERR_BAD_ARG;
    if (!ctx->pm3.on) return set_error(ctx, CUBE2_ERR_STATE, "the adaptive third level is off");
    int h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, ctx->pm3.count, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_error(ctx, e, "pm3 stats");
    out[0] = h[0];
    out[1] = h[1];
    return CUBE2_OK;
}

int cube2_pm3_map(cube2_ctx *ctx, int32_t *out) {
    if (!ctx || !out) return CUBE2_ERR_BAD_ARG;
    if (!ctx->pm3.on) return set_error(ctx, CUBE2_ERR_STATE, "the adaptive third level is off");
    const cudaError_t e = cudaMemcpyAsync(out, ctx->pm3.slot, (size_t)ctx->pm3.n_sub * 4, cudaMemcpyDeviceToDevice,
                                          ctx->stream);
    return e == cudaSuccess ? CUBE2_OK : cuda_error(ctx, e, "pm3 map");
}

const char *cube2_last_error(cube2_ctx *ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

int64_t cube2_launch_count(cube2_ctx *ctx) { return ctx ? ctx->launches : 0; }

void cube2_destroy(cube2_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
}

}  // extern "C"
