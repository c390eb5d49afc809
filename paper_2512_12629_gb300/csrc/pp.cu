// Short-range particle-particle force (paper Sec. 2.2.3 and Eq. PP):
//   F_i += V_p / (4 pi) (R(r, b_pp) - R(r, b_range)) (x_j - x_i) / r,   0 < r < b_range,
// with R(r, b) of Eq. (refforce).  The IOS order is the cell list (Sec. 2.3): the
// IOS cell is at least b_range wide, so the 27 cells around a particle's cell
// hold all its partners.  The cells of one (dz, dy) row are adjacent in memory,
// so a run of cells along x is one contiguous particle range.
//
// Arithmetic is carried out in IOS-cell units.  A particle's in-cell offset
// off/2^16 is exact in FP32 (prep kernel, once per force evaluation) and so is
// (cell step + offset) and the separation of two such values: the pair term is
// bitwise antisymmetric.  Each ordered pair is evaluated from both sides (gather
// form, no atomics, deterministic).
//
// One thread per target, in PP slot order: cell order, with the particles of
// dense cells (64 or more) reordered by a 4x4x4 sub-cell key inside their
// cell (PP's own position array and slot -> particle map; results are written
// back to the particle's index).  A warp whose 32 targets
// lie in one row of cells, narrow enough (every dense region; see wmax),
// shares one source stream: the particles of cells xa-1 .. xb+1 in the 9 rows
// around it.  It stages 64 sources at a time in shared memory; each lane tests
// all 64 (sign of r^2 - b_cut^2 shifted into two 32-bit masks, 8 instructions
// per candidate) and evaluates only the set bits, one mask word after the
// other, with a branch-free far-pair formula; pairs closer than b_pp take a
// separate, rarely entered loop.
// Other warps (sparse regions) walk each lane's own 27 cells.  The Jacobian
// product of the adjoint (pp_vjp_kernel) uses the same two paths.
// Per-particle sums are compensated: plain FP32 partials per batch are added to
// the running total with Kahan's scheme.  The path a warp takes depends only
// on the cell layout and every sum has a fixed order, so results are bitwise
// reproducible.
#include "common.cuh"

#include <string.h>

namespace cube2 {
namespace {

struct PPParams {
    const float4 *pos;          // [N] (off_x, off_y, off_z)/2^16, .w = cell id bits, in PP slot order
    const int32_t *perm;        // [N] particle index of each slot
    const int32_t *count, *start;
    float *acc0, *acc1, *acc2;
    float *vel0, *vel1, *vel2;
    unsigned long long *stats;  // [2]: in-range ordered pairs, candidates
    int64_t N;
    int n_ios, accumulate;
    float inv_bpp, inv_bcut, bcut2, bpp2;   // IOS-cell units
    float coef;                       // V_p / (4 pi s_ios^2)
    float kick;                       // 0: no kick; else v += kick * acc after the sum
    int *status;
    // adaptive third level: targets in a refined subtile (pm3_slot >= 0) use
    // the range b_3 (bcut2_3, inv_bcut_3) instead of b_cut; null when off
    const int32_t *pm3_slot;
    int pm3_T, pm3_ns;
    float bcut2_3, inv_bcut_3;
    int wmax;                         // widest warp (cells beyond the first) on the shared stream
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

constexpr int PP_WARPS_CTA = 4;
constexpr int PP_CTA = PP_WARPS_CTA * 32;

// Float offsets (and the cell id bits) for the PP kernel.
__global__ void __launch_bounds__(PP_CTA) prep_positions_kernel(const uint16_t *off0, const uint16_t *off1,
                                                                const uint16_t *off2, const int32_t *cellid,
                                                                float4 *pos, int32_t *perm, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = 1.0f / FIX;
    pos[i] = make_float4((float)off0[i] * s, (float)off1[i] * s, (float)off2[i] * s, __int_as_float(cellid[i]));
    if (perm) perm[i] = (int32_t)i;
}

// Dense cells are reordered for PP by a 4x4x4 sub-cell key (Morton order of
// the top two offset bits per axis), stably: a warp's targets then lie close
// together and have similar neighbour counts, so set-bit evaluation wastes
// fewer lanes (measured 5 % off PP at z ~ 0).  Only PP's own arrays are
// reordered (pos4 and the slot -> particle map); the particle arrays are not.
constexpr int PP_SORT_MIN = 64;   // cells with fewer particles keep their order

__device__ __forceinline__ int subcell_key(unsigned ox, unsigned oy, unsigned oz) {
    const unsigned x = ox >> 14, y = oy >> 14, z = oz >> 14;   // two bits each
    return (int)((((x >> 1) | ((y >> 1) << 1) | ((z >> 1) << 2)) << 3) | ((x & 1) | ((y & 1) << 1) | ((z & 1) << 2)));
}

__global__ void __launch_bounds__(256) pp_dense_list_kernel(const int32_t *count, int64_t n_cells, int32_t *list,
                                                            int *list_n) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_cells && count[c] >= PP_SORT_MIN) list[atomicAdd(list_n, 1)] = (int32_t)c;
}

// One warp per listed cell: histogram of the 64 keys, exclusive scan, then a
// stable scatter 32 particles at a time (rank among equal keys of the chunk
// by match masks, chunks in order).
__global__ void __launch_bounds__(256) pp_dense_sort_kernel(const uint16_t *off0, const uint16_t *off1,
                                                            const uint16_t *off2, const int32_t *count,
                                                            const int32_t *start, const int32_t *list,
                                                            const int *list_n, float4 *pos, int32_t *perm) {
    __shared__ int hist[8][64], run[8][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nwarps_total = gridDim.x * (blockDim.x >> 5);
    const int nl = *list_n;
    const float s = 1.0f / FIX;
    for (int li = blockIdx.x * (blockDim.x >> 5) + w; li < nl; li += nwarps_total) {
        const int c = list[li];
        const int st = start[c], cnt = count[c];
        hist[w][lane] = 0;
        hist[w][lane + 32] = 0;
        __syncwarp();
        for (int j = lane; j < cnt; j += 32)
            atomicAdd(&hist[w][subcell_key(off0[st + j], off1[st + j], off2[st + j])], 1);
        __syncwarp();
        // exclusive scan of 64 bins: lane holds bins 2 lane, 2 lane + 1
        const int h0 = hist[w][2 * lane], h1 = hist[w][2 * lane + 1];
        int incl = h0 + h1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int ex = incl - h0 - h1;
        run[w][2 * lane] = ex;
        run[w][2 * lane + 1] = ex + h0;
        __syncwarp();
        for (int j0 = 0; j0 < cnt; j0 += 32) {
            const int j = j0 + lane;
            const bool ok = j < cnt;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const unsigned o0 = off0[st + j], o1 = off1[st + j], o2 = off2[st + j];
                const int k = subcell_key(o0, o1, o2);
                const unsigned peers = __match_any_sync(act, k);
                const int rank = __popc(peers & ((1u << lane) - 1u));
                const int slot = run[w][k] + rank;
                __syncwarp(act);
                if (rank == 0) run[w][k] += __popc(peers);
                pos[st + slot] = make_float4((float)o0 * s, (float)o1 * s, (float)o2 * s, __int_as_float(c));
                perm[st + slot] = st + j;
            }
            __syncwarp();
        }
    }
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

// Far-pair factor R_PP(r)/r for b_pp <= r < b_cut (Eq. PP), IOS-cell units,
// branch-free.  Where r >= b_pp the first term of R_PP is 1/r^2 and the
// difference is written as m(u)/r^2 with u = r/b_cut: for u >= 1/2 the
// outer-shell branch of Eq. (refforce) gives r^2 (1/r^2 - R) =
// v^5 (192/5 - 416/5 v + 2048/35 v^2 - 64/5 v^3), v = 1 - u (an exact
// polynomial shift, free of cancellation near the cutoff); below u = 1/2 the
// inner branch gives 1 - 64/5 u^3 + 256/5 u^5 - 32 u^6 - 1536/35 u^7 + 192/5 u^8.
// Pairs closer than b_pp (and r = 0) get 0 here; close_pair() handles them.
__device__ __forceinline__ float far_pair(float r2, float inv_bcut, float bpp2) {
    const float rinv = rsqrtf(r2);
    const float u = r2 * rinv * inv_bcut;
    const float v = 1.0f - u;
    const float v2 = v * v;
    const float m_out = v2 * v2 * v * (192.0f / 5.0f + v * (-416.0f / 5.0f + v * (2048.0f / 35.0f - 64.0f / 5.0f * v)));
    const float u2 = u * u;
    const float m_in = 1.0f + u2 * u * (-64.0f / 5.0f + u2 * (256.0f / 5.0f + u * (-32.0f + u * (-1536.0f / 35.0f + 192.0f / 5.0f * u))));
    const float g = (u >= 0.5f ? m_out : m_in) * (rinv * rinv * rinv);
    return r2 >= bpp2 ? g : 0.0f;
}

// R_PP(r)/r for 0 < r < b_pp: both terms of Eq. PP are softened.
__device__ __forceinline__ float close_pair(float r2, float inv_bpp, float inv_bcut) {
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    return (ref_force_scaled(r * inv_bpp) * inv_bpp * inv_bpp - ref_force_scaled(r * inv_bcut) * inv_bcut * inv_bcut) *
           rinv;
}

// Sources of a warp whose 32 targets lie in one row of cells, x in [xa, xb]:
// for each of the 9 (dz, dy) rows, the cells xa-1 .. xb+1 as a main range and
// at most one wrapped cell, flattened into one stream.  Stream position p of
// segment s is particle beg[s] + p - cum[s]; its x coordinate in the warp's
// frame (cell xa at 0) is (cell id - adj[s]) + off_x.
constexpr int PP_SEGS = 18;
struct WarpSegs {
    int beg[PP_SEGS];
    int adj[PP_SEGS];
    int cum[PP_SEGS + 2];
};

// The widest warp (cells beyond the first) that takes the shared-stream path
// is a runtime parameter (PPParams.wmax, the context's pp_wmax, 16 unless an
// ensemble's autotuner chose another): its lanes test (w + 3) / 3 times their
// own candidates, still cheaper than the per-lane walk up to about w = 16 over
// the 256^3 run (at full occupancy w = 8, 12, 16 and 24 lie within 2 % of each
// other).

struct PPWarpShared {
    struct {
        float4 buf[64];   // staged sources of the union path
        WarpSegs seg;
        float box[8];     // the warp's target bounding box (lo x, y, z, hi x, y, z) and largest squared range
    } u;
};

struct PPShared {
    PPWarpShared w[PP_WARPS_CTA];
};

// Stage stream position p (far-away point past the end).  s: the lane's
// running segment index (positions a lane stages only increase).
__device__ __forceinline__ float4 stage_source(const PPParams &P, const WarpSegs &W, int p, int &s) {
    if (p >= W.cum[PP_SEGS]) return make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.0f);
    while (p >= W.cum[s + 1]) ++s;
    const float4 q = __ldg(&P.pos[W.beg[s] + (p - W.cum[s])]);
    const int row = s >> 1;   // (dz + 1) * 3 + (dy + 1)
    return make_float4((float)(__float_as_int(q.w) - W.adj[s]) + q.x, q.y + (float)(row % 3), q.z + (float)(row / 3),
                       0.0f);
}

// Candidate test of 32 staged sources: bit (31 - k) set where source k is
// closer than b_cut (sign of r^2 - b_cut^2, shifted in).
__device__ __forceinline__ unsigned test32(const float4 *S, float mx, float my, float mz, float bcut2) {
    unsigned m = 0u;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float4 q = S[k];
        const float rx = q.x - mx, ry = q.y - my, rz = q.z - mz;
        const float d = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, -bcut2)));
        m = __funnelshift_l(__float_as_uint(d), m, 1);
    }
    return m;
}

// Build the warp's segment table; returns the stream length.
__device__ int build_segments(const PPParams &P, WarpSegs &W, int c0, int xa, int xb) {
    const int lane = threadIdx.x & 31;
    const int n = P.n_ios;
    const int cz = c0 / (n * n), cy = (c0 / n) % n;
    // segment table: lane 2*row + which
    int len = 0;
    if (lane < PP_SEGS) {
        const int row = lane >> 1, which = lane & 1;
        const int dz = row / 3 - 1, dy = row % 3 - 1;
        const int rb = (wrap(cz + dz, n) * n + wrap(cy + dy, n)) * n;
        int beg = 0, adj = rb + xa;
        if (which == 0) {
            const int lo = xa > 0 ? xa - 1 : 0, hi = xb < n - 1 ? xb + 1 : n - 1;
            beg = __ldg(&P.start[rb + lo]);
            len = __ldg(&P.start[rb + hi]) + __ldg(&P.count[rb + hi]) - beg;
        } else if (xa == 0) {
            beg = __ldg(&P.start[rb + n - 1]);
            len = __ldg(&P.count[rb + n - 1]);
            adj += n;
        } else if (xb == n - 1) {
            beg = __ldg(&P.start[rb]);
            len = __ldg(&P.count[rb]);
            adj -= n;
        }
        W.beg[lane] = beg;
        W.adj[lane] = adj;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane < PP_SEGS) W.cum[lane + 1] = incl;
    if (lane == 0) W.cum[0] = 0;
    if (lane == PP_SEGS) W.cum[PP_SEGS + 1] = 0x7fffffff;
    __syncwarp();
    return W.cum[PP_SEGS];
}

// Test of 32 staged sources by every lane and evaluation of the set bits (the
// pairs in range), far pairs first, the rare pairs closer than b_pp after.
__device__ __forceinline__ void eval32(const float4 *S, float mx, float my, float mz, float bcut2, float ibc,
                                       float bpp2, float ibp, float coef, bool has, Sum3 &a, unsigned &pairs) {
    unsigned m = has ? test32(S, mx, my, mz, bcut2) : 0u;
    pairs += __popc(m);
    float px = 0.f, py = 0.f, pz = 0.f;
    unsigned cm = 0u;   // pairs closer than b_pp
    while (m) {
        const int k = __clz(m);
        const unsigned bit = 0x80000000u >> k;
        m ^= bit;
        const float4 q = S[k];
        const float rx = q.x - mx, ry = q.y - my, rz = q.z - mz;
        const float r2 = rx * rx + ry * ry + rz * rz;
        const float g = far_pair(r2, ibc, bpp2);
        if (r2 < bpp2) cm |= bit;
        px = fmaf(g, rx, px);
        py = fmaf(g, ry, py);
        pz = fmaf(g, rz, pz);
    }
    if (__any_sync(0xffffffffu, cm != 0u)) {
        while (cm) {
            const int k = __clz(cm);
            cm ^= 0x80000000u >> k;
            const float4 q = S[k];
            const float rx = q.x - mx, ry = q.y - my, rz = q.z - mz;
            const float r2 = rx * rx + ry * ry + rz * rz;
            if (r2 > 0.0f) {
                const float g = close_pair(r2, ibp, ibc);
                px = fmaf(g, rx, px);
                py = fmaf(g, ry, py);
                pz = fmaf(g, rz, pz);
            } else {
                --pairs;   // the target itself, or a coincident particle: no pair force
            }
        }
    }
    a.add_block(coef * px, coef * py, coef * pz);
}

// Warps inside one row of cells share one source stream (the cells xa-1 ..
// xb+1 of the 9 rows around it).  Each source is staged once by one lane and
// kept only if it lies within the warp's largest PP range of the bounding box
// of the warp's targets (no pair of it can be in range otherwise); the kept
// sources are packed in shared memory and every lane tests and evaluates them
// 32 at a time.  The target itself is in the stream and drops out at r = 0.
__device__ void union_path(const PPParams &P, const WarpSegs &W, float4 *S, float *box, int64_t i, bool has, int c0,
                           int xa, float4 me, float bcut2, float ibc, Sum3 &a, unsigned &pairs, unsigned &cands) {
    (void)i;
    const int lane = threadIdx.x & 31;
    const int n = P.n_ios;
    const int total = W.cum[PP_SEGS];
    const int cx = (has ? __float_as_int(me.w) : c0) % n;
    const float mx = (float)(cx - xa) + me.x, my = me.y + 1.0f, mz = me.z + 1.0f;
    const float bpp2 = P.bpp2, ibp = P.inv_bpp;
    // bounding box of the warp's targets and the largest squared range
    float lx = has ? mx : 1e30f, ly = has ? my : 1e30f, lz = has ? mz : 1e30f;
    float hx = has ? mx : -1e30f, hy = has ? my : -1e30f, hz = has ? mz : -1e30f;
    float reach2 = has ? bcut2 : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        reach2 = fmaxf(reach2, __shfl_xor_sync(0xffffffffu, reach2, o));
    }
    // kept in the warp's shared memory: fewer live registers in the loop
    if (lane == 0) {
        box[0] = lx; box[1] = ly; box[2] = lz;
        box[3] = hx; box[4] = hy; box[5] = hz;
        box[6] = reach2;
    }
    __syncwarp();
    int fill = 0, sa = 0;
    for (int b0 = 0; b0 < total; b0 += 32) {
        const float4 q = stage_source(P, W, b0 + lane, sa);
        const float dx = fmaxf(fmaxf(box[0] - q.x, q.x - box[3]), 0.0f);
        const float dy = fmaxf(fmaxf(box[1] - q.y, q.y - box[4]), 0.0f);
        const float dz = fmaxf(fmaxf(box[2] - q.z, q.z - box[5]), 0.0f);
        const bool keep = dx * dx + dy * dy + dz * dz < box[6];
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) S[fill + __popc(km & ((1u << lane) - 1u))] = q;
        fill += __popc(km);
        __syncwarp();
        if (fill >= 32) {
            if (has) cands += 32u;
            eval32(S, mx, my, mz, bcut2, ibc, bpp2, ibp, P.coef, has, a, pairs);
            __syncwarp();
            const float4 t = S[32 + lane];
            if (32 + lane < fill) S[lane] = t;
            fill -= 32;
            __syncwarp();
        }
    }
    if (fill > 0) {
        if (lane >= fill) S[lane] = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.0f);
        __syncwarp();
        if (has) cands += (unsigned)fill;
        eval32(S, mx, my, mz, bcut2, ibc, bpp2, ibp, P.coef, has, a, pairs);
    }
    __syncwarp();
}

// Warps whose targets span several rows or a wide x range (sparse regions):
// each lane walks its own 27 cells as 9 row ranges and evaluates the pairs in
// range as it meets them.  Plain nested loops keep the loads pipelined.  (A
// per-lane queue of the pairs in range, evaluated when full, measured 2x
// slower over the 256^3 run: lanes of warps straddling two rows of a dense
// region fill their queues at different steps and evaluate them one at a
// time; skipping the rows and end cells beyond the range saved 6 % of the
// candidates at z = 49 and cost more than that.)
__device__ void lane_path(const PPParams &P, bool has, int c, float4 me, float bcut2, float ibc, Sum3 &a,
                          unsigned &pairs, unsigned &cands) {
    if (!has) return;
    const int n = P.n_ios;
    const int cx = c % n, cy = (c / n) % n, cz = c / (n * n);
    const float bpp2 = P.bpp2, ibp = P.inv_bpp;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
            const int64_t r = ((int64_t)wrap(cz + dz, n) * n + wrap(cy + dy, n)) * n;
            const RowRanges rr(P, r, cx, n);
            cands += rr.size();
            const float fdy = (float)dy, fdz = (float)dz;
            float px = 0.f, py = 0.f, pz = 0.f;
            for (int sgi = 0; sgi < rr.nseg; ++sgi) {
#pragma unroll 4
                for (int j = rr.beg[sgi]; j < rr.end[sgi]; ++j) {
                    const float4 q = __ldg(&P.pos[j]);
                    const float fdx = (float)(rr.base[sgi] + (j >= rr.b1[sgi]) + (j >= rr.b2[sgi]));
                    const float rx = (fdx + q.x) - me.x;
                    const float ry = (fdy + q.y) - me.y;
                    const float rz = (fdz + q.z) - me.z;
                    const float r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 < bcut2 && r2 > 0.0f) {
                        float g = far_pair(r2, ibc, bpp2);
                        if (__builtin_expect(r2 < bpp2, 0)) g = close_pair(r2, ibp, ibc);   // rare
                        px = fmaf(g, rx, px);
                        py = fmaf(g, ry, py);
                        pz = fmaf(g, rz, pz);
                        ++pairs;
                    }
                }
            }
            a.add_block(P.coef * px, P.coef * py, P.coef * pz);
        }
}

// ---------------------------------------------------------------- adjoint
// d(R(r, b) b^2)/du of Eq. (refforce), u = r/b < 1 (derivative of each branch).
__device__ __forceinline__ float ref_force_deriv_scaled(float u) {
    if (u < 0.5f)
        return 64.0f / 5.0f + u * u * (-768.0f / 5.0f + u * (128.0f + u * (1536.0f / 7.0f - 1152.0f / 5.0f * u)));
    return -6.0f / (35.0f * u * u * u) +
           (256.0f / 5.0f + u * (-192.0f + u * (768.0f / 5.0f + u * (128.0f + u * (-1536.0f / 7.0f + 384.0f / 5.0f * u)))));
}

// For the pair term g(r) d of the PP force (g = R_PP(r)/r, IOS-cell units):
// gc = g(r) and gp = g'(r)/r, so that the pair's Jacobian block is
// gc I + gp d d^T.  Far pairs use the shell polynomial m(u) of far_pair and
// its derivative; pairs closer than b_pp the two-term formula and its
// derivative.
__device__ __forceinline__ void pp_jacobian_pair(float r2, float inv_bpp, float inv_bcut, float bpp2, float &gc,
                                                 float &gp) {
    const float rinv = rsqrtf(r2);
    if (r2 >= bpp2) {
        const float u = r2 * rinv * inv_bcut;
        float m, dm;
        if (u >= 0.5f) {
            const float v = 1.0f - u, v2 = v * v, v4 = v2 * v2;
            m = v4 * v * (192.0f / 5.0f + v * (-416.0f / 5.0f + v * (2048.0f / 35.0f - 64.0f / 5.0f * v)));
            dm = -v4 * (192.0f + v * (-2496.0f / 5.0f + v * (2048.0f / 5.0f - 512.0f / 5.0f * v)));
        } else {
            const float u2 = u * u;
            m = 1.0f + u2 * u * (-64.0f / 5.0f + u2 * (256.0f / 5.0f + u * (-32.0f + u * (-1536.0f / 35.0f + 192.0f / 5.0f * u))));
            dm = u2 * (-192.0f / 5.0f + u2 * (256.0f + u * (-192.0f + u * (-1536.0f / 5.0f + 1536.0f / 5.0f * u))));
        }
        const float r3 = rinv * rinv * rinv;
        gc = m * r3;
        gp = rinv * r3 * (dm * inv_bcut - 3.0f * m * rinv);
    } else {
        const float r = r2 * rinv;
        gc = (ref_force_scaled(r * inv_bpp) * inv_bpp * inv_bpp - ref_force_scaled(r * inv_bcut) * inv_bcut * inv_bcut) *
             rinv;
        const float dr = ref_force_deriv_scaled(r * inv_bpp) * inv_bpp * inv_bpp * inv_bpp -
                         ref_force_deriv_scaled(r * inv_bcut) * inv_bcut * inv_bcut * inv_bcut;
        gp = (dr - gc) * rinv * rinv;
    }
}

struct VjpIO {
    const float *v0, *v1, *v2;
    float *w0, *w1, *w2;
    float scale;   // coef / s_ios: Jacobian in cell units to d/dx in Mpc/h
};

// PP part of the vector-Jacobian product: w_i += sum_j A_ij (v_j - v_i) with
// A_ij = g I + (g'/r) d d^T (the force's Jacobian blocks are symmetric).
// Warps are dispatched as in the force: a warp inside one narrow row shares a
// source stream (positions and v_j staged together, the candidate test and
// set-bit evaluation of the force), other warps walk each lane's 27 cells.

__device__ __forceinline__ void jacobian_term(float rx, float ry, float rz, float r2, float4 vj, float vix, float viy,
                                              float viz, const PPParams &P, float &px, float &py, float &pz) {
    float gc, gp;
    pp_jacobian_pair(r2, P.inv_bpp, P.inv_bcut, P.bpp2, gc, gp);
    const float dvx = vj.x - vix, dvy = vj.y - viy, dvz = vj.z - viz;
    const float dd = gp * (rx * dvx + ry * dvy + rz * dvz);
    px += gc * dvx + dd * rx;
    py += gc * dvy + dd * ry;
    pz += gc * dvz + dd * rz;
}

__device__ void lane_vjp(const PPParams &P, const VjpIO &V, bool has, int c, float4 me, float vix, float viy,
                         float viz, Sum3 &a) {
    if (!has) return;
    const int n = P.n_ios;
    const int cx = c % n, cy = (c / n) % n, cz = c / (n * n);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
            const int64_t r = ((int64_t)wrap(cz + dz, n) * n + wrap(cy + dy, n)) * n;
            const RowRanges rr(P, r, cx, n);
            const float fdy = (float)dy, fdz = (float)dz;
            float px = 0.f, py = 0.f, pz = 0.f;
            for (int sgi = 0; sgi < rr.nseg; ++sgi) {
                for (int j = rr.beg[sgi]; j < rr.end[sgi]; ++j) {
                    const float4 q = __ldg(&P.pos[j]);
                    const float fdx = (float)(rr.base[sgi] + (j >= rr.b1[sgi]) + (j >= rr.b2[sgi]));
                    const float rx = (fdx + q.x) - me.x;
                    const float ry = (fdy + q.y) - me.y;
                    const float rz = (fdz + q.z) - me.z;
                    const float r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 < P.bcut2 && r2 > 0.0f) {
                        const float4 vj = make_float4(__ldg(&V.v0[j]), __ldg(&V.v1[j]), __ldg(&V.v2[j]), 0.f);
                        jacobian_term(rx, ry, rz, r2, vj, vix, viy, viz, P, px, py, pz);
                    }
                }
            }
            a.add_block(px, py, pz);
        }
}

// The particle index of stream position p (-1 past the end); s as in stage_source.
__device__ __forceinline__ int stream_index(const WarpSegs &W, int p, int &s) {
    if (p >= W.cum[PP_SEGS]) return -1;
    while (p >= W.cum[s + 1]) ++s;
    return W.beg[s] + (p - W.cum[s]);
}

__device__ void union_vjp(const PPParams &P, const VjpIO &V, const WarpSegs &W, float4 *S, float4 *SV, int64_t i,
                          bool has, int c0, int xa, float4 me, float vix, float viy, float viz, Sum3 &a) {
    const int lane = threadIdx.x & 31;
    const int n = P.n_ios;
    const int total = W.cum[PP_SEGS];
    const int pself = has ? W.cum[8] + (int)(i - W.beg[8]) : -1000;
    const int cx = (has ? __float_as_int(me.w) : c0) % n;
    const float mx = (float)(cx - xa) + me.x, my = me.y + 1.0f, mz = me.z + 1.0f;
    const float bcut2 = P.bcut2;
    int sa = 0, sb = 0, ta = 0, tb = 0;
    for (int b0 = 0; b0 < total; b0 += 64) {
        S[lane] = stage_source(P, W, b0 + lane, sa);
        S[32 + lane] = stage_source(P, W, b0 + 32 + lane, sb);
        const int ja = stream_index(W, b0 + lane, ta), jb = stream_index(W, b0 + 32 + lane, tb);
        SV[lane] = ja >= 0 ? make_float4(__ldg(&V.v0[ja]), __ldg(&V.v1[ja]), __ldg(&V.v2[ja]), 0.f)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        SV[32 + lane] = jb >= 0 ? make_float4(__ldg(&V.v0[jb]), __ldg(&V.v1[jb]), __ldg(&V.v2[jb]), 0.f)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        unsigned mh = test32(S, mx, my, mz, bcut2), ml = test32(S + 32, mx, my, mz, bcut2);
        const int ts = pself - b0;
        if (ts >= 0 && ts < 32) mh &= ~(0x80000000u >> ts);
        if (ts >= 32 && ts < 64) ml &= ~(0x80000000u >> (ts - 32));
        if (!has) mh = ml = 0u;
        float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned m = h ? ml : mh;
            const float4 *SB = S + 32 * h, *SVB = SV + 32 * h;
            while (m) {
                const int k = __clz(m);
                m ^= 0x80000000u >> k;
                const float4 q = SB[k];
                const float rx = q.x - mx, ry = q.y - my, rz = q.z - mz;
                const float r2 = rx * rx + ry * ry + rz * rz;
                if (r2 > 0.0f) jacobian_term(rx, ry, rz, r2, SVB[k], vix, viy, viz, P, px, py, pz);
            }
        }
        a.add_block(px, py, pz);
        __syncwarp();
    }
}

// the adjoint's product keeps the force's default shared-stream width
constexpr int PP_WMAX_VJP = 16;

struct PPVjpWarpShared {
    float4 buf[64];   // staged source positions
    float4 vbuf[64];  // and their v_j
    WarpSegs seg;
};

#ifndef PPV_MINB
#define PPV_MINB 1
#endif
__global__ void __launch_bounds__(PP_CTA, PPV_MINB) pp_vjp_kernel(PPParams P, VjpIO V) {
    __shared__ PPVjpWarpShared sh[PP_WARPS_CTA];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int wib = threadIdx.x >> 5;
    const bool has = i < P.N;
    const int n = P.n_ios;
    const float4 me = has ? P.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int c = has ? __float_as_int(me.w) : -1;
    const int c0 = __shfl_sync(0xffffffffu, c, 0);
    if (!has) c = c0;
    const int c31 = __reduce_max_sync(0xffffffffu, c);
    const int xa = c0 % n, xb = c31 % n;
    const bool one_row = (c0 / n) == (c31 / n) && xb - xa <= PP_WMAX_VJP && xb - xa + 3 <= n;
    const float vix = has ? V.v0[i] : 0.f, viy = has ? V.v1[i] : 0.f, viz = has ? V.v2[i] : 0.f;
    Sum3 a;
    if (one_row) {
        build_segments(P, sh[wib].seg, c0, xa, xb);
        union_vjp(P, V, sh[wib].seg, sh[wib].buf, sh[wib].vbuf, i, has, c0, xa, me, vix, viy, viz, a);
    } else {
        lane_vjp(P, V, has, c, me, vix, viy, viz, a);
    }
    if (has) {
        V.w0[i] += V.scale * (a.x - a.cx);
        V.w1[i] += V.scale * (a.y - a.cy);
        V.w2[i] += V.scale * (a.z - a.cz);
    }
}

// Full occupancy (16 CTAs of 4 warps, 32 registers): the per-lane walk is
// bound by load latency, and more resident warps hide more of it than the
// spilled registers cost (measured 14-16 % faster over the 256^3 run than
// 3 CTAs of 8 warps at 64 registers).
#ifndef PP_MINB
#define PP_MINB 16
#endif
// The targets of one block of PP_CTA slots: [block * PP_CTA, block * PP_CTA + PP_CTA).
// COUNT: accumulate the work counters (off unless asked for: the two counters
// live through the whole walk and, within the 32-register budget, cost up to
// a fifth of the sparse-region time).
template <bool PM3, bool COUNT>
__device__ __forceinline__ void pp_block(const PPParams &P, int64_t block, PPShared &sh) {
    const int64_t i = block * PP_CTA + threadIdx.x;
    const int wib = threadIdx.x >> 5;
    const bool has = i < P.N;
    const int n = P.n_ios;
    const float4 me = has ? P.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int c = has ? __float_as_int(me.w) : -1;
    const int c0 = __shfl_sync(0xffffffffu, c, 0);
    if (!has) c = c0;
    // cells are non-decreasing along the warp (padding lanes repeat lane 0's):
    // lane 0 and the largest cell bound its extent
    const int c31 = __reduce_max_sync(0xffffffffu, c);
    const int xa = c0 % n, xb = c31 % n;
    // warps inside one row, at most wmax + 1 cells wide, share a source stream
    const bool one_row = (c0 / n) == (c31 / n) && xb - xa <= P.wmax && xb - xa + 3 <= n;
    if (one_row) build_segments(P, sh.w[wib].u.seg, c0, xa, xb);
    // PP range of this target: b_3 inside a refined subtile of the third level
    float bcut2 = P.bcut2, ibc = P.inv_bcut;
    if (PM3 && has) {
        const int T = P.pm3_T;
        const int s = ((c / (n * n)) / T * P.pm3_ns + ((c / n) % n) / T) * P.pm3_ns + (c % n) / T;
        if (__ldg(&P.pm3_slot[s]) >= 0) {
            bcut2 = P.bcut2_3;
            ibc = P.inv_bcut_3;
        }
    }
    Sum3 a;
    unsigned pairs = 0, cands = 0;
    if (one_row)
        union_path(P, sh.w[wib].u.seg, sh.w[wib].u.buf, sh.w[wib].u.box, i, has, c0, xa, me, bcut2, ibc, a, pairs,
                   cands);
    else
        lane_path(P, has, c, me, bcut2, ibc, a, pairs, cands);
    if (has) finish(P, P.perm[i], a.x - a.cx, a.y - a.cy, a.z - a.cz);
    if constexpr (COUNT) {
        add_stats(P.stats, pairs, cands);
        if (!one_row) add_stats(P.stats + 2, pairs, cands);   // warp-uniform
    }
}

template <bool PM3, bool COUNT>
__global__ void __launch_bounds__(PP_CTA, PP_MINB) pp_kernel(PPParams P) {
    __shared__ PPShared sh;
    pp_block<PM3, COUNT>(P, blockIdx.x, sh);
}

// ------------------------------------------------- ensemble: one persistent PP
// kernel over many boxes.  Work items are (box, block) pairs; a per-step cost
// estimate orders them largest first (the load balancing of Sec. 2.2.3: work
// sorted by its density, taken in that order by whoever is free), and
// persistent CTAs take the next item from a device counter.  The host
// publishes each step's queue with a stream-ordered write of the step's epoch;
// the kernel waits for that epoch for at most timeout_ns (%globaltimer), then
// records CUBE2_ERR_TIMEOUT in the queue's status word and returns.
struct PPQueueDev {
    int head;        // next item to take
    int count;       // items of this step
    int ready;       // epoch published by the host
    int status;      // sticky ST_TIMEOUT
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// cost[k] of item k (box b = item_box[k], block j = k - base[b]): the number of
// particles in the IOS cells of its targets, a proxy of the block's pair count
__global__ void __launch_bounds__(256) pp_item_cost_kernel(const PPParams *__restrict__ boxes,
                                                            const int32_t *__restrict__ item_box,
                                                            const int32_t *__restrict__ base, int n_items,
                                                            unsigned *__restrict__ cost) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_items) return;
    const int b = item_box[k];
    const PPParams &P = boxes[b];
    const int64_t i0 = (int64_t)(k - base[b]) * PP_CTA;
    const int64_t i1 = min(i0 + PP_CTA, P.N);
    unsigned s = 0;
    for (int64_t i = i0; i < i1; ++i) s += (unsigned)__ldg(&P.count[__float_as_int(__ldg(&P.pos[i]).w)]);
    cost[k] = s;
}

// One CTA: items bucketed by floor(log2(cost + 1)), largest bucket first,
// written to order[]; the queue's counters are reset for the step.
__global__ void __launch_bounds__(1024) pp_item_order_kernel(const unsigned *__restrict__ cost, int n_items,
                                                             int32_t *__restrict__ order, PPQueueDev *q) {
    __shared__ int hist[33], offs[33];
    if (threadIdx.x < 33) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < n_items; k += blockDim.x) atomicAdd(&hist[32 - __clz(cost[k] + 1u)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 32; b >= 0; --b) {
            offs[b] = run;
            run += hist[b];
        }
        q->head = 0;
        q->count = n_items;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_items; k += blockDim.x) order[atomicAdd(&offs[32 - __clz(cost[k] + 1u)], 1)] = k;
}

__global__ void __launch_bounds__(PP_CTA, PP_MINB) pp_persistent_kernel(const PPParams *__restrict__ boxes,
                                                                       const int32_t *__restrict__ item_box,
                                                                       const int32_t *__restrict__ base,
                                                                       const int32_t *__restrict__ order,
                                                                       PPQueueDev *q, int epoch,
                                                                       unsigned long long timeout_ns) {
    __shared__ PPShared sh;
    __shared__ int s_item, s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = global_ns();
        while (atomicAdd(&q->ready, 0) != epoch) {
            if (atomicAdd(&q->status, 0) != 0 || global_ns() - t0 > timeout_ns) {
                atomicOr(&q->status, ST_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(2000);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const int count = *((volatile int *)&q->count);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&q->head, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= count) break;
        const int k = order[item];
        const int b = item_box[k];
        pp_block<false, false>(boxes[b], (int64_t)(k - base[b]), sh);
    }
}

}  // namespace

static PPParams pp_params(cube2_ctx *ctx, const cube2_particles *p, int accumulate, float kick);

cudaError_t launch_pp_vjp(cube2_ctx *ctx, const cube2_particles *p, const float *const v[3], float *const w[3]) {
    if (ctx->N == 0) return cudaSuccess;
    PPParams P = pp_params(ctx, p, 1, 0.0f);
    VjpIO V{};
    V.v0 = v[0]; V.v1 = v[1]; V.v2 = v[2];
    V.w0 = w[0]; V.w1 = w[1]; V.w2 = w[2];
    V.scale = (float)((double)P.coef / ctx->s_ios);
    ProfScope prof(ctx, P_PP_VJP, 0);
    const int nblocks = (int)((ctx->N + PP_CTA - 1) / PP_CTA);
    prep_positions_kernel<<<(unsigned)nblocks, PP_CTA, 0, ctx->stream>>>(p->off[0], p->off[1], p->off[2], ctx->cellid,
                                                                       ctx->pos4, nullptr, ctx->N);
    pp_vjp_kernel<<<(unsigned)nblocks, PP_CTA, 0, ctx->stream>>>(P, V);
    ctx->launches += 2;
    return cudaGetLastError();
}

static PPParams pp_params(cube2_ctx *ctx, const cube2_particles *p, int accumulate, float kick) {
    PPParams P{};
    P.pos = ctx->pos4;
    P.perm = ctx->pp_perm;
    P.count = p->count; P.start = p->start;
    P.acc0 = p->acc[0]; P.acc1 = p->acc[1]; P.acc2 = p->acc[2];
    if (ctx->vel32) {   // FP16 storage: the second kick updates the step's FP32 working copy
        P.vel0 = ctx->vel32; P.vel1 = ctx->vel32 + ctx->N; P.vel2 = ctx->vel32 + 2 * ctx->N;
    } else {
        P.vel0 = p->vel[0]; P.vel1 = p->vel[1]; P.vel2 = p->vel[2];
    }
    P.stats = ctx->pp_stats;
    P.N = ctx->N;
    P.n_ios = ctx->n_ios;
    P.accumulate = accumulate;
    const double s = ctx->s_ios;
    P.inv_bpp = (float)(s / ctx->cfg.b_pp);
    P.inv_bcut = (float)(s / ctx->b_range);
    P.bcut2 = (float)((ctx->b_range / s) * (ctx->b_range / s));
    P.bpp2 = (float)((ctx->cfg.b_pp / s) * (ctx->cfg.b_pp / s));
    const double vp = ctx->cfg.box * ctx->cfg.box * ctx->cfg.box / (double)ctx->N;
    P.coef = (float)(vp / (4.0 * 3.14159265358979323846) / (s * s));
    P.kick = kick;
    P.status = ctx->dev_status;
    P.wmax = ctx->pp_wmax;
    if (ctx->pm3.on) {
        P.pm3_slot = ctx->pm3.slot;
        P.pm3_T = ctx->pm3.T;
        P.pm3_ns = ctx->pm3.ns;
        P.bcut2_3 = (float)((ctx->pm3.b3 / s) * (ctx->pm3.b3 / s));
        P.inv_bcut_3 = (float)(s / ctx->pm3.b3);
    }
    return P;
}

cudaError_t launch_pp(cube2_ctx *ctx, const cube2_particles *p, int accumulate, float kick) {
    PPParams P = pp_params(ctx, p, accumulate, kick);
    if (ctx->N == 0) return cudaSuccess;
    const int nblocks = (int)((ctx->N + PP_CTA - 1) / PP_CTA);
    {
        ProfScope prof(ctx, P_PREP, 0);
        prep_positions_kernel<<<(unsigned)nblocks, PP_CTA, 0, ctx->stream>>>(p->off[0], p->off[1], p->off[2],
                                                                           ctx->cellid, ctx->pos4, ctx->pp_perm, ctx->N);
    }
    {
        ProfScope prof(ctx, P_PP_ORDER, 0);
        cudaMemsetAsync(ctx->big_n, 0, sizeof(int), ctx->stream);
        pp_dense_list_kernel<<<(unsigned)((ctx->n_cells + 255) / 256), 256, 0, ctx->stream>>>(p->count, ctx->n_cells,
                                                                                          ctx->big, ctx->big_n);
        pp_dense_sort_kernel<<<(unsigned)(ctx->num_sms * 8), 256, 0, ctx->stream>>>(
            p->off[0], p->off[1], p->off[2], p->count, p->start, ctx->big, ctx->big_n, ctx->pos4, ctx->pp_perm);
    }
    if (ctx->defer_pp) {   // an ensemble's persistent kernel runs this box's PP later
        static_assert(sizeof(PPParams) <= sizeof(ctx->pp_deferred), "deferred PP parameters");
        memcpy(ctx->pp_deferred, &P, sizeof P);
        ctx->launches += 3;
        return cudaGetLastError();
    }
    {
        ProfScope prof(ctx, P_PP, 0);
        if (P.pm3_slot)
            (ctx->pp_count ? pp_kernel<true, true> : pp_kernel<true, false>)<<<(unsigned)nblocks, PP_CTA, 0,
                                                                              ctx->stream>>>(P);
        else
            (ctx->pp_count ? pp_kernel<false, true> : pp_kernel<false, false>)<<<(unsigned)nblocks, PP_CTA, 0,
                                                                                ctx->stream>>>(P);
    }
    ctx->launches += 4;
    return cudaGetLastError();
}

size_t pp_params_bytes() { return sizeof(PPParams); }

cudaError_t launch_pp_persistent_step(cudaStream_t st, const void *boxes, const int32_t *item_box,
                                      const int32_t *base, int n_items, unsigned *cost, int32_t *order, void *queue,
                                      const int *publish_host, int epoch, unsigned long long timeout_ns, int grid) {
    const PPParams *B = static_cast<const PPParams *>(boxes);
    PPQueueDev *q = static_cast<PPQueueDev *>(queue);
    pp_item_cost_kernel<<<(unsigned)((n_items + 255) / 256), 256, 0, st>>>(B, item_box, base, n_items, cost);
    pp_item_order_kernel<<<1, 1024, 0, st>>>(cost, n_items, order, q);
    // the host's publication of this step's work count
    cudaError_t e = cudaMemcpyAsync(&q->ready, publish_host, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    pp_persistent_kernel<<<(unsigned)grid, PP_CTA, 0, st>>>(B, item_box, base, order, q, epoch, timeout_ns);
    return cudaGetLastError();
}

size_t pp_queue_bytes() { return sizeof(PPQueueDev); }

}  // namespace cube2
