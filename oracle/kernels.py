"""FP64 oracle: softening profile, reference force and optimised Green's function.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; never by the product path.

Everything here restates Sec. 2.1 of the paper (CUBE2, Yu et al. 2026):

* Eq. (denprofile)  S(r, b)        density profile of a softened particle
* Eq. (refforce)    R(r, b)        force between two S-profiles, 1/r^2 for r >= b
* Eq. (Sk)          S(k, b)        Fourier transform of S(r, b)
* Eq. (Rk)          R_alpha(k)     reference force of level alpha in k-space
* Eq. (diff)        D(k)           4-point finite difference in k-space
* Eq. (Gk)          G_alpha(k)     optimised Green's function, alias sum |n_d| <= 2

Readings of the paper taken here (where it is silent or departs from the workload):

* Mass assignment is CIC, W(k) = prod_d sinc^2(k_d/2) (the paper's TSC has the
  cube); ``order`` selects the power (2 = CIC, 3 = TSC).
* D(k) is a vector: component d is i(4/3 sin k_d - 1/6 sin 2k_d).
* D.R* is the plain (bilinear) product, which makes G real:
  G = -sum_n W^2(k_n) (d.k_n) dS2(|k_n|)/|k_n|^2 / (|d|^2 [sum_n W^2(k_n)]^2),
  with d_d = 4/3 sin k_d - 1/6 sin 2k_d and dS2 = S^2(k,b_soft) - S^2(k,b_trunc),
  S(k, infinity) = 0 (b_0 = infinity for the coarsest level).
* "max(|n|) <= 2" is the Chebyshev norm: 5^3 = 125 images.
* G = 0 where |d| = 0 (k = 0 and every mode with all k_d in {0, pi}).
* Coefficients dropped by the paper are restored as follows: G ~ -S^2/k^2 solves
  lap(u) = rho in mesh units (no 4 pi); the PP term uses R/(4 pi).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


# ------------------------------------------------------------ real space
def density_profile(r, b):
    """Eq. (denprofile): S(r,b) = 48 (b/2 - r) / (pi b^4) for r < b/2, else 0."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(r < 0.5 * b, 48.0 * (0.5 * b - r) / (math.pi * b ** 4), 0.0)


def reference_force(r, b):
    """Eq. (refforce): R(r,b), magnitude of the force between two unit S-profiles."""
    r = np.asarray(r, dtype=np.float64)
    inner = (64 * r / (5 * b ** 3) - 256 * r ** 3 / (5 * b ** 5) + 32 * r ** 4 / b ** 6
             + 1536 * r ** 5 / (35 * b ** 7) - 192 * r ** 6 / (5 * b ** 8))
    with np.errstate(divide="ignore"):
        outer_shell = (3 / (35 * r ** 2) - 32 / (5 * b ** 2) + 256 * r / (5 * b ** 3)
                       - 96 * r ** 2 / b ** 4 + 256 * r ** 3 / (5 * b ** 5) + 32 * r ** 4 / b ** 6
                       - 1536 * r ** 5 / (35 * b ** 7) + 64 * r ** 6 / (5 * b ** 8))
        newton = 1.0 / r ** 2
    return np.where(r < 0.5 * b, inner, np.where(r < b, outer_shell, newton))


def reference_force_derivative(r, b):
    """dR/dr of Eq. (refforce), branch by branch (the derivative of each
    polynomial, and -2/r^3 beyond b)."""
    r = np.asarray(r, dtype=np.float64)
    inner = (64 / (5 * b ** 3) - 768 * r ** 2 / (5 * b ** 5) + 128 * r ** 3 / b ** 6
             + 1536 * r ** 4 / (7 * b ** 7) - 1152 * r ** 5 / (5 * b ** 8))
    with np.errstate(divide="ignore"):
        outer_shell = (-6 / (35 * r ** 3) + 256 / (5 * b ** 3) - 192 * r / b ** 4 + 768 * r ** 2 / (5 * b ** 5)
                       + 128 * r ** 3 / b ** 6 - 1536 * r ** 4 / (7 * b ** 7) + 384 * r ** 5 / (5 * b ** 8))
        newton = -2.0 / r ** 3
    return np.where(r < 0.5 * b, inner, np.where(r < b, outer_shell, newton))


def pp_reference(r, b_pp, b_cut):
    """Eq. (PP): R_PP(r) = R(r, b_PP) - R(r, b_cut); zero for r >= b_cut."""
    return reference_force(r, b_pp) - reference_force(r, b_cut)


# -------------------------------------------------------------- k space
# Series of 2 - 2cos x - x sin x = sum_{j>=2} (-1)^j (2j-2) x^{2j} / (2j)!,
# used below x = 1/2 where the closed form of Eq. (Sk) cancels.
_SERIES = [(-1) ** j * (2 * j - 2) / math.factorial(2 * j) for j in range(2, 14)]


def profile_transform(k, b):
    """Eq. (Sk): S(k,b) = 12/(kb/2)^4 (2 - 2cos(kb/2) - (kb/2) sin(kb/2)).

    b = None means b = infinity, where S = 0."""
    k = np.asarray(k, dtype=np.float64)
    if b is None:
        return np.zeros_like(k)
    x = 0.5 * k * b
    small = x < 0.5
    xs = np.where(small, x, 0.0)
    series = np.zeros_like(x)
    for c in reversed(_SERIES):          # Horner in x^2
        series = series * xs * xs + c
    series = 12.0 * series
    xl = np.where(small, 1.0, x)
    closed = 12.0 / xl ** 4 * (2.0 - 2.0 * np.cos(xl) - xl * np.sin(xl))
    return np.where(small, series, closed)


def assignment_transform(k, order=2):
    """W(k) per dimension: sinc(k/2)^order (order 2 = CIC, 3 = TSC)."""
    return np.sinc(np.asarray(k, dtype=np.float64) / TWO_PI) ** order


def fd_transform(k):
    """Eq. (diff) in k-space, component-wise: D_d(k) = i * fd_transform(k_d)."""
    k = np.asarray(k, dtype=np.float64)
    return 4.0 / 3.0 * np.sin(k) - 1.0 / 6.0 * np.sin(2.0 * k)


def _sin_turns(m, n):
    """sin(2 pi m / n) for integer arrays m, exact zero at multiples of pi."""
    r = np.mod(np.asarray(m, dtype=np.int64), n)
    val = np.sin(TWO_PI * r.astype(np.float64) / n)
    return np.where((2 * r) % n == 0, 0.0, val)


def fd_transform_modes(m, n):
    """fd_transform at k = 2 pi m / n, with the exact zeros at k in {0, pi}."""
    return 4.0 / 3.0 * _sin_turns(m, n) - 1.0 / 6.0 * _sin_turns(2 * np.asarray(m), n)


def half_spectrum_modes(n):
    """Integer mode numbers m_x, m_y, m_z on the rfftn layout, m in (-n/2, n/2]."""
    m = np.fft.fftfreq(n, d=1.0 / n).astype(np.int64)
    mz = m[:, None, None]
    my = m[None, :, None]
    mx = np.arange(n // 2 + 1, dtype=np.int64)[None, None, :]
    return mx, my, mz


def half_spectrum_wavenumbers(n):
    """k_x, k_y, k_z (radians per cell) on the rfftn layout [kz][ky][kx<=n/2]."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    mx = np.arange(n // 2 + 1, dtype=np.float64)
    kz = (TWO_PI / n) * m[:, None, None]
    ky = (TWO_PI / n) * m[None, :, None]
    kx = (TWO_PI / n) * mx[None, None, :]
    return kx, ky, kz


def isolation_factor(k, length):
    """1 - sinc(k L) of Eq. (isok) (Appendix A): multiplies R(k, b) when the
    reference force is truncated at r = L (isolated boundary conditions in a
    box of side >= 2L); sinc(x) = sin(x)/x.  length None or 0 = periodic (1).
    Below kL = 0.01 the Taylor series x^2/6 - x^4/120 replaces the difference."""
    if not length:
        return 1.0
    x = np.asarray(k, dtype=np.float64) * length
    small = x < 1e-2
    xs = np.where(small, 1.0, x)
    return np.where(small, x * x / 6.0 - x ** 4 / 120.0, 1.0 - np.sin(xs) / xs)


def green(n, b_soft, b_trunc=None, alias=2, order=2, iso=None):
    """Eq. (Gk) on the rfftn half spectrum [kz][ky][kx] of an n^3 mesh.

    b_soft, b_trunc are in this mesh's cells (b_trunc None = infinity); iso
    (cells, None = periodic) truncates the level's reference force at r = iso
    by Eq. (isok), each image's R(k_n) times 1 - sinc(|k_n| iso).
    Returned unnormalised: phi = irfftn(rfftn(rho) * G) (numpy's 1/n^3)."""
    kx, ky, kz = half_spectrum_wavenumbers(n)
    mx, my, mz = half_spectrum_modes(n)
    dx, dy, dz = fd_transform_modes(mx, n), fd_transform_modes(my, n), fd_transform_modes(mz, n)
    d2 = dx * dx + dy * dy + dz * dz
    shape = np.broadcast_shapes(kx.shape, ky.shape, kz.shape)
    num = np.zeros(shape)
    den = np.zeros(shape)
    images = range(-alias, alias + 1)
    for nz in images:
        knz = kz + TWO_PI * nz
        wz = assignment_transform(knz, order) ** 2
        for ny in images:
            kny = ky + TWO_PI * ny
            wy = assignment_transform(kny, order) ** 2
            for nx in images:
                knx = kx + TWO_PI * nx
                wx = assignment_transform(knx, order) ** 2
                w2 = wx * wy * wz
                kn2 = knx * knx + kny * kny + knz * knz
                safe = np.where(kn2 > 0, kn2, 1.0)
                kn = np.sqrt(safe)
                ds2 = profile_transform(kn, b_soft) ** 2 - profile_transform(kn, b_trunc) ** 2
                ds2 = ds2 * isolation_factor(kn, iso)
                # D.R*_alpha(k_n) = (i d).(i k_n dS2/|k_n|^2) = -(d.k_n) dS2/|k_n|^2
                dr = -(dx * knx + dy * kny + dz * knz) * ds2 / safe
                num += np.where(kn2 > 0, w2 * dr, 0.0)
                den += w2
    out = np.zeros(shape)
    ok = d2 > 0
    out[ok] = num[ok] / (d2[ok] * den[ok] ** 2)
    return out


def green_at(n, modes, b_soft, b_trunc=None, alias=2, order=2, iso=None):
    """Eq. (Gk) at selected modes of an n^3 mesh, without the full table.

    modes: int array (K, 3) of (m_x, m_y, m_z) in rfftn index ranges
    (m_x in [0, n/2], m_y, m_z in [0, n)).  Same arithmetic as ``green``."""
    modes = np.asarray(modes, dtype=np.int64)
    mx = modes[:, 0]
    my = np.where(modes[:, 1] <= n // 2, modes[:, 1], modes[:, 1] - n)
    mz = np.where(modes[:, 2] <= n // 2, modes[:, 2], modes[:, 2] - n)
    # numpy's fftfreq puts the Nyquist index n/2 at -n/2 on the y and z axes
    my = np.where(modes[:, 1] == n // 2, -(n // 2), my)
    mz = np.where(modes[:, 2] == n // 2, -(n // 2), mz)
    kx, ky, kz = (TWO_PI / n) * mx, (TWO_PI / n) * my, (TWO_PI / n) * mz
    dx, dy, dz = fd_transform_modes(mx, n), fd_transform_modes(my, n), fd_transform_modes(mz, n)
    d2 = dx * dx + dy * dy + dz * dz
    num = np.zeros(len(modes))
    den = np.zeros(len(modes))
    images = range(-alias, alias + 1)
    for nz in images:
        knz = kz + TWO_PI * nz
        wz = assignment_transform(knz, order) ** 2
        for ny in images:
            kny = ky + TWO_PI * ny
            wy = assignment_transform(kny, order) ** 2
            for nx in images:
                knx = kx + TWO_PI * nx
                wx = assignment_transform(knx, order) ** 2
                w2 = wx * wy * wz
                kn2 = knx * knx + kny * kny + knz * knz
                safe = np.where(kn2 > 0, kn2, 1.0)
                kn = np.sqrt(safe)
                ds2 = profile_transform(kn, b_soft) ** 2 - profile_transform(kn, b_trunc) ** 2
                ds2 = ds2 * isolation_factor(kn, iso)
                dr = -(dx * knx + dy * kny + dz * knz) * ds2 / safe
                num += np.where(kn2 > 0, w2 * dr, 0.0)
                den += w2
    out = np.zeros(len(modes))
    ok = d2 > 0
    out[ok] = num[ok] / (d2[ok] * den[ok] ** 2)
    return out


def sorted_mode_triples(n):
    """Every triple 0 <= a <= b <= c <= n/2 of absolute mode numbers, (K, 3)
    int64, in the order c-major, then b, then a."""
    m = n // 2
    c, b, a = [], [], []
    for cc in range(m + 1):
        bb, aa = np.tril_indices(cc + 1)
        c.append(np.full(bb.size, cc))
        b.append(bb)
        a.append(aa)
    return np.stack([np.concatenate(a), np.concatenate(b), np.concatenate(c)], axis=1).astype(np.int64)


def green_by_symmetry(n, b_soft, b_trunc=None, alias=2, order=2, iso=None, chunk=65536, mapper=map):
    """Eq. (Gk) on the whole rfftn half spectrum [kz][ky][kx] of an n^3 mesh,
    evaluated once per sorted triple of |m_x|, |m_y|, |m_z| with ``green_at``
    and copied to every mode of that class.

    G is even in each k_d and symmetric under permutations of the axes (the
    alias sum runs over a set of images closed under both, and W, |D|^2 and
    D.k_n are symmetric functions of the components), which tests pin on the
    full table; this is the way to the table at meshes where ``green`` itself
    is too slow.  ``mapper`` maps a function over the chunks of triples (for
    instance the map of a process pool); chunks are evaluated independently."""
    tri = sorted_mode_triples(n)
    parts = [tri[i:i + chunk] for i in range(0, len(tri), chunk)]
    args = [(n, p, b_soft, b_trunc, alias, order, iso) for p in parts]
    vals = np.concatenate(list(mapper(_green_chunk, args)))
    # class index of every half-spectrum mode, by sorting its absolute mode numbers
    mx, my, mz = half_spectrum_modes(n)
    ax = np.broadcast_to(np.abs(mx), (n, n, n // 2 + 1))
    ay = np.broadcast_to(np.abs(my), (n, n, n // 2 + 1))
    az = np.broadcast_to(np.abs(mz), (n, n, n // 2 + 1))
    s = np.sort(np.stack([ax, ay, az]), axis=0)
    a, b, c = s[0], s[1], s[2]
    cls = c * (c + 1) * (c + 2) // 6 + b * (b + 1) // 2 + a
    return vals[cls]


def _green_chunk(args):
    n, modes, b_soft, b_trunc, alias, order, iso = args
    return green_at(n, modes, b_soft, b_trunc, alias=alias, order=order, iso=iso)
