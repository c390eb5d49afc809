"""FP64 oracle: IOS decoding, integer CIC deposit, Poisson solve, 4-point FD, interpolation.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; never by the product path.

Follows the four PM steps of Sec. 2.1.2 in order: assignment (Eq. filter, CIC
reading), Poisson solve phi(k) = rho(k) G(k), force field E = D * phi with the
4-point difference of Eq. (diff) applied in real space (the paper's route,
Sec. 2.2.2), and interpolation back with the same assignment function.

Conventions (readings of the paper where it is silent):

* IOS (Sec. 2.3): particle p sits in IOS cell c (linear id, x fastest) with
  uint16 offsets; its fixed-point coordinate is X_d = c_d 2^16 + off_d, i.e.
  x_d = X_d / 2^16 IOS cells.
* A mesh level with n_mesh cells has ratio q = n_ios / n_mesh = 2^s between
  its cell and the IOS cell.  The position in mesh cells, floored to 2^-16 of
  a mesh cell, is X >> s (s >= 0) or X << -s (s < 0).
* Cell j of a mesh spans [j, j+1) with centre j + 1/2.  With t = x - 1/2 the
  CIC weights are 1 - frac(t) on floor(t) and frac(t) on floor(t) + 1, held as
  integers at scale 2^16; the 3-D weight is their exact product (<= 2^48).
* The accumulator is uint64 per cell (exact, hence order-free).  The density
  in mean-one units is rho = acc 2^-48 n_mesh^3 / N; the FFT sees the exact
  integer overdensity acc - M with M = floor(N 2^48 / n_mesh^3) (the k = 0
  mode is dropped by G(0) = 0 anyway).
* FP32 density grid (bit-exact spec shared with the GPU):
  rho32 = RN32(acc - M) * RN32(RN64(n_mesh^3/N) 2^-48), one FP32 multiply.
* The force returned is F = -grad(u) with lap(u) = delta, lengths in Mpc/h:
  F = -H_level * interp(E), E = D * phi in mesh units.
"""
from __future__ import annotations

import numpy as np

from .kernels import green

FIX = 1 << 16
HALF = 1 << 15


# ------------------------------------------------------------------ IOS
def cell_coords(count, n_ios):
    """Per-particle IOS cell coordinates (3, N) from the per-cell counts."""
    cell = np.repeat(np.arange(n_ios ** 3, dtype=np.int64), count.astype(np.int64))
    return np.stack([cell % n_ios, (cell // n_ios) % n_ios, cell // (n_ios * n_ios)])


def fixed_coords(off, count, n_ios):
    """Fixed-point coordinates X_d = c_d 2^16 + off_d (int64, (3, N))."""
    return cell_coords(count, n_ios) * FIX + off.astype(np.int64)


def positions(off, count, n_ios, box):
    """Decoded positions in Mpc/h (FP64, (3, N))."""
    return fixed_coords(off, count, n_ios).astype(np.float64) / FIX * (box / n_ios)


def level_shift(n_ios, n_mesh):
    """s with n_ios / n_mesh = 2^s."""
    if n_ios >= n_mesh:
        q, s = n_ios // n_mesh, 0
        assert q * n_mesh == n_ios
        while (1 << s) < q:
            s += 1
        assert (1 << s) == q
        return s
    q = n_mesh // n_ios
    assert q * n_ios == n_mesh
    s = 0
    while (1 << s) < q:
        s += 1
    assert (1 << s) == q
    return -s


# ---------------------------------------------------------- CIC weights
def cic_integer_weights(X, s):
    """Lower corner index and the two integer 1-D weights (scale 2^16)."""
    xm = (X >> s) if s >= 0 else (X << (-s))
    t = xm - HALF
    i0 = t >> 16                      # floor for negative t too
    f = t - (i0 << 16)
    return i0, FIX - f, f


def _corners(X, n_mesh, s):
    """Yield (flat cell index, integer weight) for the 8 CIC corners."""
    parts = [cic_integer_weights(X[d], s) for d in range(3)]
    for cz in (0, 1):
        iz = (parts[2][0] + cz) % n_mesh
        wz = parts[2][1 + cz]
        for cy in (0, 1):
            iy = (parts[1][0] + cy) % n_mesh
            wy = parts[1][1 + cy]
            for cx in (0, 1):
                ix = (parts[0][0] + cx) % n_mesh
                wx = parts[0][1 + cx]
                yield (iz * n_mesh + iy) * n_mesh + ix, wx * wy * wz


def deposit_u64(off, count, n_ios, n_mesh):
    """Integer CIC accumulator (uint64 per cell, [z][y][x])."""
    X = fixed_coords(off, count, n_ios)
    s = level_shift(n_ios, n_mesh)
    acc = np.zeros(n_mesh ** 3, dtype=np.uint64)
    for idx, w in _corners(X, n_mesh, s):
        np.add.at(acc, idx, w.astype(np.uint64))
    return acc.reshape(n_mesh, n_mesh, n_mesh)


def mean_integer(n_particles, n_mesh):
    """M = floor(N 2^48 / n_mesh^3), exact integer arithmetic."""
    return (int(n_particles) << 48) // (n_mesh ** 3)


def _split_delta(acc, m):
    """(sign, |acc - M|) with |.| as uint64, exact."""
    acc = acc.astype(np.uint64)
    m = np.uint64(m)
    ge = acc >= m
    mag = np.where(ge, acc - m, m - acc)
    return np.where(ge, 1.0, -1.0), mag


def density(acc, n_particles):
    """FP64 overdensity grid (acc - M) 2^-48 n^3/N (mean-one density minus ~1)."""
    n = acc.shape[0]
    sign, mag = _split_delta(acc, mean_integer(n_particles, n))
    return sign * mag.astype(np.float64) * (2.0 ** -48 * n ** 3 / n_particles)


def density_fp32(acc, n_particles):
    """FP32 density grid, bit-exact spec: RN32(acc - M) * RN32(n^3/N * 2^-48)."""
    n = acc.shape[0]
    sign, mag = _split_delta(acc, mean_integer(n_particles, n))
    rn = mag.astype(np.float32) * sign.astype(np.float32)
    scale = np.float32(float(n ** 3) / float(n_particles) * 2.0 ** -48)
    return (rn * scale).astype(np.float32)


# ----------------------------------------------------------- solve / FD
def solve_potential(rho, g):
    """phi = IDFT[DFT[rho] G] (numpy's unnormalised forward, 1/n^3 inverse)."""
    return np.fft.irfftn(np.fft.rfftn(rho) * g, s=rho.shape, axes=(0, 1, 2))


def fd_gradient(phi):
    """Eq. (diff) as a real-space convolution E_d = D * phi (periodic).

    E(n) = 2/3 [phi(n+1) - phi(n-1)] - 1/12 [phi(n+2) - phi(n-2)] along d;
    component d = 0 is x (array axis 2)."""
    out = []
    for axis in (2, 1, 0):
        p1 = np.roll(phi, -1, axis=axis)
        m1 = np.roll(phi, 1, axis=axis)
        p2 = np.roll(phi, -2, axis=axis)
        m2 = np.roll(phi, 2, axis=axis)
        out.append(2.0 / 3.0 * (p1 - m1) - 1.0 / 12.0 * (p2 - m2))
    return np.stack(out)


def interpolate(field, off, count, n_ios):
    """CIC gather of a (3, n, n, n) field with the deposit's weights -> (3, N)."""
    n = field.shape[1]
    X = fixed_coords(off, count, n_ios)
    s = level_shift(n_ios, n)
    flat = field.reshape(3, -1)
    out = np.zeros((3, X.shape[1]))
    for idx, w in _corners(X, n, s):
        out += flat[:, idx] * (w.astype(np.float64) * 2.0 ** -48)
    return out


# ------------------------------------------------------------- PM force
def level_params(w):
    """Per level: (n_mesh, H [Mpc/h], b_soft [cells], b_trunc [cells] or None)."""
    out = []
    prev_b = None                             # softening of the coarser level, Mpc/h
    for lev in w.levels:
        h = w.box / lev.n_mesh
        b_soft = lev.beta
        b_trunc = None if prev_b is None else prev_b / h
        out.append((lev.n_mesh, h, b_soft, b_trunc))
        prev_b = lev.beta * h
    return out


def green_tables(w, alias=2):
    """Eq. Gk per level, with the workload's assignment order (2 CIC, 3 TSC).
    With w.iso_length > 0 the coarsest level (the only one whose force reaches
    past its softening) is isolated by Eq. isok at r = iso_length (Appendix A);
    the finer levels' kernels vanish beyond the coarser softening already."""
    order = getattr(w, "assign_order", 2)
    iso = getattr(w, "iso_length", 0.0)
    return [green(n, bs, bt, alias=alias, order=order, iso=(iso / h if iso and bt is None else None))
            for (n, h, bs, bt) in level_params(w)]


def pm_force_level(off, count, n_ios, n_mesh, h, g):
    """F = -H interp(D * phi) for one level; also returns (acc, rho, phi)."""
    n_part = int(count.sum())
    acc = deposit_u64(off, count, n_ios, n_mesh)
    rho = density(acc, n_part)
    phi = solve_potential(rho, g)
    e = fd_gradient(phi)
    return -h * interpolate(e, off, count, n_ios), dict(acc=acc, rho=rho, phi=phi)


def pm_force(off, count, w, greens=None):
    """Sum of all PM levels of workload ``w`` (F = -grad u, (3, N))."""
    greens = green_tables(w) if greens is None else greens
    level_force = pm_force_level_tsc if getattr(w, "assign_order", 2) == 3 else pm_force_level
    total = 0.0
    for (n, h, _bs, _bt), g in zip(level_params(w), greens):
        f, _ = level_force(off, count, w.n_ios, n, h, g)
        total = total + f
    return total


def deposit_u64_at(off, count, start, n_ios, n_mesh, cells):
    """Integer CIC accumulator at selected mesh cells only (flat ids, x fastest).

    For each selected cell, gathers the particles of every IOS cell near it
    (a window that holds all particles whose CIC cloud can reach the cell)
    and sums their exact corner weights that land on it, as ``deposit_u64``."""
    s = level_shift(n_ios, n_mesh)
    cells = np.asarray(cells, dtype=np.int64)
    out = np.zeros(len(cells), dtype=np.uint64)
    for k, cell in enumerate(cells):
        js = (int(cell % n_mesh), int((cell // n_mesh) % n_mesh), int(cell // (n_mesh * n_mesh)))
        # a particle of IOS cell c sits at mesh coordinates [c, c + 1) * 2^-s and
        # touches the cells floor(x - 1/2) and floor(x - 1/2) + 1
        if s >= 0:
            win = [range(((j - 2) << s), ((j + 2) << s) + 1) for j in js]
        else:
            win = [range((j - 2) >> (-s), ((j + 2) >> (-s)) + 1) for j in js]
        seen = set()
        total = 0
        for iz in win[2]:
            for iy in win[1]:
                for ix in win[0]:
                    c = ((iz % n_ios) * n_ios + iy % n_ios) * n_ios + ix % n_ios
                    if c in seen:
                        continue
                    seen.add(c)
                    a, b = int(start[c]), int(start[c]) + int(count[c])
                    if b == a:
                        continue
                    cxyz = np.array([c % n_ios, (c // n_ios) % n_ios, c // (n_ios * n_ios)], dtype=np.int64)
                    X = cxyz[:, None] * FIX + off[:, a:b].astype(np.int64)
                    for idx, wgt in _corners(X, n_mesh, s):
                        total += int(wgt[idx == cell].sum())
        out[k] = np.uint64(total % (1 << 64))
    return out


# ------------------------------------------------------ TSC (order 3)
# The paper's own assignment (Eq. filter): triangular-shaped cloud, W(k) =
# prod_d sinc^3(k_d/2).  With u the position in mesh cells, i = floor(u) the
# cell holding it and d = u - (i + 1/2) in [-1/2, 1/2), the 1-D weights are
# (1/2 - d)^2/2, 3/4 - d^2 and (1/2 + d)^2/2 on cells i - 1, i, i + 1.  The
# position is the IOS fixed point in mesh units, floored to 2^-16 mesh cell
# as for CIC; weights and sums are FP64 (no exact-integer form: a 3-D weight
# would need 99 bits).
def tsc_weights_1d(X, s):
    """Cell i and the three weights (cells i-1, i, i+1) per particle, FP64."""
    xm = (X >> s) if s >= 0 else (X << (-s))
    i = xm >> 16
    d = (xm - (i << 16)).astype(np.float64) / FIX - 0.5
    return i, (0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2)


def _tsc_corners(X, n_mesh, s):
    """Yield (flat cell index, weight) for the 27 TSC cells."""
    parts = [tsc_weights_1d(X[d], s) for d in range(3)]
    for jz in (-1, 0, 1):
        iz = (parts[2][0] + jz) % n_mesh
        wz = parts[2][1][jz + 1]
        for jy in (-1, 0, 1):
            iy = (parts[1][0] + jy) % n_mesh
            wy = parts[1][1][jy + 1]
            for jx in (-1, 0, 1):
                ix = (parts[0][0] + jx) % n_mesh
                yield (iz * n_mesh + iy) * n_mesh + ix, parts[0][1][jx + 1] * wy * wz


def density_tsc(off, count, n_ios, n_mesh):
    """FP64 overdensity (n^3/N) sum_i W(u_i, c) - 1 with TSC weights."""
    X = fixed_coords(off, count, n_ios)
    s = level_shift(n_ios, n_mesh)
    rho = np.zeros(n_mesh ** 3)
    for idx, w in _tsc_corners(X, n_mesh, s):
        np.add.at(rho, idx, w)
    n_part = int(count.sum())
    return (rho * (n_mesh ** 3 / n_part) - 1.0).reshape(n_mesh, n_mesh, n_mesh)


def interpolate_tsc(field, off, count, n_ios):
    """TSC gather of a (3, n, n, n) field with the deposit's weights -> (3, N)."""
    n = field.shape[1]
    X = fixed_coords(off, count, n_ios)
    s = level_shift(n_ios, n)
    flat = field.reshape(3, -1)
    out = np.zeros((3, X.shape[1]))
    for idx, w in _tsc_corners(X, n, s):
        out += flat[:, idx] * w
    return out


def pm_force_level_tsc(off, count, n_ios, n_mesh, h, g):
    """F = -H interp_TSC(D * phi) with phi = G * rho_TSC; also returns (rho, phi)."""
    rho = density_tsc(off, count, n_ios, n_mesh)
    phi = solve_potential(rho, g)
    e = fd_gradient(phi)
    return -h * interpolate_tsc(e, off, count, n_ios), dict(rho=rho, phi=phi)


# ------------------------------------------- point evaluation of a level
def particle_cells(count, start, targets):
    """IOS cell of each selected particle (flat ids), from counts and starts."""
    ends = start.astype(np.int64) + count.astype(np.int64)
    return np.searchsorted(ends, np.asarray(targets, dtype=np.int64), side="right")


def pm_force_level_at(phi, off, count, start, n_ios, h, targets):
    """F = -H interp(D * phi) of one level at selected particles only, (3, K).

    The same steps as ``pm_force_level`` after the solve (Eq. diff as the
    real-space 4-point difference, then the CIC gather with the deposit's
    integer weights), but the difference is formed only at the 8 cells each
    selected particle gathers from: E_d(c) = 2/3 [phi(c+e_d) - phi(c-e_d)] -
    1/12 [phi(c+2e_d) - phi(c-2e_d)], periodic."""
    n = phi.shape[0]
    targets = np.asarray(targets, dtype=np.int64)
    c = particle_cells(count, start, targets)
    cc = np.stack([c % n_ios, (c // n_ios) % n_ios, c // (n_ios * n_ios)])
    X = cc * FIX + off[:, targets].astype(np.int64)
    s = level_shift(n_ios, n)
    parts = [cic_integer_weights(X[d], s) for d in range(3)]
    out = np.zeros((3, len(targets)))
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                idx = [parts[0][0] + ox, parts[1][0] + oy, parts[2][0] + oz]
                wgt = (parts[0][1 + ox] * parts[1][1 + oy] * parts[2][1 + oz]).astype(np.float64) * 2.0 ** -48
                for d in range(3):
                    def at(step):
                        j = list(idx)
                        j[d] = j[d] + step
                        return phi[j[2] % n, j[1] % n, j[0] % n]
                    e = 2.0 / 3.0 * (at(1) - at(-1)) - 1.0 / 12.0 * (at(2) - at(-2))
                    out[d] += wgt * e
    return -h * out
