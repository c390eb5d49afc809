"""FP64 oracle of the adaptive third PM level (Sec. 2.1.1, Eq. PM3; Sec. 2.2.3):
local meshes, one per subtile, of a resolution chosen per subtile.

TEST INFRASTRUCTURE ONLY.  Imported by tests/; never by the product path.  The
GPU path has no third level yet: this module is the reference it will be
checked against.

Readings (the paper gives the method, not every detail):

* Subtiles: the box of n_ios^3 IOS cells is cut into subtiles of T^3 IOS
  cells.  Subtile s has its own PM3 mesh spacing H_3 = H_fine / r_s (integer
  refinement r_s of the finest global level) and softening b_3 = beta_3 H_3
  (Sec. 2.2.3: b_3 = beta_3 H_3, beta_3 = 3.5 by default).  The choice of r_s
  from the subtile's clustering (rho_max) is an input here: the paper
  calibrates it from timings (its Fig. PMtime), which this oracle does not need.
* A particle of subtile s feels the global levels as in the two-level method,
  the PM3 force of Eq. (PM3) with the reference force R(r, b_3) - R(r, b_fine)
  (truncated at the finest global softening, as the paper's R_3 is at b_2), and
  the PP force of Eq. (PP) with range b_3 instead of b_fine.
* The PM3 mesh of s covers the subtile plus a buffer of B cells on each side,
  B = ceil(b_fine / H_3) + 4 (the kernel's reach, the 4-point difference's two
  cells, the CIC cloud and one spare), rounded up to a 2^a 3^b mesh on the high
  side; it is solved as a periodic mesh (the paper's local PM meshes are:
  periodic images lie beyond the truncated kernel's reach).  Every particle
  inside the local box is a source, deposited by CIC from its decoded FP64
  position; forces are gathered for the subtile's own particles only.
* r_s = 1 with beta_3 = beta_fine makes the PM3 kernel vanish and the PP range
  b_fine: the two-level method.
"""
from __future__ import annotations

import math

import numpy as np

from .kdk import pp_params
from .kernels import green
from .mesh import fd_gradient, level_params, pm_force, positions, solve_potential
from .pp import pp_force


def _fft_size(m):
    """Smallest 2^a 3^b >= m."""
    best = None
    for a in range(0, 16):
        for b in range(0, 10):
            v = 2 ** a * 3 ** b
            if v >= m and (best is None or v < best):
                best = v
    return best


def local_mesh(w, T, r, beta3):
    """(H_3, b_3, buffer cells B, mesh cells m) of a PM3 mesh with refinement r."""
    n_fine, h_fine, b_soft_fine, _ = level_params(w)[-1]
    b_fine = b_soft_fine * h_fine
    h3 = h_fine / r
    b3 = beta3 * h3
    s_ios = w.box / w.n_ios
    inner = T * s_ios / h3
    if abs(inner - round(inner)) > 1e-9:
        raise ValueError("the subtile must span a whole number of PM3 cells")
    B = int(math.ceil(b_fine / h3 - 1e-12)) + 4
    m = _fft_size(int(round(inner)) + 2 * B)
    if m * h3 > w.box + 1e-9:
        raise ValueError("the local PM3 box must not exceed the simulation box")
    return h3, b3, B, m


def _cic(u, m):
    """The 8 CIC corners of positions u (3, K) in cells: (flat index, weight)."""
    t = u - 0.5
    i0 = np.floor(t).astype(np.int64)
    f = t - i0
    out = []
    for cz in (0, 1):
        iz = (i0[2] + cz) % m
        wz = f[2] if cz else 1.0 - f[2]
        for cy in (0, 1):
            iy = (i0[1] + cy) % m
            wy = f[1] if cy else 1.0 - f[1]
            for cx in (0, 1):
                ix = (i0[0] + cx) % m
                wx = f[0] if cx else 1.0 - f[0]
                out.append(((iz * m + iy) * m + ix, wx * wy * wz))
    return out


def pm3_green(w, T, r, beta3, alias=2):
    """Eq. (Gk) for the PM3 mesh of refinement r (soft b_3, truncated at b_fine)."""
    n_fine, h_fine, b_soft_fine, _ = level_params(w)[-1]
    h3, b3, _B, m = local_mesh(w, T, r, beta3)
    return green(m, b3 / h3, b_soft_fine * h_fine / h3, alias=alias)


def pm3_force_subtile(pos, w, T, sub, r, beta3, n_particles=None, alias=2, g=None):
    """PM3 force (3, K) on the particles of subtile ``sub`` = (sx, sy, sz), and
    their indices (K,): Eq. (PM3) on the subtile's local mesh (g: its table,
    pm3_green, computed here when None)."""
    n_part = pos.shape[1] if n_particles is None else n_particles
    n_fine, h_fine, b_soft_fine, _ = level_params(w)[-1]
    b_fine = b_soft_fine * h_fine
    h3, b3, B, m = local_mesh(w, T, r, beta3)
    s_ios = w.box / w.n_ios
    side = T * s_ios
    origin = np.asarray(sub, dtype=np.float64) * side - B * h3
    rel = (pos - origin[:, None]) % w.box                     # in [0, box)
    inside = np.all(rel < m * h3, axis=0)
    u = rel[:, inside] / h3
    # sources: CIC onto the local periodic mesh, mean-one density units
    rho = np.zeros(m ** 3)
    vp = w.box ** 3 / n_part
    for idx, wt in _cic(u, m):
        np.add.at(rho, idx, wt * (vp / h3 ** 3))
    rho = rho.reshape(m, m, m)
    if g is None:
        g = green(m, b3 / h3, b_fine / h3, alias=alias)
    e = fd_gradient(solve_potential(rho, g))
    # targets: the subtile's own particles
    lo = B * h3
    own = np.all((rel >= lo) & (rel < lo + side), axis=0)
    ut = rel[:, own] / h3
    flat = e.reshape(3, -1)
    f = np.zeros((3, ut.shape[1]))
    for idx, wt in _cic(ut, m):
        f += flat[:, idx] * wt
    return -h3 * f, np.nonzero(own)[0]


def subtile_of(off, count, n_ios, T):
    """Subtile index (3, N) of every particle (from its IOS cell)."""
    cell = np.repeat(np.arange(n_ios ** 3, dtype=np.int64), count.astype(np.int64))
    c = np.stack([cell % n_ios, (cell // n_ios) % n_ios, cell // (n_ios * n_ios)])
    return c // T


def adaptive_force(off, count, start, w, T, refine, beta3, greens=None, alias=2):
    """Total force (3, N) with the adaptive third level: the global levels of
    ``w``, PM3 per subtile with refinement refine[sz, sy, sx] and softening
    beta3 cells, PP per subtile with range b_3 = beta3 H_3.

    A subtile whose b_3 equals the finest global softening has the kernel
    R(r, b_3) - R(r, b_fine) = 0: its PM3 force is zero and is not formed.
    The PP force is evaluated once per distinct range over all the targets
    that have it (each target's sum is independent of the others')."""
    if w.n_ios % T:
        raise ValueError("T must divide n_ios")
    n_part = int(count.sum())
    pos = positions(off, count, w.n_ios, w.box)
    total = pm_force(off, count, w, greens)
    b_pp, b_fine = pp_params(w)
    sub = subtile_of(off, count, w.n_ios, T)
    ns = w.n_ios // T
    refine = np.asarray(refine).reshape(ns, ns, ns)
    geo = {int(r): local_mesh(w, T, int(r), beta3) for r in np.unique(refine)}
    vanishes = {r: abs(g[1] - b_fine) <= 1e-12 * b_fine for r, g in geo.items()}
    tables = {r: pm3_green(w, T, r, beta3, alias) for r in geo if not vanishes[r]}
    by_range = {}
    for sz in range(ns):
        for sy in range(ns):
            for sx in range(ns):
                r = int(refine[sz, sy, sx])
                mine = np.nonzero((sub[0] == sx) & (sub[1] == sy) & (sub[2] == sz))[0]
                if mine.size == 0:
                    continue
                if not vanishes[r]:
                    f3, idx = pm3_force_subtile(pos, w, T, (sx, sy, sz), r, beta3, n_part, alias, tables[r])
                    assert np.array_equal(np.sort(idx), mine)
                    total[:, idx] += f3
                by_range.setdefault(geo[r][1], []).append(mine)
    for b3, parts in by_range.items():
        t = np.concatenate(parts)
        total[:, t] += pp_force(off, count, start, w.n_ios, w.box, b_pp, b3, targets=t)
    return total
