"""FP64 oracle: short-range particle-particle (PP) force with a cell list.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; never by the product path.

Sec. 2.2.3 and Eq. (PP): every particle receives, from every other particle
closer than the PP range b_cut (the softening of the finest PM level), the
force V_p R_PP(r) / (4 pi) along the pair separation, with
R_PP = R(r, b_PP) - R(r, b_cut) (Eq. refforce).  The IOS ordering doubles as
the linked list (Sec. 2.3): the particles of IOS cell c are the index range
[start_c, start_c + count_c).  The IOS cell is at least b_cut wide, so the 27
cells around a particle's cell hold every partner.  V_p = L^3 / N is the
mass of a particle in mean-density-one units.
"""
from __future__ import annotations

import math

import numpy as np

from .kernels import pp_reference
from .mesh import FIX, cell_coords


def _neighbour_pairs(count, start, n_ios, offset):
    """All (i, j) with i in cell c and j in cell c + offset (periodic)."""
    n3 = n_ios ** 3
    cells = np.arange(n3, dtype=np.int64)
    cx, cy, cz = cells % n_ios, (cells // n_ios) % n_ios, cells // (n_ios * n_ios)
    ox, oy, oz = offset
    nb = (((cz + oz) % n_ios) * n_ios + (cy + oy) % n_ios) * n_ios + (cx + ox) % n_ios
    ci = count.astype(np.int64)
    cj = ci[nb]
    npair = ci * cj
    keep = npair > 0
    cells, nb, ci_k, cj_k, npair = cells[keep], nb[keep], ci[keep], cj[keep], npair[keep]
    total = int(npair.sum())
    if total == 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z
    first = np.zeros_like(npair)
    np.cumsum(npair[:-1], out=first[1:])
    local = np.arange(total, dtype=np.int64) - np.repeat(first, npair)
    rep_cj = np.repeat(cj_k, npair)
    i = np.repeat(start.astype(np.int64)[cells], npair) + local // rep_cj
    j = np.repeat(start.astype(np.int64)[nb], npair) + local % rep_cj
    return i, j


def pp_force(off, count, start, n_ios, box, b_pp, b_cut, n_particles=None, targets=None):
    """PP force (3, N) [or (3, len(targets))] in FP64.

    The separation of a pair is formed exactly in fixed point from the cell
    offset (-1, 0, +1 per axis) and the uint16 in-cell offsets."""
    n_part = int(count.sum()) if n_particles is None else n_particles
    s_ios = box / n_ios
    assert b_cut <= s_ios * (1 + 1e-12), "PP range must fit in one IOS cell"
    vp = box ** 3 / n_part
    off64 = off.astype(np.int64)
    want = None
    if targets is not None:
        want = np.zeros(n_part, dtype=bool)
        want[np.asarray(targets)] = True
    out = np.zeros((3, n_part))
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                i, j = _neighbour_pairs(count, start, n_ios, (ox, oy, oz))
                if want is not None:
                    sel = want[i]
                    i, j = i[sel], j[sel]
                if i.size == 0:
                    continue
                d = np.empty((3, i.size))
                for ax, o in enumerate((ox, oy, oz)):
                    d[ax] = (o * FIX + off64[ax, j] - off64[ax, i]) * (s_ios / FIX)
                r = np.sqrt((d * d).sum(axis=0))
                m = (r > 0) & (r < b_cut) & (i != j)
                if not m.any():
                    continue
                i, d, r = i[m], d[:, m], r[m]
                mag = vp * pp_reference(r, b_pp, b_cut) / (4.0 * math.pi * r)
                for ax in range(3):
                    out[ax] += np.bincount(i, weights=mag * d[ax], minlength=n_part)
    return out if targets is None else out[:, np.asarray(targets)]


def pp_force_brute(pos, box, b_pp, b_cut, n_particles=None):
    """All-pairs minimum-image PP force on decoded positions (3, N), for pins."""
    n = pos.shape[1]
    vp = box ** 3 / (n if n_particles is None else n_particles)
    d = pos[:, None, :] - pos[:, :, None]          # d[:, i, j] = x_j - x_i
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(axis=0))
    m = (r > 0) & (r < b_cut)
    rs = np.where(m, r, 1.0)
    mag = np.where(m, vp * pp_reference(rs, b_pp, b_cut) / (4.0 * math.pi * rs), 0.0)
    return (d * mag[None]).sum(axis=2)


def pp_force_at(off, count, start, n_ios, box, b_pp, b_cut, targets, n_particles=None):
    """PP force (3, K) on selected particles only, by the same rule as ``pp_force``:
    each target's 27 neighbour cells are gathered directly."""
    n_part = int(count.sum()) if n_particles is None else n_particles
    s_ios = box / n_ios
    vp = box ** 3 / n_part
    targets = np.asarray(targets, dtype=np.int64)
    starts = start.astype(np.int64)
    ends = starts + count.astype(np.int64)
    cell_of = np.searchsorted(ends, targets, side="right")
    out = np.zeros((3, len(targets)))
    for k, (i, c) in enumerate(zip(targets, cell_of)):
        cc = (c % n_ios, (c // n_ios) % n_ios, c // (n_ios * n_ios))
        oi = off[:, i].astype(np.int64)
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    nb = ((((cc[2] + oz) % n_ios) * n_ios + (cc[1] + oy) % n_ios) * n_ios
                          + (cc[0] + ox) % n_ios)
                    j = np.arange(starts[nb], ends[nb])
                    j = j[j != i]
                    if j.size == 0:
                        continue
                    d = np.empty((3, j.size))
                    for ax, o in enumerate((ox, oy, oz)):
                        d[ax] = (o * FIX + off[ax, j].astype(np.int64) - oi[ax]) * (s_ios / FIX)
                    r = np.sqrt((d * d).sum(axis=0))
                    m = (r > 0) & (r < b_cut)
                    if not m.any():
                        continue
                    d, r = d[:, m], r[m]
                    mag = vp * pp_reference(r, b_pp, b_cut) / (4.0 * math.pi * r)
                    out[:, k] += (d * mag).sum(axis=1)
    return out


def pp_force_at_many(off, count, start, n_ios, box, b_pp, b_cut, targets, n_particles=None):
    """``pp_force_at`` for many targets at once, (3, K): for each of the 27
    cell offsets, every (target, source) pair of the target's neighbour cell
    is formed in one array and the pair terms are summed per target."""
    n_part = int(count.sum()) if n_particles is None else n_particles
    s_ios = box / n_ios
    vp = box ** 3 / n_part
    targets = np.asarray(targets, dtype=np.int64)
    starts = start.astype(np.int64)
    cnt = count.astype(np.int64)
    c = np.searchsorted(starts + cnt, targets, side="right")
    cc = np.stack([c % n_ios, (c // n_ios) % n_ios, c // (n_ios * n_ios)])
    oi = off[:, targets].astype(np.int64)
    out = np.zeros((3, len(targets)))
    k_all = np.arange(len(targets), dtype=np.int64)
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                nb = ((((cc[2] + oz) % n_ios) * n_ios + (cc[1] + oy) % n_ios) * n_ios + (cc[0] + ox) % n_ios)
                m = cnt[nb]
                tot = int(m.sum())
                if tot == 0:
                    continue
                k = np.repeat(k_all, m)
                first = np.repeat(np.cumsum(m) - m, m)
                j = np.repeat(starts[nb], m) + (np.arange(tot, dtype=np.int64) - first)
                keep = j != targets[k]
                k, j = k[keep], j[keep]
                d = np.empty((3, j.size))
                for ax, o in enumerate((ox, oy, oz)):
                    d[ax] = (o * FIX + off[ax, j].astype(np.int64) - oi[ax, k]) * (s_ios / FIX)
                r = np.sqrt((d * d).sum(axis=0))
                sel = (r > 0) & (r < b_cut)
                if not sel.any():
                    continue
                k, d, r = k[sel], d[:, sel], r[sel]
                mag = vp * pp_reference(r, b_pp, b_cut) / (4.0 * math.pi * r)
                for ax in range(3):
                    out[ax] += np.bincount(k, weights=mag * d[ax], minlength=len(targets))
    return out


__all__ = ["pp_force", "pp_force_at", "pp_force_at_many", "pp_force_brute", "cell_coords"]
