"""FP64 oracle: vector-Jacobian products of the PM + PP force (adjoint building blocks).

TEST INFRASTRUCTURE ONLY.  Imported by tests/ only; never by the product path.

The force of Sec. 2.1 as a function of continuous particle positions x
(Mpc/h, shape (3, N)); the IOS quantisation of Sec. 2.3 is treated as the
identity, so positions enter as plain numbers.  For a PM level with n^3 cells
of size H, positions in mesh cells are u = x / H and, with the conventions of
``oracle.mesh`` (cell c spans [c, c+1), CIC W(u, c) = prod_d w(u_d - c_d - 1/2),
w(t) = max(0, 1 - |t|)):

    rho(c) = (n^3 / N) sum_i W(u_i, c)             assignment (Eq. filter, CIC reading)
    phi    = G * rho                                Poisson solve with the Eq. (Gk) table
    E_d    = D_d * phi                              4-point difference (Eq. diff)
    F_i    = -H sum_c W(u_i, c) E(c)                interpolation, F = -grad u

and the PP term (Eq. PP) is F_i = sum_{j != i} g(r_ij) (x_j - x_i) with
g(r) = V_p R_PP(r) / (4 pi r), r < b_cut, minimum image.

For a cotangent v (3, N) the vector-Jacobian product w_i = d<v, F(x)>/dx_i is
(chain rule; G is even and D_d odd, so the transpose of D_d * G * is
-G * D_d *):

    PM:  w_i = -sum_c grad_u W(u_i, c) (E(c) . v_i) + sum_c grad_u W(u_i, c) psi(c),
         psi = G * s,   s = (n^3 / N) sum_d D_d * mu_d,   mu_d(c) = sum_j W(u_j, c) v_{j,d}
    PP:  w_i = sum_{j != i} A_ij (v_j - v_i),   A = g I + (g'(r) / r) d d^T,   d = x_j - x_i.
"""
from __future__ import annotations

import math

import numpy as np

from .kernels import pp_reference, reference_force_derivative
from .mesh import FIX, fd_gradient, level_params, solve_potential
from .pp import _neighbour_pairs


def cic_corners(u, n):
    """The 8 CIC corners of positions u (3, N) in mesh cells: a list of
    (flat cell index, weight W, gradient of W with respect to u (3, N))."""
    t = u - 0.5
    i0 = np.floor(t).astype(np.int64)
    f = t - i0
    w = [1.0 - f, f]                       # weights of the lower / upper corner per axis
    dw = [-np.ones_like(f), np.ones_like(f)]
    out = []
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                c = (cx, cy, cz)
                idx = (((i0[2] + cz) % n) * n + (i0[1] + cy) % n) * n + (i0[0] + cx) % n
                wd = [w[c[d]][d] for d in range(3)]
                W = wd[0] * wd[1] * wd[2]
                grad = np.stack([dw[c[0]][0] * wd[1] * wd[2], wd[0] * dw[c[1]][1] * wd[2],
                                 wd[0] * wd[1] * dw[c[2]][2]])
                out.append((idx, W, grad))
    return out


def _deposit(corners, vals, n):
    """sum over particles of W * vals onto the mesh ([z][y][x])."""
    m = np.zeros(n ** 3)
    for idx, W, _ in corners:
        np.add.at(m, idx, W * vals)
    return m.reshape(n, n, n)


def pm_force_level(x, box, n, n_particles, g):
    """F (3, N) of one PM level at continuous positions x."""
    h = box / n
    corners = cic_corners(x / h, n)
    rho = _deposit(corners, np.ones(x.shape[1]), n) * (n ** 3 / n_particles)
    e = fd_gradient(solve_potential(rho, g)).reshape(3, -1)
    f = np.zeros_like(x)
    for idx, W, _ in corners:
        f -= h * W * e[:, idx]
    return f


def pm_vjp_level(x, v, box, n, n_particles, g):
    """d<v, F_level(x)>/dx (3, N)."""
    h = box / n
    corners = cic_corners(x / h, n)
    rho = _deposit(corners, np.ones(x.shape[1]), n) * (n ** 3 / n_particles)
    e = fd_gradient(solve_potential(rho, g)).reshape(3, -1)
    mu = np.stack([_deposit(corners, v[d], n) for d in range(3)])
    # s = (n^3/N) sum_d D_d * mu_d: component d of fd_gradient(mu_d) is D_d * mu_d
    s = sum(fd_gradient(mu[d])[d] for d in range(3)) * (n ** 3 / n_particles)
    psi = solve_potential(s, g).reshape(-1)
    w = np.zeros_like(x)
    for idx, _W, grad in corners:
        ev = (e[:, idx] * v).sum(axis=0)
        w += grad * (psi[idx] - ev)
    return w


def _pairs(x, box, b_cut):
    """All ordered pairs (i, j), i != j, closer than b_cut (minimum image):
    indices and separations d = x_j - x_i (3, P)."""
    n = x.shape[1]
    d = x[:, None, :] - x[:, :, None]            # d[:, i, j] = x_j - x_i
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(axis=0))
    i, j = np.nonzero((r > 0) & (r < b_cut))
    return i, j, d[:, i, j], r[i, j]


def _pairs_cells(x, box, b_cut):
    """The pairs of ``_pairs`` found through a cell list: cells of side
    box / nc >= b_cut (nc >= 3), every particle against the particles of its
    27 neighbouring cells (minimum image)."""
    nc = int(box // b_cut)
    if nc < 3:
        return _pairs(x, box, b_cut)
    side = box / nc
    c3 = np.floor(x / side).astype(np.int64) % nc
    cid = (c3[2] * nc + c3[1]) * nc + c3[0]
    order = np.argsort(cid, kind="stable")
    cnt = np.bincount(cid, minlength=nc ** 3)
    beg = np.cumsum(cnt) - cnt
    cells = np.arange(nc ** 3, dtype=np.int64)
    cx, cy, cz = cells % nc, (cells // nc) % nc, cells // (nc * nc)
    out_i, out_j = [], []
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                nb = (((cz + oz) % nc) * nc + (cy + oy) % nc) * nc + (cx + ox) % nc
                npair = cnt * cnt[nb]
                keep = npair > 0
                if not keep.any():
                    continue
                ck, nbk, ci, cj, np_k = cells[keep], nb[keep], cnt[keep], cnt[nb][keep], npair[keep]
                tot = int(np_k.sum())
                first = np.repeat(np.cumsum(np_k) - np_k, np_k)
                local = np.arange(tot, dtype=np.int64) - first
                rep_cj = np.repeat(cj, np_k)
                a = np.repeat(beg[ck], np_k) + local // rep_cj
                b = np.repeat(beg[nbk], np_k) + local % rep_cj
                out_i.append(order[a])
                out_j.append(order[b])
    if not out_i:
        z = np.zeros(0, dtype=np.int64)
        return z, z, np.zeros((3, 0)), np.zeros(0)
    i, j = np.concatenate(out_i), np.concatenate(out_j)
    d = x[:, j] - x[:, i]
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(axis=0))
    m = (r > 0) & (r < b_cut) & (i != j)
    return i[m], j[m], d[:, m], r[m]


def _pair_search(x, box, b_cut):
    """All-pairs for small sets, the cell list beyond 4096 particles."""
    return _pairs(x, box, b_cut) if x.shape[1] <= 4096 else _pairs_cells(x, box, b_cut)


def pp_force(x, box, n_particles, b_pp, b_cut):
    """PP force (3, N) at continuous positions (every pair closer than b_cut)."""
    i, j, d, r = _pair_search(x, box, b_cut)
    g = box ** 3 / n_particles * pp_reference(r, b_pp, b_cut) / (4 * math.pi * r)
    f = np.zeros_like(x)
    for ax in range(3):
        f[ax] = np.bincount(i, weights=g * d[ax], minlength=x.shape[1])
    return f


def pp_vjp(x, v, box, n_particles, b_pp, b_cut):
    """d<v, F_PP(x)>/dx (3, N) (every pair closer than b_cut)."""
    i, j, d, r = _pair_search(x, box, b_cut)
    vp = box ** 3 / n_particles / (4 * math.pi)
    rpp = pp_reference(r, b_pp, b_cut)
    drpp = reference_force_derivative(r, b_pp) - reference_force_derivative(r, b_cut)
    g = vp * rpp / r
    gp = vp * (drpp / r - rpp / r ** 2)
    dv = v[:, j] - v[:, i]
    term = g * dv + (gp / r) * d * (d * dv).sum(axis=0)
    w = np.zeros_like(x)
    for ax in range(3):
        w[ax] = np.bincount(i, weights=term[ax], minlength=x.shape[1])
    return w


def pp_vjp_cells(off, count, start, n_ios, box, b_pp, b_cut, v, n_particles=None):
    """pp_vjp for IOS data with the cell list of ``oracle.pp`` (the IOS cell is
    at least b_cut wide, so the 27 cells around a particle hold its partners);
    separations are formed exactly from the fixed-point offsets."""
    n_part = int(count.sum()) if n_particles is None else n_particles
    s_ios = box / n_ios
    vp = box ** 3 / n_part / (4 * math.pi)
    off64 = off.astype(np.int64)
    w = np.zeros((3, n_part))
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                i, j = _neighbour_pairs(count, start, n_ios, (ox, oy, oz))
                if i.size == 0:
                    continue
                d = np.empty((3, i.size))
                for ax, o in enumerate((ox, oy, oz)):
                    d[ax] = (o * FIX + off64[ax, j] - off64[ax, i]) * (s_ios / FIX)
                r = np.sqrt((d * d).sum(axis=0))
                m = (r > 0) & (r < b_cut) & (i != j)
                i, j, d, r = i[m], j[m], d[:, m], r[m]
                rpp = pp_reference(r, b_pp, b_cut)
                drpp = reference_force_derivative(r, b_pp) - reference_force_derivative(r, b_cut)
                g = vp * rpp / r
                gp = vp * (drpp / r - rpp / r ** 2)
                dv = v[:, j] - v[:, i]
                term = g * dv + (gp / r) * d * (d * dv).sum(axis=0)
                for ax in range(3):
                    w[ax] += np.bincount(i, weights=term[ax], minlength=n_part)
    return w


def force(x, wl, greens):
    """Total force (every PM level plus PP) of workload wl at positions x."""
    n_part = x.shape[1]
    f = np.zeros_like(x)
    for (n, _h, _bs, _bt), g in zip(level_params(wl), greens):
        f += pm_force_level(x, wl.box, n, n_part, g)
    n_f, h_f, b_soft, _ = level_params(wl)[-1]
    return f + pp_force(x, wl.box, n_part, wl.b_pp, b_soft * h_f)


def force_vjp(x, v, wl, greens):
    """d<v, F(x)>/dx for the total force of workload wl."""
    n_part = x.shape[1]
    w = np.zeros_like(x)
    for (n, _h, _bs, _bt), g in zip(level_params(wl), greens):
        w += pm_vjp_level(x, v, wl.box, n, n_part, g)
    n_f, h_f, b_soft, _ = level_params(wl)[-1]
    return w + pp_vjp(x, v, wl.box, n_part, wl.b_pp, b_soft * h_f)


# --------------------------------------------------- trajectory and loss
def quantise_drift(x, dx, wl):
    """x + dx with the displacement rounded to the IOS grid (2^-16 IOS cell,
    round half to even) and wrapped: the fixed-point drift of Sec. 2.3 on
    positions that lie on that grid (X + rint(d) = rint(X + d) for integer X)."""
    q = wl.box / wl.n_ios / FIX
    return (x + np.rint(dx / q) * q) % wl.box


def kdk_trajectory(x0, p0, wl, greens, a, ios=False):
    """KDK steps a[0] -> a[-1] (Sec. 2.2; kick K(a0, ah), drift Dr(a0, a1),
    kick K(ah, a1), dp/da = 1.5 Omega_m F / (a^2 E)) at continuous positions,
    or with ``ios`` on the IOS grid (every drift rounded as ``quantise_drift``;
    x0 must lie on the grid).  Returns the states [(x_k, p_k)] before the first
    and after every step."""
    from .kdk import drift_integral, kick_integral
    c = 1.5 * wl.omega_m
    x, p = x0.copy(), p0.copy()
    f = force(x, wl, greens)
    out = [(x, p)]
    for a0, a1 in zip(a[:-1], a[1:]):
        ah = 0.5 * (a0 + a1)
        pm = p + c * kick_integral(a0, ah, wl.omega_m, wl.omega_l) * f
        dx = drift_integral(a0, a1, wl.omega_m, wl.omega_l) * pm
        x = quantise_drift(x, dx, wl) if ios else (x + dx) % wl.box
        f = force(x, wl, greens)
        p = pm + c * kick_integral(ah, a1, wl.omega_m, wl.omega_l) * f
        out.append((x, p))
    return out


def density_loss(x, wl, target):
    """L = mean over the finest mesh of (delta - target)^2, delta the CIC overdensity."""
    n = wl.levels[-1].n_mesh
    h = wl.box / n
    rho = _deposit(cic_corners(x / h, n), np.ones(x.shape[1]), n) * (n ** 3 / x.shape[1])
    return float(np.mean((rho - 1.0 - target) ** 2))


def density_loss_grad(x, wl, target):
    """(L, dL/dx) of ``density_loss``."""
    n = wl.levels[-1].n_mesh
    h = wl.box / n
    npart = x.shape[1]
    corners = cic_corners(x / h, n)
    rho = _deposit(corners, np.ones(npart), n) * (n ** 3 / npart)
    r = (rho - 1.0 - target).reshape(-1)
    g = 2.0 * r / n ** 3
    w = np.zeros_like(x)
    for idx, _W, grad in corners:
        w += grad * g[idx]
    return float(np.mean(r ** 2)), w * (n ** 3 / (npart * h))


def loss_gradient(x0, p0, wl, greens, a, target, ios=False):
    """(L, dL/dx0, dL/dp0) through the KDK steps of ``kdk_trajectory``:
    reverse mode, step by step, with the force products above.  With ``ios``
    the forward steps round their drifts to the IOS grid and the reverse sweep
    takes that rounding as the identity (the products are evaluated at the
    grid positions the trajectory visits)."""
    from .kdk import drift_integral, kick_integral
    c = 1.5 * wl.omega_m
    traj = kdk_trajectory(x0, p0, wl, greens, a, ios=ios)
    loss, xbar = density_loss_grad(traj[-1][0], wl, target)
    pbar = np.zeros_like(xbar)
    for k in range(len(a) - 2, -1, -1):
        a0, a1 = a[k], a[k + 1]
        ah = 0.5 * (a0 + a1)
        x_pre, x_post = traj[k][0], traj[k + 1][0]
        xbar = xbar + c * kick_integral(ah, a1, wl.omega_m, wl.omega_l) * force_vjp(x_post, pbar, wl, greens)
        pbar = pbar + drift_integral(a0, a1, wl.omega_m, wl.omega_l) * xbar
        xbar = xbar + c * kick_integral(a0, ah, wl.omega_m, wl.omega_l) * force_vjp(x_pre, pbar, wl, greens)
    return loss, xbar, pbar
