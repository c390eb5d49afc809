"""Periodic direct summation (Ewald) of softened gravity, for pinning the oracle.

TEST INFRASTRUCTURE ONLY.  Used by tests/ to check the oracle's PM+PP force
against the total reference force R(r, b_PP) of Eq. (force_decomp) summed
over all periodic images; never by the product path.

F_i = -grad u(x_i) with lap u = delta (mean density one, particle mass
V_p = L^3/N): the periodic Coulomb sum by the Ewald split (real-space erfc
part over 5^3 images, reciprocal part over |m_d| <= m_max), plus the
near-field softening correction V_p (R(r, b_PP) - 1/r^2)/(4 pi) along the
pair separation for minimum-image pairs closer than b_PP.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

from .kernels import reference_force


def ewald_force(pos, box, b_pp, n_particles=None, alpha=None, m_max=10, images=2):
    n = pos.shape[1]
    vp = box ** 3 / (n if n_particles is None else n_particles)
    alpha = 6.0 / box if alpha is None else alpha
    d0 = pos[:, :, None] - pos[:, None, :]            # x_i - x_j
    out = np.zeros((3, n))
    rng = range(-images, images + 1)
    for nz in rng:
        for ny in rng:
            for nx in rng:
                d = d0 + box * np.array([nx, ny, nz], dtype=np.float64)[:, None, None]
                r = np.sqrt((d * d).sum(axis=0))
                ok = r > 0
                rs = np.where(ok, r, 1.0)
                g = (erfc(alpha * rs) / rs ** 2
                     + 2.0 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * rs) ** 2) / rs)
                g = np.where(ok, g / rs, 0.0)
                out -= vp / (4.0 * math.pi) * (d * g[None]).sum(axis=2)
    m = np.arange(-m_max, m_max + 1)
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    kv = (2.0 * math.pi / box) * np.stack([mx.ravel(), my.ravel(), mz.ravel()])
    k2 = (kv * kv).sum(axis=0)
    keep = k2 > 0
    kv, k2 = kv[:, keep], k2[keep]
    coef = np.exp(-k2 / (4.0 * alpha ** 2)) / k2         # (K,)
    phase = kv.T @ pos                                    # (K, N): k . x_j
    c, s = np.cos(phase), np.sin(phase)
    sc, ss = c.sum(axis=1), s.sum(axis=1)                 # sum_j cos/sin(k.x_j)
    # sum_j sin(k.(x_i - x_j)) = sin(k.x_i) sum cos - cos(k.x_i) sum sin
    sfac = s * sc[:, None] - c * ss[:, None]              # (K, N)
    out -= (vp / box ** 3) * (kv @ (coef[:, None] * sfac))
    # near-field softening: replace 1/r^2 by R(r, b_PP) below b_PP
    dm = d0 - box * np.rint(d0 / box)
    r = np.sqrt((dm * dm).sum(axis=0))
    ok = (r > 0) & (r < b_pp)
    rs = np.where(ok, r, 1.0)
    corr = np.where(ok, (reference_force(rs, b_pp) - 1.0 / rs ** 2) / rs, 0.0)
    out -= vp / (4.0 * math.pi) * (dm * corr[None]).sum(axis=2)
    return out
