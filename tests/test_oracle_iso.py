"""Pins of the oracle's isolated boundary conditions (Appendix A, Eq. isok) and
of the pairwise force accuracy test of Sec. 3.1.

1. The factor 1 - sinc(kL) of Eq. (isok) is checked against a numerical
   Fourier transform of the potential whose force is the inverse-square law
   truncated at r = L (it is -1/r + 1/L inside, 0 outside): the closed form is
   not re-typed, the integral is done by quadrature.
2. Two particles at a time in the 64 Mpc/h box of the isolated workload: the
   total force (both PM levels + PP) against the reference V_p R(r, b_PP)/(4 pi)
   of Eq. (force_decomp), for separations from 0.05 to 24 Mpc/h.  The same
   pairs with the periodic coarse table instead show the pull of the periodic
   images at large r, so a missing or wrong isolation factor fails.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from inputs.workloads import ISO_PAIRS
from inputs.zeldovich import ios_from_positions
from oracle import kernels as K
from oracle import mesh as M
from oracle import pp as P
from oracle.kdk import pp_params


def test_isolation_factor_is_the_transform_of_the_truncated_force():
    L = 7.3
    for k in (0.05, 0.3, 1.1, 2.9, 8.0):
        # 3-D transform of a radial function: 4 pi int f(r) sin(kr)/(kr) r^2 dr
        val, _ = integrate.quad(lambda r: (-1.0 / r + 1.0 / L) * math.sin(k * r) / k * r, 0.0, L, limit=400)
        ft = 4.0 * math.pi * val
        # the untruncated potential -1/r transforms to -4 pi / k^2
        assert ft / (-4.0 * math.pi / k ** 2) == pytest.approx(float(K.isolation_factor(k, L)), rel=1e-9, abs=1e-12)
    assert K.isolation_factor(3.0, None) == 1.0


def test_green_table_isolation_only_changes_images_off_the_axes():
    # on the box's own modes along an axis, |k| L_iso = pi m: sinc vanishes and
    # the factor is 1; elsewhere it is not
    n, iso = 16, 8.0
    gi = K.green(n, 3.5, None, iso=iso)
    gp = K.green(n, 3.5, None)
    assert np.abs(gi - gp).max() > 1e-3 * np.abs(gp).max()
    g_axis_i = K.green_at(n, [(3, 0, 0), (0, 5, 0)], 3.5, None, alias=0, iso=iso)
    g_axis_p = K.green_at(n, [(3, 0, 0), (0, 5, 0)], 3.5, None, alias=0)
    np.testing.assert_allclose(g_axis_i, g_axis_p, rtol=1e-12)


@pytest.fixture(scope="module")
def pairs():
    """Per pair: separation r, F.r_hat / R - 1 and angle, isolated and periodic."""
    w = ISO_PAIRS
    params = M.level_params(w)
    gi = M.green_tables(w)
    gp0 = K.green(params[0][0], params[0][2], None)          # coarse level, periodic
    b_pp, b_cut = pp_params(w)
    rng = np.random.Generator(np.random.Philox(w.seed))
    rows = []
    for r in np.geomspace(0.05, 24.0, 44):
        xa = rng.uniform(0.0, w.box, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.stack([xa, (xa + r * u) % w.box], axis=1)
        st = ios_from_positions(pos, np.zeros((3, 2)), w.n_ios, w.box)
        off, count, start = st["off"], st["count"], st["start"]
        x = M.positions(off, count, w.n_ios, w.box)
        d = x[:, 1] - x[:, 0]
        d -= w.box * np.rint(d / w.box)
        rr = float(np.linalg.norm(d))
        ref = w.box ** 3 / 2 / (4 * math.pi) * float(K.reference_force(rr, b_pp))
        (n0, h0, _, _), (n1, h1, _, _) = params
        f_fine, _ = M.pm_force_level(off, count, w.n_ios, n1, h1, gi[1])
        f_pp = P.pp_force(off, count, start, w.n_ios, w.box, b_pp, b_cut)
        row = [rr]
        for g0 in (gi[0], gp0):
            f_c, _ = M.pm_force_level(off, count, w.n_ios, n0, h0, g0)
            f0 = (f_c + f_fine + f_pp)[:, 0]                  # force on particle 0, towards 1
            row.append(float(np.dot(f0, d) / rr) / ref - 1.0)
            row.append(math.acos(max(-1.0, min(1.0, float(np.dot(f0, d)) / (np.linalg.norm(f0) * rr)))))
        rows.append(row)
    return np.array(rows)


def _bins(rows):
    for lo, hi in ((0.05, 0.3), (0.3, 2.0), (2.0, 6.0), (6.0, 12.0), (12.0, 18.0), (18.0, 24.1)):
        m = (rows[:, 0] >= lo) & (rows[:, 0] < hi)
        yield lo, hi, rows[m]


def test_pairwise_force_accuracy_isolated(pairs):
    for lo, hi, b in _bins(pairs):
        e, th = b[:, 1], b[:, 2]
        # mean residual (bias) at the percent level, scatter of a few percent
        # at the force-matching scales b_PP < r < b_coarse, the direction
        # within a few degrees
        assert abs(e.mean()) < 0.02, (lo, hi, e.mean())
        assert e.std() < 0.04, (lo, hi, e.std())
        assert np.abs(e).max() < 0.1, (lo, hi, np.abs(e).max())
        assert th.max() < 0.1, (lo, hi, th.max())
    # well inside the PP range the force is the PP kernel's to rounding
    small = pairs[pairs[:, 0] < 0.1]
    assert np.abs(small[:, 1]).max() < 2e-3


def test_periodic_table_feels_the_images(pairs):
    far = pairs[pairs[:, 0] >= 14.0]
    # the periodic images pull back: the radial force falls short by several
    # percent (growing with r), the isolated table does not
    assert far[:, 3].mean() < -0.05
    assert abs(far[:, 1].mean()) < 0.02


def _golden(name):
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_pairwise_accuracy_within_the_papers_reported_envelope(pairs):
    # the paper's TSC, three-level test reports 2 % rms and 7 % max; the same
    # test on this method's CIC two-level layout stays within 1.5x of both
    ref = _golden("pairwise_accuracy.txt")
    e = pairs[:, 1]
    assert np.sqrt(np.mean(e ** 2)) <= 1.5 * ref["rms_relative_error"]
    assert np.abs(e).max() <= 1.5 * ref["max_relative_error"]
