"""Pins of the oracle's TSC assignment (the paper's Eq. filter): partition of
unity, the first and second moments of the 1-D weights, the transform of the
assignment of one particle against sinc^3, and the physics the CIC variant is
pinned by (zero self-force, momentum conservation, Newtonian far field)."""
import math

import numpy as np
import pytest

from inputs import C1
from inputs.workloads import Level
from inputs.zeldovich import ios_from_positions, random_ios
from oracle import kernels as K
from oracle import kdk as D
from oracle import mesh as M


def test_tsc_weights_moments():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 40 * M.FIX, 5000)
    for s in (-1, 0, 1):
        i, w = M.tsc_weights_1d(X, s)
        xm = (X >> s) if s >= 0 else (X << -s)
        u = xm / M.FIX
        w = np.stack(w)
        centres = (i + np.array([-1, 0, 1])[:, None]) + 0.5
        assert np.all(w >= 0)
        assert np.allclose(w.sum(axis=0), 1.0, atol=1e-15)
        assert np.allclose((w * centres).sum(axis=0), u, atol=1e-12)            # centre of mass kept
        assert np.allclose((w * (centres - u) ** 2).sum(axis=0), 0.25, atol=1e-12)  # variance 3 * 1/12


def test_tsc_transform_of_one_particle_is_aliased_sinc_cubed():
    # a particle at a cell centre: the DFT of its sampled cloud is, per axis,
    # the alias sum of W(k) = sinc^3(k/2) over k + 2 pi n, whose closed form
    # for the sampled quadratic spline is 3/4 + cos(k)/4 (Hockney & Eastwood)
    n = 16
    st = ios_from_positions(np.array([[5.5], [7.5], [9.5]]), np.zeros((3, 1)), n, float(n))
    rho = M.density_tsc(st["off"], st["count"], n, n) + 1.0   # (n^3/N) W with N = 1
    spec = np.abs(np.fft.rfftn(rho / n ** 3))
    kx, ky, kz = K.half_spectrum_wavenumbers(n)
    closed = lambda k: 0.75 + 0.25 * np.cos(k)
    assert np.allclose(spec, np.abs(closed(kx) * closed(ky) * closed(kz)), atol=1e-12)
    k = np.linspace(-np.pi, np.pi, 41)
    alias = sum(K.assignment_transform(k + 2 * np.pi * m, 3) for m in range(-4000, 4001))
    assert np.allclose(alias, closed(k), atol=1e-9)


def test_tsc_force_physics():
    w = C1.with_(n_ios=8, box=16.0, levels=(Level(16, 2.0),), b_pp=0.2, assign_order=3)
    greens = M.green_tables(w)
    # one particle: no self-force
    st = ios_from_positions(np.array([[3.3], [7.9], [12.2]]), np.zeros((3, 1)), 8, 16.0)
    f = D.total_force(st["off"], st["count"], st["start"], w, greens)
    assert np.abs(f).max() < 1e-12
    # momentum conservation on a clumped set
    st = random_ios(600, 8, 16.0, seed=4, clustered=0.5)
    f = D.total_force(st["off"], st["count"], st["start"], w, greens)
    assert np.abs(f.sum(axis=1)).max() < 1e-10 * np.abs(f).sum()
    # two particles far apart (beyond the softening): Newtonian attraction
    wl = C1.with_(n_ios=16, box=64.0, levels=(Level(64, 2.0),), b_pp=0.2, assign_order=3)
    gl = M.green_tables(wl)
    sep = 10.3
    pos = np.array([[20.0, 20.0 + sep], [31.7, 31.7], [12.9, 12.9]])
    st = ios_from_positions(pos, np.zeros((3, 2)), 16, 64.0)
    f = D.total_force(st["off"], st["count"], st["start"], wl, gl)
    vp = 64.0 ** 3 / 2
    newton = vp / (4 * math.pi * sep ** 2)
    xs = M.positions(st["off"], st["count"], 16, 64.0)
    i_left = int(np.argmin(xs[0]))
    assert f[0, i_left] > 0
    assert abs(f[0, i_left] / newton - 1.0) < 0.05
