"""Pins of the oracle's total PM+PP force and KDK against physics and direct summation."""
import math

import numpy as np
import pytest
from scipy import integrate

from inputs import C1
from inputs.workloads import Level
from inputs.zeldovich import growth_d, growth_f, hubble_e, ios_from_positions, random_ios
from oracle import ewald as E
from oracle import kdk as KD
from oracle import mesh as M
from oracle import pp as P

# beta = 3.5 variant of C1 with 4-cell IOS/PP cells: the paper's default softening
C1_B35 = C1.with_(n_ios=16, levels=(Level(64, 3.5),))


def _force(st, w, greens=None):
    return KD.total_force(st["off"], st["count"], st["start"], w, greens)


def _unit(w):
    """Force between two particles one IOS cell apart."""
    return w.box ** 3 / (4 * math.pi * (w.box / w.n_ios) ** 2)


def test_single_particle_feels_no_force():
    for w in (C1, C1_B35):
        st = ios_from_positions(np.array([[10.37], [3.1], [41.9]]), np.zeros((3, 1)), w.n_ios, w.box)
        f = _force(st, w)
        assert np.abs(f).max() < 1e-10 * _unit(w)


def test_uniform_lattice_feels_no_force():
    n = 16
    g = (np.arange(n) + 0.5) * (C1.box / n)
    q = np.stack(np.meshgrid(g, g, g, indexing="ij")[::-1]).reshape(3, -1)
    w = C1.with_(n_ios=16, levels=(Level(32, 2.0),), b_pp=0.4)
    st = ios_from_positions(q, np.zeros_like(q), w.n_ios, w.box)
    f = _force(st, w)
    assert np.abs(f).max() < 1e-9 * _unit(w) / n ** 3


def test_momentum_is_conserved():
    st = random_ios(400, 32, C1.box, seed=5, clustered=0.6)
    f = _force(st, C1)
    assert np.abs(f.sum(axis=1)).max() < 1e-10 * np.abs(f).sum()


def test_pp_cell_list_matches_brute_force_and_is_antisymmetric():
    w = C1
    st = random_ios(600, 32, w.box, seed=9, clustered=0.7)
    b_pp, b_cut = KD.pp_params(w)
    f = P.pp_force(st["off"], st["count"], st["start"], w.n_ios, w.box, b_pp, b_cut)
    x = M.positions(st["off"], st["count"], w.n_ios, w.box)
    fb = P.pp_force_brute(x, w.box, b_pp, b_cut)
    assert np.allclose(f, fb, rtol=1e-12, atol=1e-12 * np.abs(fb).max())
    assert np.abs(f.sum(axis=1)).max() < 1e-12 * np.abs(f).sum()
    sub = P.pp_force(st["off"], st["count"], st["start"], w.n_ios, w.box, b_pp, b_cut,
                     targets=[3, 77, 500])
    assert np.array_equal(sub, f[:, [3, 77, 500]])
    at = P.pp_force_at(st["off"], st["count"], st["start"], w.n_ios, w.box, b_pp, b_cut, [0, 3, 77, 500, 599])
    assert np.allclose(at, f[:, [0, 3, 77, 500, 599]], rtol=1e-12, atol=1e-12 * np.abs(f).max())
    # the vectorised point evaluator, on every particle (repeats included)
    t = np.concatenate([np.arange(600), [3, 3, 599]])
    many = P.pp_force_at_many(st["off"], st["count"], st["start"], w.n_ios, w.box, b_pp, b_cut, t)
    assert np.allclose(many, f[:, t], rtol=1e-12, atol=1e-12 * np.abs(f).max())


def _ewald_errors(w, n, seed):
    st = random_ios(n, w.n_ios, w.box, seed=seed)
    f = _force(st, w)
    x = M.positions(st["off"], st["count"], w.n_ios, w.box)
    fe = E.ewald_force(x, w.box, w.b_pp)
    return np.linalg.norm(f - fe, axis=0) / np.linalg.norm(fe, axis=0)


def test_total_force_matches_ewald_direct_sum_default_softening():
    # paper's default beta = 3.5: a few per cent (Sec. 3.1: rms 2%, max 7% for TSC)
    err = _ewald_errors(C1_B35, 48, seed=21)
    assert np.sqrt(np.mean(err ** 2)) < 0.05 and err.max() < 0.15


def test_total_force_matches_ewald_direct_sum_two_cell_softening():
    # CIC with a 2-cell PP range: looser envelope, errors at the matching scale
    err = _ewald_errors(C1, 48, seed=22)
    assert np.median(err) < 0.12 and np.sqrt(np.mean(err ** 2)) < 0.2


@pytest.mark.parametrize("sep", [8.0, 12.0, 20.0])
def test_two_body_force_is_newtonian_beyond_a_few_cells(sep):
    w = C1
    rng = np.random.default_rng(int(sep))
    for _ in range(4):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        c = rng.uniform(0, w.box, 3)
        pos = np.stack([c, (c + sep * u) % w.box], axis=1)
        st = ios_from_positions(pos, np.zeros((3, 2)), w.n_ios, w.box)
        f = _force(st, w)
        x = M.positions(st["off"], st["count"], w.n_ios, w.box)
        fe = E.ewald_force(x, w.box, w.b_pp)
        assert np.linalg.norm(f[:, 0] - fe[:, 0]) < 0.03 * np.linalg.norm(fe[:, 0])
        # attractive: the force on particle 0 points towards particle 1
        d = x[:, 1] - x[:, 0]
        d -= w.box * np.rint(d / w.box)
        assert f[:, 0] @ d > 0


def _pancake(w, amp, a):
    """Plane-wave Zel'dovich state: psi_x = amp sin(2 pi q_x / L)."""
    n = w.n_p
    g = (np.arange(n) + 0.5) * (w.box / n)
    q = np.stack(np.meshgrid(g, g, g, indexing="ij")[::-1]).reshape(3, -1)
    psi = np.zeros_like(q)
    psi[0] = amp * np.sin(2 * math.pi * q[0] / w.box)
    d, f = growth_d(a, w.omega_m, w.omega_l), growth_f(a, w.omega_m, w.omega_l)
    e = float(hubble_e(a, w.omega_m, w.omega_l))
    pos = q + d * psi
    mom = a * a * e * f * d * psi
    st = ios_from_positions(pos, mom, w.n_ios, w.box)
    return st, d, psi, pos


def test_zeldovich_pancake_force():
    # linear theory: F = -grad u = D psi at the particle
    w = C1.with_(n_p=32)
    a = 0.1
    st, d, _, _ = _pancake(w, amp=1.0, a=a)
    f = _force(st, w)
    x = M.positions(st["off"], st["count"], w.n_ios, w.box)
    # invert x = q + D amp sin(k q) for q by fixed-point iteration
    k = 2 * math.pi / w.box
    q = x[0].copy()
    for _ in range(50):
        q = x[0] - d * 1.0 * np.sin(k * q)
    want = d * np.sin(k * q)
    amp_lin = d * 1.0 * k                                  # delta amplitude, small
    assert amp_lin < 0.02                                  # linear regime
    assert np.abs(f[0] - want).max() < 0.02 * d
    assert np.abs(f[1:]).max() < 1e-3 * d


def test_zeldovich_pancake_kdk_tracks_linear_growth():
    w = C1.with_(n_p=32)
    a0, a1, steps = 0.05, 0.2, 6
    st, d0, _, _ = _pancake(w, amp=2.0, a=a0)
    state = dict(off=st["off"], count=st["count"], start=st["start"],
                 vel=st["vel"].astype(np.float64), acc=None)
    greens = M.green_tables(w)
    a_s = np.linspace(a0, a1, steps + 1)
    for i in range(steps):
        state = KD.kdk_step(state, w, a_s[i], a_s[i + 1], greens)
    x = M.positions(state["off"], state["count"], w.n_ios, w.box)
    k = 2 * math.pi / w.box
    d1 = growth_d(a1, w.omega_m, w.omega_l)
    # mean displacement amplitude from the first Fourier mode of x - q along x
    g = (np.arange(w.n_p) + 0.5) * (w.box / w.n_p)
    # particles keep their lattice plane ordering in x; recover q by inversion
    q = x[0].copy()
    for _ in range(80):
        q = x[0] - d1 * 2.0 * np.sin(k * q)
    disp = x[0] - q
    amp = 2 * np.mean(disp * np.sin(k * q))
    assert abs(amp / (d1 * 2.0) - 1) < 0.03


def test_kick_drift_integrals():
    # Einstein-de Sitter closed forms
    a0, a1 = 0.02, 0.5
    assert KD.kick_integral(a0, a1, 1.0, 0.0) == pytest.approx(2 * (math.sqrt(a1) - math.sqrt(a0)), rel=1e-13)
    assert KD.drift_integral(a0, a1, 1.0, 0.0) == pytest.approx(2 * (1 / math.sqrt(a0) - 1 / math.sqrt(a1)), rel=1e-13)
    # flat LCDM against adaptive quadrature
    e = lambda a: math.sqrt(0.3 / a ** 3 + 0.7)
    for lo, hi in ((0.02, 0.0396), (0.5, 1.0)):
        k, _ = integrate.quad(lambda a: 1 / (a * a * e(a)), lo, hi, epsrel=1e-13)
        dr, _ = integrate.quad(lambda a: 1 / (a ** 3 * e(a)), lo, hi, epsrel=1e-13)
        assert KD.kick_integral(lo, hi, 0.3, 0.7) == pytest.approx(k, rel=1e-12)
        assert KD.drift_integral(lo, hi, 0.3, 0.7) == pytest.approx(dr, rel=1e-12)


def test_drift_rebin_fixed_point():
    st = random_ios(200, 8, 16.0, seed=4, clustered=0.5)
    v0 = np.zeros((3, 200))
    off, count, start, vel = KD.drift_rebin(st["off"], st["count"], v0, 1.0, 8, 16.0)
    assert np.array_equal(off, st["off"]) and np.array_equal(count, st["count"])
    # move every particle by exactly one IOS cell along +y (s_ios = 2): same offsets,
    # counts rolled by one row, order stable
    v = np.zeros((3, 200))
    v[1] = 2.0
    off2, count2, _, _ = KD.drift_rebin(st["off"], st["count"], v, 1.0, 8, 16.0)
    assert np.array_equal(count2.reshape(8, 8, 8), np.roll(st["count"].reshape(8, 8, 8), 1, axis=1))
    X0 = M.fixed_coords(st["off"], st["count"], 8)
    X1 = M.fixed_coords(off2, count2, 8)
    X0[1] = (X0[1] + (1 << 16)) % (8 << 16)
    key0 = (X0[2] >> 16) * 64 + (X0[1] >> 16) * 8 + (X0[0] >> 16)
    assert np.array_equal(X1, X0[:, np.argsort(key0, kind="stable")])
