"""Pins of the oracle's integer CIC deposit, density conversion, solve and FD."""
import math
from fractions import Fraction

import numpy as np
import pytest

from inputs.zeldovich import random_ios
from oracle import kernels as K
from oracle import mesh as M


def _exact_cic(X, n_ios, n_mesh):
    """Brute force: CIC weights from the definition, with exact rationals.

    The position in mesh cells is floored to 2^-16 of a mesh cell; each of the
    n_mesh^3 cells gets prod_d max(0, 1 - |x_d - (j_d + 1/2)|) (periodic)."""
    q = Fraction(n_ios, n_mesh)
    out = {}
    for p in range(X.shape[1]):
        xs = []
        for d in range(3):
            xm = Fraction(int(X[d, p]), 1 << 16) / q                # mesh cells
            xs.append(Fraction(math.floor(xm * (1 << 16)), 1 << 16))
        w1 = []
        for d in range(3):
            ws = {}
            for j in range(n_mesh):
                dist = abs(xs[d] - (j + Fraction(1, 2)))
                dist = min(dist, n_mesh - dist)
                if dist < 1:
                    ws[j] = 1 - dist
            w1.append(ws)
        for jz, wz in w1[2].items():
            for jy, wy in w1[1].items():
                for jx, wx in w1[0].items():
                    key = (jz, jy, jx)
                    out[key] = out.get(key, 0) + wx * wy * wz
    return out


@pytest.mark.parametrize("n_ios,n_mesh", [(4, 8), (4, 2), (4, 4), (8, 16)])
def test_integer_cic_equals_exact_rational_cic(n_ios, n_mesh):
    st = random_ios(12, n_ios, 10.0, seed=7)
    acc = M.deposit_u64(st["off"], st["count"], n_ios, n_mesh)
    X = M.fixed_coords(st["off"], st["count"], n_ios)
    exact = _exact_cic(X, n_ios, n_mesh)
    got = {k: Fraction(int(acc[k]), 1 << 48) for k in zip(*np.nonzero(acc))}
    exact = {k: v for k, v in exact.items() if v != 0}
    assert got == exact


def test_deposit_conserves_mass_and_is_order_free():
    st = random_ios(3000, 16, 32.0, seed=3, clustered=0.5)
    for n_mesh in (8, 32, 64):
        acc = M.deposit_u64(st["off"], st["count"], 16, n_mesh)
        assert int(acc.sum(dtype=np.uint64)) == 3000 << 48


def test_particle_at_cell_centre_fills_one_cell():
    off = np.full((3, 1), 1 << 15, dtype=np.uint16)
    count = np.zeros(4 ** 3, dtype=np.int32)
    count[1 + 4 * (2 + 4 * 3)] = 1
    acc = M.deposit_u64(off, count, 4, 4)
    assert acc[3, 2, 1] == 1 << 48 and int(acc.sum()) == 1 << 48
    acc8 = M.deposit_u64(off, count, 4, 8)          # fine mesh: corner of 8 cells
    assert sorted(set(acc8[acc8 > 0].tolist())) == [1 << 45]


def _rn32_exact(v):
    """Round a non-negative Python int to the nearest float32 (ties to even)."""
    if v < (1 << 24):
        return float(v)
    e = v.bit_length() - 24
    q, rem = v >> e, v & ((1 << e) - 1)
    half = 1 << (e - 1)
    if rem > half or (rem == half and q & 1):
        q += 1
    return float(q) * 2.0 ** e


def test_uint64_to_float32_rounding_is_correct():
    rng = np.random.default_rng(0)
    vals = [0, 1, (1 << 24) + 1, (1 << 25) + 2, (1 << 25) + 6, (1 << 48) + (1 << 24),
            (1 << 63) + (1 << 39), (1 << 64) - 1, (1 << 53) + 1, 3 << 40 | (1 << 16)]
    vals += [int(x) for x in rng.integers(0, 1 << 62, 2000, dtype=np.uint64)]
    vals += [(int(x) << 16) | (1 << 15) for x in rng.integers(1 << 24, 1 << 40, 500, dtype=np.uint64)]
    arr = np.array(vals, dtype=np.uint64).astype(np.float32)
    assert [float(a) for a in arr] == [np.float32(_rn32_exact(v)) for v in vals]


def test_density_spec_matches_definition():
    st = random_ios(500, 8, 16.0, seed=11)
    acc = M.deposit_u64(st["off"], st["count"], 8, 16)
    d32 = M.density_fp32(acc, 500)
    m = M.mean_integer(500, 16)
    scale = np.float32(16 ** 3 / 500 * 2.0 ** -48)
    for idx in [(0, 0, 0), (3, 5, 7), (15, 15, 15)]:
        delta = int(acc[idx]) - m
        want = np.float32(np.float32(np.sign(delta) * _rn32_exact(abs(delta))) * scale)
        assert d32[idx] == want
    rho = M.density(acc, 500)
    assert abs(rho.mean()) < 1e-12                         # overdensity: mean ~ 0
    assert np.allclose(rho + 1.0, acc.astype(np.float64) * 2.0 ** -48 * 16 ** 3 / 500, atol=1e-12)


def test_fd_gradient_equals_spectral_derivative():
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((8, 12, 16))
    e = M.fd_gradient(phi)
    for d, axis in enumerate((2, 1, 0)):
        n = phi.shape[axis]
        kk = 2 * np.pi * np.fft.fftfreq(n)
        shape = [1, 1, 1]
        shape[axis] = n
        spec = np.fft.ifft(np.fft.fft(phi, axis=axis) * (1j * K.fd_transform(kk)).reshape(shape),
                           axis=axis).real
        assert np.allclose(e[d], spec, atol=1e-12)


def test_solve_recovers_poisson_for_single_mode():
    # G ~ -1/k^2 (b -> 0 would be exact); check lap(phi) = rho for a long mode
    n = 32
    x = np.arange(n)
    rho = np.cos(2 * np.pi * x / n)[None, None, :] * np.ones((n, n, 1))
    g = K.green(n, 0.5, None)
    phi = M.solve_potential(rho, g)
    k = 2 * np.pi / n
    # phi = G(k) rho exactly for a single mode
    assert np.allclose(phi, g[0, 0, 1] * rho, atol=1e-12)
    assert abs(g[0, 0, 1] * k * k + 1) < 0.25 * k * k    # O(k^2) FD/assignment terms


@pytest.mark.parametrize("n_ios,n_mesh", [(8, 16), (8, 4), (8, 8), (4, 16)])
def test_point_deposit_equals_full_deposit(n_ios, n_mesh):
    st = random_ios(700, n_ios, 16.0, seed=8, clustered=0.5)
    acc = M.deposit_u64(st["off"], st["count"], n_ios, n_mesh).ravel()
    rng = np.random.default_rng(2)
    cells = rng.integers(0, n_mesh ** 3, 60)
    at = M.deposit_u64_at(st["off"], st["count"], st["start"], n_ios, n_mesh, cells)
    assert np.array_equal(at, acc[cells])


def test_point_green_equals_full_table():
    g = K.green(24, 2.0, 9.0)
    rng = np.random.default_rng(4)
    modes = np.stack([rng.integers(0, 13, 80), rng.integers(0, 24, 80), rng.integers(0, 24, 80)], 1)
    modes[:4] = [[12, 12, 12], [0, 0, 0], [12, 0, 5], [3, 12, 12]]
    assert np.array_equal(K.green_at(24, modes, 2.0, 9.0), g[modes[:, 2], modes[:, 1], modes[:, 0]])


@pytest.mark.parametrize("n_ios,n_mesh", [(16, 32), (16, 8), (12, 24), (16, 16)])
def test_point_level_force_equals_full_gather(n_ios, n_mesh):
    # pm_force_level_at forms the 4-point difference only at the gathered
    # cells; it must equal the whole-mesh difference followed by the gather,
    # wrapped cells and every level ratio included
    st = random_ios(3000, n_ios, float(n_ios), seed=5, clustered=0.4)
    acc = M.deposit_u64(st["off"], st["count"], n_ios, n_mesh)
    phi = M.solve_potential(M.density(acc, 3000), K.green(n_mesh, 2.0, None))
    h = n_ios / n_mesh
    full = -h * M.interpolate(M.fd_gradient(phi), st["off"], st["count"], n_ios)
    t = np.random.default_rng(0).integers(0, 3000, 200)
    at = M.pm_force_level_at(phi, st["off"], st["count"], st["start"], n_ios, h, t)
    assert np.array_equal(at, full[:, t])
