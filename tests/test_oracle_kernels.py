"""Pins of the oracle's kernel functions (Sec. 2.1) against quadrature and closed forms."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kernels as K


@pytest.mark.parametrize("b", [0.3, 1.0, 2.0, 7.0])
def test_profile_has_unit_mass(b):
    # Eq. (denprofile) integrates to one
    m, _ = integrate.quad(lambda r: 4 * math.pi * r * r * K.density_profile(r, b), 0, b / 2,
                          epsabs=0, epsrel=1e-13)
    assert abs(m - 1.0) < 1e-12


@pytest.mark.parametrize("b", [0.5, 2.0])
def test_reference_force_continuity_and_limits(b):
    eps = 1e-9
    for r in (0.5 * b, b):
        lo, hi = K.reference_force(r * (1 - eps), b), K.reference_force(r * (1 + eps), b)
        assert abs(lo - hi) < 1e-6 * abs(lo)
    assert abs(K.reference_force(0.5 * b, b) * b * b - 2.7714285714) < 1e-8
    r = np.array([1.0, 1.5, 3.0]) * b
    assert np.allclose(K.reference_force(r, b), 1 / r ** 2, rtol=1e-14)
    r0 = 1e-6 * b                           # R ~ 64 r / (5 b^3) near 0 (F(0) = 0)
    assert abs(K.reference_force(r0, b) / (64 * r0 / (5 * b ** 3)) - 1) < 1e-9
    assert K.reference_force(0.0, b) == 0.0


@pytest.mark.parametrize("b", [1.0, 3.5])
def test_profile_transform_is_fourier_transform_of_profile(b):
    # S(k) = int 4 pi r^2 S(r) sin(kr)/(kr) dr, by quadrature
    for k in (0.01, 0.7, 2.0, 5.0, 11.0, 30.0):
        val, _ = integrate.quad(
            lambda r: 4 * math.pi * r * r * K.density_profile(r, b) * np.sinc(k * r / math.pi),
            0, b / 2, epsabs=0, epsrel=1e-13, limit=200)
        assert abs(K.profile_transform(k, b) - val) < 1e-11 * max(1.0, abs(val)) + 1e-14


def test_profile_transform_series_branch_is_continuous():
    b = 2.0
    k_lo, k_hi = 0.5 * (1 - 1e-12) * 2 / b, 0.5 * 2 / b
    assert abs(K.profile_transform(k_lo, b) - K.profile_transform(k_hi, b)) < 1e-13
    assert K.profile_transform(0.0, b) == pytest.approx(1.0, abs=1e-15)
    # first series terms: 1 - x^2/15 + x^4/560
    x = 0.01
    assert abs(K.profile_transform(2 * x / b, b) - (1 - x * x / 15 + x ** 4 / 560)) < 1e-15


@pytest.mark.parametrize("b", [1.0, 2.0])
def test_reference_force_is_transform_of_profile_squared(b):
    # R(r) = (2/pi) int S(k)^2 k j1(kr) dk  (force between two S-profiles)
    kmax = 400.0 / b
    k = np.linspace(1e-9, kmax, 400001)
    s2 = K.profile_transform(k, b) ** 2
    for r in (0.1 * b, 0.3 * b, 0.6 * b, 0.9 * b, 1.4 * b):
        x = k * r
        j1 = np.where(x > 1e-3, (np.sin(x) - x * np.cos(x)) / np.where(x > 1e-3, x, 1) ** 2, x / 3)
        val = 2 / math.pi * integrate.simpson(s2 * k * j1, x=k)
        assert abs(val - K.reference_force(r, b)) < 2e-5 * K.reference_force(r, b)


def test_fd_transform_is_dft_of_stencil():
    # Eq. (diff): D(n) = 4/3 [d(n+1) - d(n-1)]/2 - 1/3 [d(n+2) - d(n-2)]/4
    n = 16
    stencil = np.zeros(n)
    stencil[-1] += 4 / 3 / 2      # delta(n+1) at n = -1
    stencil[1] -= 4 / 3 / 2
    stencil[-2] -= 1 / 3 / 4
    stencil[2] += 1 / 3 / 4
    kk = 2 * math.pi * np.fft.fftfreq(n)
    assert np.allclose(np.fft.fft(stencil), 1j * K.fd_transform(kk), atol=1e-14)


def test_cic_alias_sum_matches_closed_form():
    # sum_n sinc^4((k + 2 pi n)/2) = 1 - 2/3 sin^2(k/2) (Hockney & Eastwood)
    k = np.linspace(0, math.pi, 33)
    s = sum(K.assignment_transform(k + 2 * math.pi * m) ** 2 for m in range(-2, 3))
    exact = 1 - 2 / 3 * np.sin(k / 2) ** 2
    rel = np.abs(s / exact - 1)
    assert rel.max() < 2e-3 and rel[0] == 0
    s_full = sum(K.assignment_transform(k + 2 * math.pi * m) ** 2 for m in range(-400, 401))
    assert np.allclose(s_full, exact, rtol=2e-8)


@pytest.fixture(scope="module", params=["cic", "tsc-iso"])
def g24(request):
    # the symmetries the GPU's reduced table storage relies on, for CIC and
    # for TSC with an isolated coarsest level
    if request.param == "cic":
        return K.green(24, 2.0, 9.0)
    return K.green(24, 3.5, None, order=3, iso=5.0)


def test_green_symmetries(g24):
    g = g24
    n = 24
    assert g[0, 0, 0] == 0.0
    assert np.all(np.isfinite(g))
    # full spectrum via Hermitian symmetry, then test cubic symmetry
    full = np.empty((n, n, n))
    full[:, :, : n // 2 + 1] = g
    idx = (-np.arange(n)) % n
    full[:, :, n // 2 + 1:] = g[idx][:, idx][:, :, 1: n // 2][:, :, ::-1]
    assert np.allclose(full, np.transpose(full, (1, 0, 2)), rtol=1e-12, atol=1e-14)
    assert np.allclose(full, np.transpose(full, (2, 1, 0)), rtol=1e-12, atol=1e-14)
    assert np.allclose(full, full[idx], rtol=1e-12, atol=1e-14)          # kz -> -kz
    assert np.allclose(full, full[:, :, idx], rtol=1e-12, atol=1e-14)    # kx -> -kx
    # |d| = 0 on the corners of the Brillouin zone: G = 0
    assert g[n // 2, n // 2, n // 2] == 0.0 and g[0, n // 2, 0] == 0.0


def test_green_continuum_limit():
    # untruncated level: G -> -S(k,b)^2 / k^2 at small k
    n, b = 96, 2.0
    g = K.green(n, b, None)
    kx, _, _ = K.half_spectrum_wavenumbers(n)
    for m in (1, 2, 3):
        k = kx[0, 0, m]
        ref = -K.profile_transform(k, b) ** 2 / k ** 2
        # FD and assignment corrections enter at O(k^2)
        assert abs(g[0, 0, m] / ref - 1) < 0.25 * k * k
    # truncated level: G -> -(S^2(b) - S^2(b_t)) / k^2
    gt = K.green(n, b, 14.0)
    k = kx[0, 0, 1]
    ref = -(K.profile_transform(k, b) ** 2 - K.profile_transform(k, 14.0) ** 2) / k ** 2
    assert abs(gt[0, 0, 1] / ref - 1) < 0.25 * k * k


@pytest.mark.parametrize("n,order,iso", [(16, 2, None), (24, 2, None), (12, 3, 4.0)])
def test_green_by_symmetry_equals_full_table(n, order, iso):
    # the table built once per sorted |m| triple and expanded by the symmetries
    # equals the mode-by-mode table up to the order of the alias sum
    tri = K.sorted_mode_triples(n)
    m = n // 2
    assert len(tri) == (m + 1) * (m + 2) * (m + 3) // 6
    assert np.all((tri[:, 0] <= tri[:, 1]) & (tri[:, 1] <= tri[:, 2]) & (tri[:, 2] <= m))
    g = K.green(n, 2.0, 7.0, order=order, iso=iso)
    gs = K.green_by_symmetry(n, 2.0, 7.0, order=order, iso=iso, chunk=37)
    assert np.abs(gs - g).max() <= 1e-13 * np.abs(g).max()


def test_velocity_codec_follows_the_binary16_format():
    # pins of the compressed velocity storage from the binary16 format itself:
    # 11 significant bits, so the round trip errs by half an ulp of the code
    # plus the FP32 roundings of the division and the decode: within one ulp
    # (2^-11 of the scale for codes in [1/2, 1), 2^-12 below 1/2); the
    # largest component of each cell is +-1 x scale exactly; empty and
    # all-zero cells give zero codes; powers of two times the scale are exact
    from oracle import kdk as KD
    rng = np.random.default_rng(7)
    count = np.array([0, 5, 1, 0, 7, 3], dtype=np.int32)
    n = int(count.sum())
    vel = (rng.normal(size=(3, n)) * rng.lognormal(0.0, 2.0, size=n)).astype(np.float32)
    vel[:, 5] = 0.0                                # the one-particle cell: all zero
    vel[1, 6] = 0.25 * np.abs(vel[:, 6:13]).max()  # a power of two times its cell's scale
    codes, scale = KD.encode_velocities(vel, count)
    assert codes.dtype == np.float16 and scale.dtype == np.float32
    assert scale[0] == 0 and scale[3] == 0 and scale[2] == 0
    back = KD.decode_velocities(codes, scale, count).astype(np.float64)
    cell = np.repeat(np.arange(count.size), count)
    s = scale[cell].astype(np.float64)
    ratio = np.abs(vel / np.where(s > 0, s, 1.0))
    ulp = np.where(ratio >= 0.5, 2.0 ** -11, 2.0 ** -12)
    assert np.all(np.abs(back - vel) <= ulp * s * (1 + 1e-6) + 1e-30)
    assert np.all(np.abs(codes.astype(np.float32)).max(axis=0)[count[cell] > 0] <= 1.0)
    for c in np.nonzero(scale > 0)[0]:
        sel = cell == c
        assert np.abs(codes[:, sel].astype(np.float32)).max() == 1.0
    assert back[1, 6] == vel[1, 6]
    assert not codes[:, 5].any()
