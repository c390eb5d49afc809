"""Seeded synthetic inputs: Zel'dovich (1LPT) initial conditions in IOS form.

This module only *generates inputs*.  It holds none of the force method's
arithmetic (no deposit, Green's function, FFT solve, interpolation, PP or
KDK); both the CUDA path and the FP64 oracle consume what it returns.

Recipe (the paper sets its initial conditions with 1LPT, Sec. 3.2; its CAMB
spectrum is replaced here by a closed-form one):

* Gaussian white noise on the n_p^3 Lagrangian lattice, drawn with
  ``numpy.random.Generator(Philox(seed))``.
* Linear spectrum P(k) = A k T(k)^2 with the BBKS (1986) transfer function,
  shape parameter Gamma = Omega_m h, amplitude A fixed by sigma_8 (top-hat of
  8 Mpc/h) at a = 1.
* Linear growth D(a) of flat LCDM (D(1) = 1) and f = dlnD/dlna.
* Displacement psi(k) = i k delta(k) / k^2; positions x = q + D psi; canonical
  momenta p = a^2 E(a) f D psi  (H_0 = 1 units, lengths in Mpc/h).
* Quantisation to IOS: x / s_ios in fixed point with 2^16 sub-cells per IOS
  cell (round half to even, periodic wrap), particles sorted stably by linear
  cell id (x fastest) with the lattice index as tie-break; per-cell counts
  and their exclusive scan (starts).  Particles on the unperturbed lattice sit
  at IOS cell centres (offset 32768) when n_ios = n_p.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

FIX = 1 << 16  # fixed-point sub-cells per IOS cell


# ---------------------------------------------------------------- cosmology
def hubble_e(a, om, ol):
    """E(a) = H(a)/H_0 for a flat matter + Lambda universe."""
    return np.sqrt(om * np.asarray(a, dtype=np.float64) ** -3 + ol)


def _growth_unnormalised(a, om, ol):
    f = lambda x: 1.0 / (x * hubble_e(x, om, ol)) ** 3
    val, _ = integrate.quad(f, 0.0, a, epsabs=0.0, epsrel=1e-12, limit=200)
    return 2.5 * om * hubble_e(a, om, ol) * val, val


def growth_d(a, om, ol):
    """Linear growing mode D(a), normalised to D(1) = 1."""
    return _growth_unnormalised(a, om, ol)[0] / _growth_unnormalised(1.0, om, ol)[0]


def growth_f(a, om, ol):
    """f = dlnD/dlna of the growing mode."""
    e = hubble_e(a, om, ol)
    _, integral = _growth_unnormalised(a, om, ol)
    return -1.5 * om / (a ** 3 * e ** 2) + 1.0 / (a ** 2 * e ** 3 * integral)


# ----------------------------------------------------------------- spectrum
def bbks_transfer(k, om, h):
    """BBKS transfer function, k in h/Mpc, Gamma = Omega_m h."""
    k = np.asarray(k, dtype=np.float64)
    q = k / (om * h)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (np.log1p(2.34 * q) / (2.34 * q)
             * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)
    return np.where(q > 0, t, 1.0)


def _sigma_r_unit(r, om, h):
    """sigma(R) for P(k) = k T(k)^2 (A = 1)."""
    def integrand(lnk):
        k = math.exp(lnk)
        x = k * r
        w = 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3 if x > 1e-4 else 1.0 - x * x / 10.0
        return k ** 3 * k * float(bbks_transfer(k, om, h)) ** 2 * w * w / (2.0 * math.pi ** 2)
    val, _ = integrate.quad(integrand, math.log(1e-6), math.log(1e3), limit=500, epsrel=1e-10)
    return math.sqrt(val)


def spectrum_amplitude(om, h, sigma8):
    """A such that P(k) = A k T(k)^2 has sigma(8 Mpc/h) = sigma8 at a = 1."""
    return (sigma8 / _sigma_r_unit(8.0, om, h)) ** 2


def linear_power(k, om, h, sigma8):
    return spectrum_amplitude(om, h, sigma8) * k * bbks_transfer(k, om, h) ** 2


# ------------------------------------------------------------ random field
def gaussian_displacement(n, box, om, h, sigma8, seed):
    """Zel'dovich displacement field psi at a = 1 on an n^3 lattice.

    Returns (3, n, n, n) float64 indexed [d][z][y][x] (d = 0 is x)."""
    rng = np.random.Generator(np.random.Philox(seed))
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    kf = 2.0 * np.pi / box
    kz = np.fft.fftfreq(n, d=1.0 / n)[:, None, None] * kf
    ky = np.fft.fftfreq(n, d=1.0 / n)[None, :, None] * kf
    kx = np.fft.rfftfreq(n, d=1.0 / n)[None, None, :] * kf
    k2 = kx * kx + ky * ky + kz * kz
    k = np.sqrt(k2)
    pk = np.zeros_like(k)
    nz = k2 > 0
    pk[nz] = linear_power(k[nz], om, h, sigma8)
    # <|delta_k|^2> = P(k) n^6 / L^3 for the unnormalised DFT; <|w_k|^2> = n^3
    dk = wk * np.sqrt(pk * n ** 3 / box ** 3)
    dk[0, 0, 0] = 0.0
    inv_k2 = np.zeros_like(k2)
    inv_k2[nz] = 1.0 / k2[nz]
    psi = np.empty((3, n, n, n))
    for d, kd in enumerate((kx, ky, kz)):
        psi[d] = np.fft.irfftn(1j * kd * inv_k2 * dk, s=(n, n, n), axes=(0, 1, 2))
    return psi


# --------------------------------------------------------------- IOS state
def quantise_ios(pos, n_ios, box, order_key=None):
    """Encode positions (3, N) [Mpc/h] into IOS arrays.

    Returns dict(off=(3,N) uint16, count=(n_ios^3,) int32,
    start=(n_ios^3,) int32, perm=(N,) int64 order applied to the input)."""
    s_ios = box / n_ios
    fixed = np.rint(np.asarray(pos, dtype=np.float64) / s_ios * FIX).astype(np.int64)
    fixed %= n_ios * FIX
    cell3 = fixed >> 16
    off = (fixed & (FIX - 1)).astype(np.uint16)
    cell = (cell3[2] * n_ios + cell3[1]) * n_ios + cell3[0]
    perm = np.argsort(cell, kind="stable")
    count = np.bincount(cell, minlength=n_ios ** 3).astype(np.int32)
    start = np.zeros_like(count)
    np.cumsum(count[:-1], out=start[1:])
    return dict(off=np.ascontiguousarray(off[:, perm]), count=count, start=start, perm=perm)


def zeldovich_ios(w):
    """IOS initial state for a workload ``w`` (see inputs.workloads).

    Returns dict(off, count, start, vel (3,N) float32, a (float))."""
    n, box = w.n_p, w.box
    a = w.a_init
    a_disp = a if w.displace_to_a is None else w.displace_to_a
    psi = gaussian_displacement(n, box, w.omega_m, w.h, w.sigma8, w.seed)
    d = growth_d(a_disp, w.omega_m, w.omega_l)
    f = growth_f(a_disp, w.omega_m, w.omega_l)
    e = float(hubble_e(a_disp, w.omega_m, w.omega_l))
    hp = box / n
    grid = (np.arange(n) + 0.5) * hp
    q = np.stack(np.meshgrid(grid, grid, grid, indexing="ij")[::-1])  # [d][z][y][x]
    pos = (q + d * psi).reshape(3, -1)
    mom = (a_disp ** 2 * e * f * d * psi).reshape(3, -1)
    st = quantise_ios(pos, w.n_ios, box)
    vel = np.ascontiguousarray(mom[:, st["perm"]].astype(np.float32))
    return dict(off=st["off"], count=st["count"], start=st["start"], vel=vel, a=a)


def ios_from_positions(pos, vel, n_ios, box):
    """IOS state for explicit positions (3,N) [Mpc/h] and momenta (3,N)."""
    st = quantise_ios(pos, n_ios, box)
    v = np.ascontiguousarray(np.asarray(vel, dtype=np.float32)[:, st["perm"]])
    return dict(off=st["off"], count=st["count"], start=st["start"], vel=v)


def random_ios(n_particles, n_ios, box, seed, clustered=0.0):
    """Uniform (or, with clustered > 0, clumped) random particles in IOS form.

    ``clustered`` in [0, 1) is the fraction of particles drawn inside a few
    Gaussian clumps of width ~1 IOS cell, to give uneven cell counts."""
    rng = np.random.Generator(np.random.Philox(seed))
    n_cl = int(round(clustered * n_particles))
    pos = rng.uniform(0.0, box, size=(3, n_particles - n_cl))
    if n_cl:
        n_clumps = max(1, n_cl // 200)
        centres = rng.uniform(0.0, box, size=(3, n_clumps))
        which = rng.integers(0, n_clumps, size=n_cl)
        clump = centres[:, which] + rng.normal(0.0, box / n_ios, size=(3, n_cl))
        pos = np.concatenate([pos, clump % box], axis=1)
    vel = rng.normal(0.0, 1.0, size=(3, n_particles))
    return ios_from_positions(pos, vel, n_ios, box)
