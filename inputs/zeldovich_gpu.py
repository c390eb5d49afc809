"""Seeded synthetic inputs on the GPU: the Zel'dovich recipe of
``inputs.zeldovich`` for boxes too large for host arrays (1024^3 particles).

This module only *generates inputs*; it holds none of the force method's
arithmetic.  The recipe is the one of ``inputs.zeldovich`` (BBKS spectrum with
sigma_8 normalisation, linear growth D, displacement psi(k) = i k delta(k)/k^2,
positions x = q + D psi on the n_p^3 lattice, quantisation to IOS with 2^16
sub-cells per cell, particles sorted stably by cell id with the lattice index
as tie-break).  The Gaussian field comes from ``torch.randn`` with a seeded
``torch.Generator`` on the device, whose stream is not numpy's Philox: a box
drawn here is a different realisation from the host generator's, and both the
CUDA path and the oracle's sampled checks read the IOS arrays returned here.
The transforms run through torch (cuFFT) in FP32; the displacement is rounded
to the IOS grid in FP64.  With ``momenta=True`` the canonical momenta
p = a^2 E f D psi (the host recipe's, at the displacement's scale factor) are
returned as well, in FP32 and in the IOS order.
"""
from __future__ import annotations

import math

import torch

from .zeldovich import FIX, growth_d, growth_f, hubble_e, spectrum_amplitude


def _fftfreq_k(n, kf, device):
    f = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float32)
    return f * kf


def zeldovich_ios_torch(w, device="cuda", momenta=False):
    """IOS arrays for workload ``w`` (n_ios must equal n_p): dict(off=(3,N)
    int16 storage of the uint16 offsets, count, start=(n_ios^3,) int32, and
    with ``momenta`` vel=(3,N) float32), all on ``device``."""
    n, box = w.n_p, w.box
    if w.n_ios != n:
        raise ValueError("the device generator places one particle per IOS cell before displacement")
    a_disp = w.a_init if w.displace_to_a is None else w.displace_to_a
    amp = spectrum_amplitude(w.omega_m, w.h, w.sigma8)
    d_growth = growth_d(a_disp, w.omega_m, w.omega_l)
    gen = torch.Generator(device=device).manual_seed(int(w.seed))
    white = torch.randn((n, n, n), generator=gen, device=device, dtype=torch.float32)
    dk = torch.fft.rfftn(white)
    del white
    kf = 2.0 * math.pi / box
    kz = _fftfreq_k(n, kf, device)[:, None, None]
    ky = _fftfreq_k(n, kf, device)[None, :, None]
    kx = (torch.fft.rfftfreq(n, d=1.0 / n, device=device, dtype=torch.float32) * kf)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k = torch.sqrt(k2)
    # P(k) = A k T_BBKS(k)^2, Gamma = Omega_m h; <|delta_k|^2> = P n^6 / L^3
    q = k / (w.omega_m * w.h)
    qs = torch.where(q > 0, q, torch.ones_like(q))
    t = torch.log1p(2.34 * qs) / (2.34 * qs) * (1.0 + 3.89 * qs + (16.1 * qs) ** 2 + (5.46 * qs) ** 3
                                                 + (6.71 * qs) ** 4) ** -0.25
    pk = amp * k * t * t
    del q, qs, t, k
    dk *= torch.sqrt(pk * (n ** 3 / box ** 3))
    del pk
    dk[0, 0, 0] = 0
    inv_k2 = torch.where(k2 > 0, 1.0 / torch.where(k2 > 0, k2, torch.ones_like(k2)), torch.zeros_like(k2))
    del k2
    s_ios = box / w.n_ios
    cell = None
    offs, moms = [], []
    mom_fac = a_disp ** 2 * float(hubble_e(a_disp, w.omega_m, w.omega_l)) * growth_f(a_disp, w.omega_m, w.omega_l) \
        * d_growth
    idx = torch.arange(n, device=device, dtype=torch.int64)
    for d, kd in enumerate((kx, ky, kz)):
        psi = torch.fft.irfftn(1j * kd * inv_k2 * dk, s=(n, n, n))
        # X = (i_d + 1/2 + D psi / s) 2^16 on the lattice point of axis d, wrapped
        disp = torch.round(psi.double() * (d_growth / s_ios * FIX)).to(torch.int64)
        if momenta:
            moms.append((psi * mom_fac).view(-1))
        del psi
        lattice = (idx.view(1, 1, n) if d == 0 else (idx.view(1, n, 1) if d == 1 else idx.view(n, 1, 1)))
        fixed = torch.remainder(lattice * FIX + FIX // 2 + disp, n * FIX).view(-1)
        del disp
        c = fixed >> 16
        offs.append((fixed & (FIX - 1)).to(torch.int32).to(torch.int16))
        cell = c if cell is None else cell + c * (n ** d)
        del fixed, c
    del dk, inv_k2
    order = torch.sort(cell, stable=True).indices
    cell_sorted = cell[order]
    off = torch.stack([o[order] for o in offs])
    vel = torch.stack([m[order] for m in moms]) if momenta else None
    del offs, moms, order
    count = torch.bincount(cell_sorted, minlength=w.n_ios ** 3).to(torch.int32)
    del cell, cell_sorted
    start = (torch.cumsum(count, 0, dtype=torch.int64) - count).to(torch.int32)
    out = dict(off=off, count=count, start=start)
    if momenta:
        out["vel"] = vel
    return out
