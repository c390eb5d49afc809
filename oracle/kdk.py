"""FP64 oracle: total force and the kick-drift-kick step over IOS particles.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py; never by the product path.

Time integration (Sec. 2.2.3 kick/drift, Sec. 2.3 leap-frog, Sec. 3.2
constant Delta a), in H_0 = 1 units with lengths in Mpc/h and canonical
momentum p = a^2 dx/dt:

    dp/da = (3/2) Omega_m F / (a^2 E(a)),   dx/da = p / (a^3 E(a)),
    E(a) = sqrt(Omega_m a^-3 + Omega_L),    F = -grad u, lap u = delta.

KDK: kick by K(a0, a_h), drift by Dr(a0, a1), recompute F, kick by
K(a_h, a1), with a_h = (a0 + a1)/2, K(a,b) = int_a^b da/(a^2 E) and
Dr(a,b) = int_a^b da/(a^3 E) by Gauss-Legendre quadrature.

Drift in IOS fixed point: X <- (X + rint(p Dr 2^16 / s_ios)) mod (n_ios 2^16)
with round-half-even, then a stable re-sort by new cell id (ties keep the
previous particle order), which rebuilds counts and starts (Sec. 2.3).
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import FIX, fixed_coords, green_tables, level_params, pm_force
from .pp import pp_force


def hubble_e(a, om, ol):
    return np.sqrt(om * a ** -3.0 + ol)


def _gauss_legendre(fn, a0, a1, npts=48):
    x, wts = np.polynomial.legendre.leggauss(npts)
    mid, half = 0.5 * (a1 + a0), 0.5 * (a1 - a0)
    return float(half * np.sum(wts * fn(mid + half * x)))


def kick_integral(a0, a1, om, ol):
    """K(a0, a1) = int da / (a^2 E(a))."""
    return _gauss_legendre(lambda a: 1.0 / (a * a * hubble_e(a, om, ol)), a0, a1)


def drift_integral(a0, a1, om, ol):
    """Dr(a0, a1) = int da / (a^3 E(a))."""
    return _gauss_legendre(lambda a: 1.0 / (a ** 3 * hubble_e(a, om, ol)), a0, a1)


def pp_params(w):
    """(b_PP, b_cut) in Mpc/h: PP range = softening of the finest PM level."""
    n_fine, h_fine, b_soft, _ = level_params(w)[-1]
    return w.b_pp, b_soft * h_fine


def total_force(off, count, start, w, greens=None):
    """F = sum over PM levels + PP, (3, N) FP64."""
    b_pp, b_cut = pp_params(w)
    f = pm_force(off, count, w, greens)
    return f + pp_force(off, count, start, w.n_ios, w.box, b_pp, b_cut)


def drift_rebin(off, count, vel, dr, n_ios, box, acc=None):
    """Fixed-point drift then stable re-bin; returns (off, count, start, vel[, acc])."""
    s_ios = box / n_ios
    X = fixed_coords(off, count, n_ios)
    X = X + np.rint(vel * (dr * FIX / s_ios)).astype(np.int64)
    X %= n_ios * FIX
    c3 = X >> 16
    cell = (c3[2] * n_ios + c3[1]) * n_ios + c3[0]
    order = np.argsort(cell, kind="stable")
    new_off = (X & (FIX - 1)).astype(np.uint16)[:, order]
    new_count = np.bincount(cell, minlength=n_ios ** 3).astype(np.int32)
    new_start = np.zeros_like(new_count)
    np.cumsum(new_count[:-1], out=new_start[1:])
    out = [np.ascontiguousarray(new_off), new_count, new_start, vel[:, order]]
    if acc is not None:
        out.append(acc[:, order])
    return tuple(out)


def kdk_step(state, w, a0, a1, greens=None):
    """One KDK step.  state: dict(off, count, start, vel (FP64), acc = F(x0) or None).

    Returns the new state with acc = F at the new positions."""
    greens = green_tables(w) if greens is None else greens
    om, ol = w.omega_m, w.omega_l
    ah = 0.5 * (a0 + a1)
    off, count, start = state["off"], state["count"], state["start"]
    vel = np.asarray(state["vel"], dtype=np.float64)
    acc = state.get("acc")
    if acc is None:
        acc = total_force(off, count, start, w, greens)
    vel = vel + 1.5 * om * kick_integral(a0, ah, om, ol) * acc
    off, count, start, vel = drift_rebin(off, count, vel, drift_integral(a0, a1, om, ol),
                                         w.n_ios, w.box)
    acc = total_force(off, count, start, w, greens)
    vel = vel + 1.5 * om * kick_integral(ah, a1, om, ol) * acc
    return dict(off=off, count=count, start=start, vel=vel, acc=acc)


# ------------------------------------------------- compressed velocities
# Sec. 2.3 stores velocities compactly next to the IOS positions (the paper
# points to its predecessor for the formula, which is not in the text).  The
# reading used here, the large workload's: each velocity component as an IEEE
# binary16 code times an FP32 scale per IOS cell, the largest |v_d| of the
# cell's particles, so that every code lies in [-1, 1].
def velocity_scales(vel, count):
    """FP32 per-cell scale: max over the cell's particles and components of |v_d|."""
    v = np.abs(np.asarray(vel, dtype=np.float32)).max(axis=0)
    cell = np.repeat(np.arange(count.size, dtype=np.int64), count.astype(np.int64))
    scale = np.zeros(count.size, dtype=np.float32)
    np.maximum.at(scale, cell, v)
    return scale


def encode_velocities(vel, count):
    """(codes float16 (3, N), scale float32 (n_cells,)): code = RN_half(RN32(v / scale)),
    0 in cells whose scale is 0."""
    v = np.asarray(vel, dtype=np.float32)
    scale = velocity_scales(v, count)
    cell = np.repeat(np.arange(count.size, dtype=np.int64), count.astype(np.int64))
    s = scale[cell]
    safe = np.where(s > 0, s, np.float32(1.0))
    codes = np.where(s > 0, v / safe, np.float32(0.0)).astype(np.float16)
    return codes, scale


def decode_velocities(codes, scale, count):
    """FP32 velocities RN32(float(code) * scale) of each particle's cell."""
    cell = np.repeat(np.arange(count.size, dtype=np.int64), count.astype(np.int64))
    return np.asarray(codes, dtype=np.float16).astype(np.float32) * scale[cell]
