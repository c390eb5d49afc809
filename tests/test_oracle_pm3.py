"""Pins of the oracle's adaptive third PM level (oracle/pm3.py; Sec. 2.1.1 Eq.
PM3, Sec. 2.2.3): local PM3 meshes per subtile with the PP range shrunk to
b_3 = beta_3 H_3.

1. Refinement 1 with beta_3 equal to the finest global level's softening is
   the two-level method, exactly (the PM3 kernel vanishes, the PP range is
   unchanged).
2. A uniform refinement of 2 on the local meshes equals a third *global* level
   of the same spacing computed by the global-mesh oracle (integer CIC on the
   periodic box, one FFT of the whole box): the local box, its buffer and the
   truncated kernel reproduce it to 1e-4 of the rms force.
3. Refinements chosen per subtile from the clustering keep the total force
   within the two-level method's accuracy against periodic direct summation
   (Ewald with the R(r, b_PP) near field), and momentum nearly conserved (the
   PP range changes across subtile faces, so not exactly).
"""
import numpy as np
import pytest

from inputs.workloads import Level, Workload
from inputs.zeldovich import random_ios
from oracle import ewald as E
from oracle import kdk as KD
from oracle import mesh as M
from oracle import pm3 as P3

# 32 Mpc/h, 8^3 IOS cells of 4 Mpc/h, coarse 8^3 and fine 32^3 meshes with the
# paper's softening of 3.5 cells (PP range 3.5 Mpc/h), subtiles of 4^3 IOS cells
W = Workload(name="pm3-8c-8x32mesh", n_p=8, box=32.0, n_ios=8, levels=(Level(8, 3.5), Level(32, 3.5)), b_pp=0.3)
T = 4


@pytest.fixture(scope="module")
def state():
    st = random_ios(1000, W.n_ios, W.box, seed=83, clustered=0.6)
    return st["off"], st["count"], st["start"]


def test_refinement_one_is_the_two_level_method(state):
    off, count, start = state
    f2 = KD.total_force(off, count, start, W)
    fa = P3.adaptive_force(off, count, start, W, T, np.ones(8), 3.5)
    assert np.array_equal(fa, f2) or np.abs(fa - f2).max() <= 1e-13 * np.abs(f2).max()


def test_local_meshes_equal_a_global_third_level(state):
    off, count, start = state
    fa = P3.adaptive_force(off, count, start, W, T, 2 * np.ones(8), 3.5)
    wg = W.with_(levels=(Level(8, 3.5), Level(32, 3.5), Level(64, 3.5)))
    fg = KD.total_force(off, count, start, wg)
    d = np.linalg.norm(fa - fg, axis=0)
    rms = np.sqrt(np.mean(np.linalg.norm(fg, axis=0) ** 2))
    assert d.max() <= 1e-4 * rms, d.max() / rms
    # and the third level is not trivial: it moves the force by more than that
    f2 = KD.total_force(off, count, start, W)
    assert np.linalg.norm(fg - f2, axis=0).max() > 1e-2 * rms


def test_adaptive_refinement_accuracy_and_momentum(state):
    off, count, start = state
    # refine the subtiles holding the densest IOS cells (the paper's rho_max rule)
    cnt = count.reshape(W.n_ios, W.n_ios, W.n_ios)
    ns = W.n_ios // T
    rho_max = cnt.reshape(ns, T, ns, T, ns, T).max(axis=(1, 3, 5))
    refine = np.where(rho_max >= np.median(rho_max), 2, 1)
    assert 0 < (refine == 2).sum() < refine.size
    fa = P3.adaptive_force(off, count, start, W, T, refine, 3.5)
    f2 = KD.total_force(off, count, start, W)
    pos = M.positions(off, count, W.n_ios, W.box)
    fe = E.ewald_force(pos, W.box, W.b_pp)

    def rms_rel(f):
        e = np.linalg.norm(f - fe, axis=0) / np.linalg.norm(fe, axis=0)
        return float(np.sqrt(np.mean(e ** 2)))

    ra, r2 = rms_rel(fa), rms_rel(f2)
    assert ra < 0.06 and ra < 1.25 * r2, (ra, r2)
    assert np.abs(fa.sum(axis=1)).max() < 2e-4 * np.abs(fa).sum()
