"""Pins of the FP64 adjoint oracle (oracle/adjoint.py): the vector-Jacobian
products against central finite differences of the forward force (FP64,
continuous positions), the continuous forward against the IOS forward at IOS
positions, and dR/dr against differences of R."""
import numpy as np
import pytest

from inputs import C2_SMALL
from inputs.workloads import Level
from inputs.zeldovich import random_ios
from oracle import adjoint as A
from oracle import kernels as K
from oracle import mesh as M


def test_reference_force_derivative_matches_differences():
    for b in (0.3, 1.0, 2.5):
        r = np.linspace(0.01, 1.6 * b, 997)
        r = r[(np.abs(r - 0.5 * b) > 1e-3) & (np.abs(r - b) > 1e-3)]
        h = 1e-6 * b
        fd = (K.reference_force(r + h, b) - K.reference_force(r - h, b)) / (2 * h)
        an = K.reference_force_derivative(r, b)
        assert np.allclose(an, fd, rtol=1e-6, atol=1e-6 * np.abs(an).max())


def _directional(fn, x, v, e, h):
    return ((v * fn(x + h * e)).sum() - (v * fn(x - h * e)).sum()) / (2 * h)


@pytest.mark.parametrize("n,bs,bt", [(16, 2.0, None), (16, 2.0, 3.5), (12, 3.5, None)])
def test_pm_vjp_matches_finite_differences(n, bs, bt):
    rng = np.random.default_rng(n + int(bs * 10))
    box, npart = 24.0, 300
    x = rng.uniform(0, box, (3, npart))
    v = rng.normal(size=(3, npart))
    g = K.green(n, bs, bt)
    w = A.pm_vjp_level(x, v, box, n, npart, g)
    for k in range(3):
        e = rng.normal(size=(3, npart))
        fd = _directional(lambda y: A.pm_force_level(y, box, n, npart, g), x, v, e, 1e-6)
        assert abs((w * e).sum() - fd) <= 1e-6 * (np.abs(w).sum() + abs(fd))
    # single components: one particle, one axis
    for i, d in ((0, 0), (7, 1), (123, 2)):
        e = np.zeros((3, npart))
        e[d, i] = 1.0
        fd = _directional(lambda y: A.pm_force_level(y, box, n, npart, g), x, v, e, 1e-6)
        assert abs(w[d, i] - fd) <= 1e-6 * np.abs(w).max()


def test_pp_vjp_matches_finite_differences():
    rng = np.random.default_rng(5)
    box, npart, b_pp, b_cut = 8.0, 400, 0.15, 1.0
    x = rng.uniform(0, box, (3, npart))
    x[:, 1] = x[:, 0] + [0.05, 0.02, -0.03]          # a pair closer than b_pp
    v = rng.normal(size=(3, npart))
    w = A.pp_vjp(x, v, box, npart, b_pp, b_cut)
    for k in range(3):
        e = rng.normal(size=(3, npart))
        fd = _directional(lambda y: A.pp_force(y, box, npart, b_pp, b_cut), x, v, e, 1e-7)
        assert abs((w * e).sum() - fd) <= 1e-6 * (np.abs(w).sum() + abs(fd))
    for i, d in ((0, 0), (1, 2), (77, 1)):
        e = np.zeros((3, npart))
        e[d, i] = 1.0
        fd = _directional(lambda y: A.pp_force(y, box, npart, b_pp, b_cut), x, v, e, 1e-7)
        assert abs(w[d, i] - fd) <= 1e-6 * np.abs(w).max()
    # momentum: the PP force is translation invariant, so the VJP sums to zero
    assert np.abs(w.sum(axis=1)).max() <= 1e-10 * np.abs(w).sum()


def test_continuous_forward_equals_ios_forward_at_ios_positions():
    w = C2_SMALL.with_(n_p=16, box=16.0, n_ios=16, levels=(Level(8, 3.5), Level(32, 2.0)))
    st = random_ios(16 ** 3, 16, w.box, seed=3, clustered=0.3)
    x = M.positions(st["off"], st["count"], w.n_ios, w.box)
    greens = M.green_tables(w)
    for (n, h, _bs, _bt), g in zip(M.level_params(w), greens):
        ref, _ = M.pm_force_level(st["off"], st["count"], w.n_ios, n, h, g)
        got = A.pm_force_level(x, w.box, n, x.shape[1], g)
        # the coarse level floors one bit of the position (2^-17 cell) in the IOS forward
        tol = 1e-12 if n >= w.n_ios else 1e-4
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_total_force_vjp_two_levels():
    w = C2_SMALL.with_(n_p=8, box=16.0, n_ios=8, levels=(Level(8, 3.5), Level(16, 2.0)), b_pp=0.3)
    rng = np.random.default_rng(11)
    npart = 8 ** 3
    x = rng.uniform(0, w.box, (3, npart))
    v = rng.normal(size=(3, npart))
    greens = M.green_tables(w)
    wv = A.force_vjp(x, v, w, greens)
    e = rng.normal(size=(3, npart))
    fd = _directional(lambda y: A.force(y, w, greens), x, v, e, 1e-6)
    assert abs((wv * e).sum() - fd) <= 1e-6 * (np.abs(wv).sum() + abs(fd))


def test_cell_list_pp_vjp_equals_all_pairs():
    st = random_ios(3000, 8, 8.0, seed=21, clustered=0.6)
    x = M.positions(st["off"], st["count"], 8, 8.0)
    v = np.random.default_rng(2).normal(size=x.shape)
    ref = A.pp_vjp(x, v, 8.0, x.shape[1], 0.12, 1.0)
    got = A.pp_vjp_cells(st["off"], st["count"], st["start"], 8, 8.0, 0.12, 1.0, v)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_loss_gradient_matches_finite_differences():
    """Central differences of the loss through 3 KDK steps, eps = 1e-4 cell in
    displacement (and the matching step in velocity), on 64 random components
    (32 positions, 32 velocities)."""
    from inputs import C1
    wl = C1.with_(n_p=6, box=12.0, n_ios=6, levels=(Level(12, 2.0),), b_pp=0.2)
    rng = np.random.default_rng(17)
    npart = 6 ** 3
    x0 = rng.uniform(0, wl.box, (3, npart))
    p0 = rng.normal(0, 2.0, (3, npart))
    greens = M.green_tables(wl)
    a = [0.1, 0.12, 0.14, 0.16]
    target = rng.normal(0, 0.3, (12, 12, 12))
    loss, gx, gp = A.loss_gradient(x0, p0, wl, greens, a, target)

    def lossf(x, p):
        return A.density_loss(A.kdk_trajectory(x, p, wl, greens, a)[-1][0], wl, target)

    assert abs(loss - lossf(x0, p0)) <= 1e-12 * loss
    eps = 1e-4 * wl.box / 12
    for k in range(32):
        i, d = int(rng.integers(npart)), int(rng.integers(3))
        e = np.zeros((3, npart))
        e[d, i] = eps
        fd = (lossf(x0 + e, p0) - lossf(x0 - e, p0)) / (2 * eps)
        assert abs(gx[d, i] - fd) <= 1e-6 * np.abs(gx).max(), (i, d, gx[d, i], fd)
        fdp = (lossf(x0, p0 + e) - lossf(x0, p0 - e)) / (2 * eps)
        assert abs(gp[d, i] - fdp) <= 1e-6 * np.abs(gp).max(), (i, d, gp[d, i], fdp)


def test_cell_list_pairs_equal_all_pairs():
    # the cell list the continuous-position PP uses beyond 4096 particles
    # finds exactly the pairs of the all-pairs search
    rng = np.random.default_rng(12)
    box, b_cut = 20.0, 1.3
    x = np.concatenate([rng.uniform(0, box, (3, 1500)), (7.0 + rng.normal(0, 0.8, (3, 500))) % box], axis=1)
    i0, j0, d0, r0 = A._pairs(x, box, b_cut)
    i1, j1, d1, r1 = A._pairs_cells(x, box, b_cut)
    k0, k1 = np.lexsort((j0, i0)), np.lexsort((j1, i1))
    assert np.array_equal(i0[k0], i1[k1]) and np.array_equal(j0[k0], j1[k1])
    assert np.array_equal(d0[:, k0], d1[:, k1]) and np.array_equal(r0[k0], r1[k1])


def test_ios_trajectory_equals_the_fixed_point_kdk_step():
    # the adjoint oracle's IOS mode (drifts rounded to the 2^-16 grid) visits
    # the same positions and momenta as the IOS KDK step of oracle/kdk.py
    from inputs import C1
    from inputs.zeldovich import zeldovich_ios
    from oracle import kdk as KD
    w = C1.with_(n_p=16, box=32.0, n_ios=16, levels=(Level(32, 2.0),), b_pp=0.2)
    st = zeldovich_ios(w)
    greens = M.green_tables(w)
    a0 = 1.0 / (1.0 + w.z_init)
    a = [a0 + k * (1.0 - a0) / 50 for k in range(4)]
    x0 = M.positions(st["off"], st["count"], w.n_ios, w.box)
    v0 = np.asarray(st["vel"], dtype=np.float32).astype(np.float64)
    xf, pf = A.kdk_trajectory(x0, v0, w, greens, a, ios=True)[-1]
    state = dict(off=st["off"], count=st["count"], start=st["start"], vel=v0, acc=None)
    for k in range(3):
        state = KD.kdk_step(state, w, a[k], a[k + 1], greens)
    xk = M.positions(state["off"], state["count"], w.n_ios, w.box)
    i1, i2 = np.lexsort(xf[::-1]), np.lexsort(xk[::-1])
    assert np.array_equal(xf[:, i1], xk[:, i2])
    assert np.allclose(pf[:, i1], state["vel"][:, i2], rtol=1e-10, atol=1e-12 * np.abs(pf).max())
