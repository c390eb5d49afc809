"""Full-size parity: the 256^3 two-level workload in the configuration bench.py
times, checked on sampled outputs the oracle computes one by one (deposit
cells bit-exact, Green's-table modes, PP forces of sampled particles) and on
properties that hold at any size (momentum conservation, determinism, particle
conservation through a KDK step)."""
import numpy as np
import pytest

from inputs import C2
from inputs.zeldovich import random_ios, zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import kdk as okdk  # noqa: E402
from oracle import kernels as okern  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from oracle import pp as opp  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402

W = C2


@pytest.fixture(scope="module")
def setup():
    st = zeldovich_ios(W)
    ctx = cube2.init_mesh(cube2.make_config(W))
    for l in range(len(W.levels)):
        ctx.set_green(l)
    return st, ctx


def test_green_tables_at_sampled_modes(setup):
    st, ctx = setup
    rng = np.random.default_rng(11)
    for l, (n, _h, bs, bt) in enumerate(omesh.level_params(W)):
        g = ctx.get_green(l).cpu().numpy().astype(np.float64) * float(n) ** 3
        modes = np.stack([rng.integers(0, n // 2 + 1, 400), rng.integers(0, n, 400), rng.integers(0, n, 400)], 1)
        modes[:5] = [[n // 2, n // 2, n // 2], [0, 0, 1], [1, 0, 0], [n // 2, 0, 0], [n // 4, n - 1, 3]]
        ref = okern.green_at(n, modes, bs, bt)
        got = g[modes[:, 2], modes[:, 1], modes[:, 0]]
        assert np.all(np.abs(got - ref) <= 2.0 ** -23 * np.abs(ref) + 1e-7 * np.abs(ref).max())


def test_deposit_bit_exact_at_sampled_cells(setup):
    st, ctx = setup
    p = cube2.IOSState.from_numpy(st)
    rng = np.random.default_rng(12)
    for l, lev in enumerate(W.levels):
        n = lev.n_mesh
        acc = ctx.deposit_u64(l, p).cpu().numpy().view(np.uint64).ravel()
        cells = rng.integers(0, n ** 3, 150 if n >= 512 else 60)
        ref = omesh.deposit_u64_at(st["off"], st["count"], st["start"], W.n_ios, n, cells)
        assert np.array_equal(acc[cells], ref)
        # exact mass: every particle contributes 2^48 (summed in two 32-bit halves
        # so that no partial sum wraps)
        total = (int((acc >> np.uint64(32)).sum()) << 32) + int((acc & np.uint64(0xFFFFFFFF)).sum())
        assert total == W.n_particles << 48
    ctx.check()


def test_pp_and_total_force_full_size(setup):
    st, ctx = setup
    # a clumped full-size particle set (uneven cells) with the workload's geometry
    cl = random_ios(W.n_particles, W.n_ios, W.box, seed=13, clustered=0.3)
    p = cube2.IOSState.from_numpy(cl)
    b_pp, b_cut = okdk.pp_params(W)
    ctx.pp_force(p, accumulate=False)
    ctx.check()
    f = p.acc.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(14)
    dense = np.argsort(-cl["count"])[:3]
    targets = np.concatenate([rng.integers(0, W.n_particles, 600),
                              [int(cl["start"][c]) for c in dense]])
    ref = opp.pp_force_at(cl["off"], cl["count"], cl["start"], W.n_ios, W.box, b_pp, b_cut, targets)
    got = f[:, targets]
    pair_scale = W.box ** 3 / W.n_particles / (4 * np.pi * b_cut ** 2)
    err = np.linalg.norm(got - ref, axis=0)
    assert np.all(err <= 1e-5 * (pair_scale + np.linalg.norm(ref, axis=0)))
    # PP and total force conserve momentum (pairwise antisymmetry, symmetric CIC + D)
    assert np.abs(f.sum(axis=1)).max() < 1e-5 * np.abs(f).sum()
    ctx.force(p)
    ctx.check()
    ft = p.acc.cpu().numpy().astype(np.float64)
    assert np.isfinite(ft).all()
    assert np.abs(ft.sum(axis=1)).max() < 1e-4 * np.abs(ft).sum()


def test_kdk_step_full_size_is_deterministic_and_conserves_particles(setup):
    st, ctx = setup
    a = W.scale_factors()
    outs = []
    for _ in range(2):
        p = cube2.IOSState.from_numpy(st)
        ctx.force(p)
        ctx.kdk_step(p, a[0], a[1])
        ctx.check()
        outs.append(p)
    assert int(outs[0].count.sum().item()) == W.n_particles
    for x, y in zip((outs[0].off, outs[0].count, outs[0].vel, outs[0].acc),
                    (outs[1].off, outs[1].count, outs[1].vel, outs[1].acc)):
        assert torch.equal(x, y)
    start = torch.cumsum(outs[0].count, 0) - outs[0].count
    assert torch.equal(start.to(torch.int32), outs[0].start)
