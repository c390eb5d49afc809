"""PP work counters (cube2_pp_count, cube2_pp_stats, cube2_pp_stats_paths):
off unless switched on, consistent between the two paths, reset by reading,
without effect on the forces, and counting the ordered pairs closer than the
PP range that an FP64 count of the same positions finds (to the pairs whose
FP32 and FP64 squared separations fall on opposite sides of the range)."""
import numpy as np
import pytest

from inputs import C1
from inputs.workloads import Level
from inputs.zeldovich import random_ios, zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import adjoint as oadj  # noqa: E402
from oracle import kdk as okdk  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402

CLUSTER = C1.with_(name="clustered", n_ios=16, levels=(Level(32, 2.0),), b_pp=0.4)


def _case(name):
    if name == "C1":
        return C1, zeldovich_ios(C1)
    return CLUSTER, random_ios(5000, 16, CLUSTER.box, seed=32, clustered=0.8)


def _positions(st, n, box):
    """Continuous positions [Mpc/h] (3, N) of an IOS state, in its particle order."""
    cell = np.repeat(np.arange(n ** 3), st["count"])
    c = np.stack([cell % n, (cell // n) % n, cell // (n * n)])
    return (c + st["off"].astype(np.float64) / 65536.0) * (box / n)


@pytest.mark.parametrize("name", ["C1", "CLUSTER"])
def test_pp_work_counters(name):
    w, st = _case(name)
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    p = cube2.IOSState.from_numpy(st)
    ctx.pp_force(p)                          # counting is off by default
    assert ctx.pp_stats() == (0, 0)
    plain = p.acc.clone()
    ctx.pp_count(True)
    ctx.pp_force(p)
    pairs, cands, lane_pairs, lane_cands = ctx.pp_stats_paths()
    assert torch.equal(p.acc, plain)         # the counted launch computes the same forces
    assert 0 < pairs <= cands and 0 <= lane_pairs <= pairs and 0 <= lane_cands <= cands
    assert ctx.pp_stats_paths() == (0, 0, 0, 0)   # reading resets
    ctx.pp_force(p)
    assert ctx.pp_stats() == (pairs, cands)
    ctx.pp_count(False)
    _, b_cut = okdk.pp_params(w)
    i, _, _, _ = oadj._pair_search(_positions(st, w.n_ios, w.box), w.box, b_cut)
    print(f"{name}: {pairs} pairs ({lane_pairs} on the per-lane walk), {cands} candidates; FP64 count {i.size}")
    assert abs(pairs - i.size) <= max(2, 1e-4 * i.size)
    ctx.close()
