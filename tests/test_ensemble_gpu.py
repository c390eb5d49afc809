"""The ensemble graph (cube2_ensemble_*) against the same steps launched box
by box: every box's state after the recorded steps must be bitwise identical
(the kernels are deterministic and the graph only reorders independent
boxes).  The single-box path itself is checked against the oracle in
test_parity_gpu (case C4_24: a radix-3 ensemble box)."""
import numpy as np
import pytest

from inputs.workloads import c4_ensemble
from inputs.zeldovich import zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2512_12629_gb300 import cube2  # noqa: E402


def _schedule(ws, n_steps):
    # constant steps of the 50-step z = 49 -> 0 spacing from each box's start
    a0 = 1.0 / (1.0 + ws[0].z_init)
    da = (1.0 - a0) / 50
    return np.array([[a0 + k * da for k in range(n_steps + 1)] for _ in ws])


def _boxes(n_boxes, n_steps, sizes, seed):
    ws = c4_ensemble(n_boxes=n_boxes, seed=seed, n_steps=n_steps, sizes=sizes)
    ctxs, states = [], []
    for w in ws:
        st = zeldovich_ios(w)
        ctx = cube2.init_mesh(cube2.make_config(w, n_particles=int(st["count"].sum())))
        ctx.set_green(0)
        p = cube2.IOSState.from_numpy(st)
        ctx.force(p)
        ctxs.append(ctx)
        states.append(p)
    return ws, ctxs, states


@pytest.mark.parametrize("n_streams", [1, 3, 16])
def test_ensemble_graph_equals_box_by_box(n_streams):
    ws, ctxs, states = _boxes(5, 3, (16, 24, 32), seed=7)
    ref = [p.clone() for p in states]
    sched = _schedule(ws, 3)
    ens = cube2.Ensemble(ctxs, states, sched, n_streams=n_streams)
    kernels, psteps = ens.info()
    assert psteps == 3 * sum(w.n_particles for w in ws)
    assert kernels > 0
    ens.launch()
    torch.cuda.synchronize()
    for c, p, a in zip(ctxs, ref, sched):
        for k in range(len(a) - 1):
            c.kdk_step(p, a[k], a[k + 1])
    torch.cuda.synchronize()
    for c, p, q in zip(ctxs, states, ref):
        c.check()
        for x, y in zip((p.off, p.count, p.start, p.vel, p.acc), (q.off, q.count, q.start, q.vel, q.acc)):
            assert torch.equal(x, y)
    # a second launch replays the same three steps from the evolved state
    later = sched
    ens.launch()
    torch.cuda.synchronize()
    for c, p, a in zip(ctxs, ref, later):
        for k in range(len(a) - 1):
            c.kdk_step(p, a[k], a[k + 1])
    torch.cuda.synchronize()
    for c, p, q in zip(ctxs, states, ref):
        c.check()
        assert torch.equal(p.vel, q.vel) and torch.equal(p.off, q.off)
    ens.close()


def test_ensemble_rejects_bad_arguments():
    ws, ctxs, states = _boxes(2, 2, (16,), seed=9)
    sched = _schedule(ws, 2)
    with pytest.raises(cube2.Cube2Error):
        cube2.Ensemble([ctxs[0], ctxs[0]], states, sched)          # one context twice
    bad = sched.copy()
    bad[1, 1] = bad[1, 0]
    with pytest.raises(cube2.Cube2Error):
        cube2.Ensemble(ctxs, states, bad)                           # non-increasing schedule
    ctxs[0].profile(16)
    with pytest.raises(cube2.Cube2Error):
        cube2.Ensemble(ctxs, states, sched)                         # profiling on
    ctxs[0].profile(0)
    cube2.Ensemble(ctxs, states, sched).close()
