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


def _box_by_box(ctxs, ref, sched):
    for c, p, a in zip(ctxs, ref, sched):
        for k in range(len(a) - 1):
            c.kdk_step(p, a[k], a[k + 1])
    torch.cuda.synchronize()


def _assert_equal_states(ctxs, states, ref):
    for c, p, q in zip(ctxs, states, ref):
        c.check()
        for x, y in zip((p.off, p.count, p.start, p.vel, p.acc), (q.off, q.count, q.start, q.vel, q.acc)):
            assert torch.equal(x, y)


@pytest.mark.parametrize("n_streams,ctas", [(1, 1), (3, 4), (16, 16)])
def test_persistent_pp_ensemble_equals_box_by_box(n_streams, ctas):
    # step by step, one persistent PP kernel over every box taking (box, block)
    # items from the cost-ordered device queue: the same per-target sums as the
    # boxes' own PP launches, so the states agree bitwise
    ws, ctxs, states = _boxes(5, 3, (16, 24, 32), seed=7)
    ref = [p.clone() for p in states]
    sched = _schedule(ws, 3)
    ens = cube2.Ensemble(ctxs, states, sched,
                         opts=cube2.ensemble_opts(n_streams=n_streams, persistent_pp=True, pp_ctas_per_sm=ctas))
    for _ in range(2):
        ens.launch()
        ens.check()
        _box_by_box(ctxs, ref, sched)
        _assert_equal_states(ctxs, states, ref)
    ens.close()


def test_persistent_wait_runs_out_when_the_host_withholds_the_queue():
    # the host never publishes the work counts: every persistent kernel's wait
    # ends after its bound and records CUBE2_ERR_TIMEOUT; no GPU fault, and the
    # ensemble works again once publication is back
    ws, ctxs, states = _boxes(2, 2, (16,), seed=11)
    saved = [p.clone() for p in states]
    sched = _schedule(ws, 2)
    ens = cube2.Ensemble(ctxs, states, sched,
                         opts=cube2.ensemble_opts(n_streams=2, persistent_pp=True, pp_ctas_per_sm=2, timeout_ms=200.0))
    ens.publish(False)
    ens.launch()
    with pytest.raises(cube2.Cube2Error) as e:
        ens.check()
    assert e.value.code == cube2.ERR_TIMEOUT
    ens.check()                                  # cleared
    ens.publish(True)
    for p, q in zip(states, saved):
        for x, y in zip((p.off, p.count, p.start, p.vel, p.acc), (q.off, q.count, q.start, q.vel, q.acc)):
            x.copy_(y)
    for c in ctxs:
        c.check()
    ref = [p.clone() for p in states]
    ens.launch()
    ens.check()
    _box_by_box(ctxs, ref, sched)
    _assert_equal_states(ctxs, states, ref)
    ens.close()


def test_autotuner_picks_a_candidate_and_restores_the_states():
    ws, ctxs, states = _boxes(4, 2, (16, 32), seed=13)
    before = [p.clone() for p in states]
    sched = _schedule(ws, 2)
    best, ms = cube2.ensemble_autotune(ctxs, states, sched,
                                       start=cube2.ensemble_opts(n_streams=8, persistent_pp=True, pp_ctas_per_sm=8),
                                       trials=1)
    assert ms > 0 and best.persistent_pp == 1
    assert best.pp_ctas_per_sm in (4, 8, 16) and best.pp_wmax in (0, 8, 16, 24) and best.n_streams in (8, 16, 32)
    torch.cuda.synchronize()
    _assert_equal_states(ctxs, states, before)
    # the chosen options record and run like any other
    ref = [p.clone() for p in states]
    ens = cube2.Ensemble(ctxs, states, sched, opts=best)
    ens.launch()
    ens.check()
    _box_by_box(ctxs, ref, sched)
    _assert_equal_states(ctxs, states, ref)
    ens.close()
