"""cube2_force_vjp (CUDA path through the C ABI) against the FP64 adjoint
oracle, element by element, at the stored IOS positions.

Tolerance: the force's own bar.  With r_i = |w_gpu - w_or| / max(|w_or|,
1e-3 rms|w_or|): median <= 1e-5 and 99.9th percentile <= 1e-3 (the product
is FP32 arithmetic of the same depth as the force: one FFT solve per term,
CIC sums, pair sums; its cotangent deposit uses FP32 atomics in arbitrary
order, which moves only the last bits)."""
import numpy as np
import pytest

from inputs import C1, C2_SMALL
from inputs.workloads import Level
from inputs.zeldovich import random_ios, zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import adjoint as A  # noqa: E402
from oracle import kdk as okdk  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402

CLUSTER = C1.with_(name="clustered", n_ios=16, levels=(Level(32, 2.0),), b_pp=0.4)


def _case(name):
    if name == "C1":
        return C1, zeldovich_ios(C1)
    if name == "C2_SMALL":
        return C2_SMALL, zeldovich_ios(C2_SMALL)
    if name == "CLUSTER":
        return CLUSTER, random_ios(5000, 16, CLUSTER.box, seed=32, clustered=0.8)
    raise KeyError(name)


def _oracle_vjp(w, st, v):
    x = omesh.positions(st["off"], st["count"], w.n_ios, w.box)
    n_part = x.shape[1]
    out = np.zeros_like(x)
    for (n, _h, _bs, _bt), g in zip(omesh.level_params(w), omesh.green_tables(w)):
        out += A.pm_vjp_level(x, v, w.box, n, n_part, g)
    b_pp, b_cut = okdk.pp_params(w)
    return out + A.pp_vjp_cells(st["off"], st["count"], st["start"], w.n_ios, w.box, b_pp, b_cut, v)


@pytest.mark.parametrize("name", ["C1", "C2_SMALL", "CLUSTER"])
def test_force_vjp_matches_oracle(name):
    w, st = _case(name)
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    for l in range(len(w.levels)):
        ctx.set_green(l)
    ctx.adjoint_init()
    p = cube2.IOSState.from_numpy(st)
    v = np.random.default_rng(3).normal(size=(3, n_part))
    got = ctx.force_vjp(p, torch.from_numpy(v.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    ctx.check()
    ref = _oracle_vjp(w, st, v)
    err = np.linalg.norm(got - ref, axis=0)
    mag = np.linalg.norm(ref, axis=0)
    rel = err / np.maximum(mag, 1e-3 * np.sqrt(np.mean(mag ** 2)))
    med, p999 = np.median(rel), np.quantile(rel, 0.999)
    print(f"{name}: median {med:.2e} p99.9 {p999:.2e} max {rel.max():.2e}")
    assert med <= 1e-5 and p999 <= 1e-3, (med, p999)


def test_force_vjp_needs_init_and_is_linear():
    w, st = _case("C1")
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    ctx.set_green(0)
    p = cube2.IOSState.from_numpy(st)
    v = torch.randn(3, n_part, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    with pytest.raises(cube2.Cube2Error):
        ctx.force_vjp(p, v)
    ctx.adjoint_init()
    w1 = ctx.force_vjp(p, v)
    w2 = ctx.force_vjp(p, 2.0 * v)
    w3 = ctx.force_vjp(p, torch.zeros_like(v))
    ctx.check()
    assert torch.allclose(w2, 2.0 * w1, rtol=1e-4, atol=1e-4 * w1.abs().max().item())
    assert w3.abs().max().item() == 0.0


def test_loss_gradient_through_kdk_steps_matches_oracle():
    """The whole chain (checkpointed KDK steps, density loss, reverse steps
    through the re-bin maps) against the FP64 oracle's continuous
    trajectory from the same initial state.  The GPU trajectory rounds each
    drift to the IOS grid (2^-17 cell at most per step), so the two differ by
    that much; the gradients agree statistically."""
    from oracle import mesh as M
    w = C1.with_(n_p=16, box=32.0, n_ios=16, levels=(Level(32, 2.0),), b_pp=0.2)
    st = zeldovich_ios(w)
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    ctx.set_green(0)
    ctx.adjoint_init()
    p0 = cube2.IOSState.from_numpy(st)
    ctx.force(p0)
    a0 = 1.0 / (1.0 + w.z_init)
    a = [a0 + k * (1.0 - a0) / 50 for k in range(4)]
    rng = np.random.default_rng(8)
    target = rng.normal(0.0, 0.5, (32, 32, 32))
    loss, gx, gp = cube2.loss_gradient(ctx, p0, torch.from_numpy(target.astype(np.float32)).cuda(), a)
    ctx.check()
    x0 = M.positions(st["off"], st["count"], w.n_ios, w.box)
    v0 = np.asarray(st["vel"], dtype=np.float32).astype(np.float64)
    lo, ox, op = A.loss_gradient(x0, v0, w, M.green_tables(w), a, target, ios=True)
    assert abs(loss - lo) <= 1e-4 * lo
    rng = np.random.default_rng(64)
    for got, ref in ((gx.cpu().numpy().astype(np.float64), ox), (gp.cpu().numpy().astype(np.float64), op)):
        err = np.linalg.norm(got - ref, axis=0)
        mag = np.linalg.norm(ref, axis=0)
        rel = err / np.maximum(mag, 1e-3 * np.sqrt(np.mean(mag ** 2)))
        med, p99 = np.median(rel), np.quantile(rel, 0.99)
        # 32 random components of each gradient at the 1e-3 bar (own size, floor 1e-3 of the rms)
        comp = rng.choice(ref.size, 32, replace=False)
        crel = (np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3 * np.sqrt(np.mean(ref ** 2)))).ravel()[comp]
        print(f"gradient: median {med:.2e} p99 {p99:.2e}; 32 random components max {crel.max():.2e}")
        assert med <= 5e-4 and p99 <= 5e-3, (med, p99)
        assert crel.max() <= 1e-3, crel.max()


def test_fused_reverse_sweep_equals_step_by_step():
    """cube2_kdk_adjoint (one force product per step) against
    cube2_kdk_adjoint_step applied step by step (two per step)."""
    w = C1.with_(n_p=16, box=32.0, n_ios=16, levels=(Level(32, 2.0),), b_pp=0.2)
    st = zeldovich_ios(w)
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    ctx.set_green(0)
    ctx.adjoint_init()
    p0 = cube2.IOSState.from_numpy(st)
    ctx.force(p0)
    a0 = 1.0 / (1.0 + w.z_init)
    a = [a0 + k * (1.0 - a0) / 50 for k in range(4)]
    states, perms = [p0], []
    p = p0.clone()
    for k in range(3):
        ctx.kdk_step(p, a[k], a[k + 1])
        perms.append(ctx.kdk_permutation())
        states.append(p.clone())
    g = torch.Generator("cuda").manual_seed(5)
    xb0 = torch.randn(3, n_part, device="cuda", generator=g)
    pb0 = torch.randn(3, n_part, device="cuda", generator=g)
    xb1, pb1 = xb0.clone(), pb0.clone()
    ctx.kdk_adjoint(states, perms, a, xb1, pb1)
    xb2, pb2 = xb0.clone(), pb0.clone()
    for k in range(2, -1, -1):
        ctx.kdk_adjoint_step(states[k], states[k + 1], perms[k], xb2, pb2, a[k], a[k + 1])
    ctx.check()
    for u, v in ((xb1, xb2), (pb1, pb2)):
        assert torch.allclose(u, v, rtol=1e-4, atol=1e-4 * v.abs().max().item())


def test_gradient_on_the_differentiation_schedule_matches_oracle():
    """The differentiation workload's layout and schedule (1 Mpc/h per
    particle, a mesh of 2 cells per particle with a 2-cell softening, 10
    constant-Delta-a KDK steps z = 9 -> 0, density MSE loss against the final
    density of the seed-4 realisation) at 32^3 particles: the GPU gradient
    with respect to the initial positions and momenta against the FP64
    oracle's reverse sweep along its own IOS trajectory (drifts rounded to the
    2^-16 grid, as on the GPU; the oracle's gradient equals central
    differences of its loss, test_oracle_adjoint).  Ten steps into the
    nonlinear regime the FP32 and FP64 trajectories part (their losses differ
    by ~1e-3): the agreement is statistical, the direction of each gradient
    and its relative L2 difference; the component bar of 1e-3 holds where the
    trajectories stay together (the 3-step test)."""
    from inputs.workloads import WORKLOADS
    from oracle import mesh as M
    c3 = WORKLOADS["pm1-128c-256mesh"]
    w = c3.with_(n_p=32, box=32.0, n_ios=32, levels=(Level(64, 2.0),))
    st = zeldovich_ios(w)
    n_part = int(st["count"].sum())
    a = w.scale_factors()
    assert len(a) == 11 and abs(1.0 / a[0] - 10.0) < 1e-12 and a[-1] == 1.0
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    ctx.set_green(0)
    ctx.adjoint_init()
    # target: the final overdensity of the seed-4 realisation (oracle trajectory)
    tgt = zeldovich_ios(w.with_(seed=4))
    xt = M.positions(tgt["off"], tgt["count"], w.n_ios, w.box)
    vt = np.asarray(tgt["vel"], dtype=np.float32).astype(np.float64)
    greens = M.green_tables(w)
    xf = A.kdk_trajectory(xt, vt, w, greens, a, ios=True)[-1][0]
    n = 64
    h = w.box / n
    target = A._deposit(A.cic_corners(xf / h, n), np.ones(xf.shape[1]), n) * (n ** 3 / xf.shape[1]) - 1.0
    p0 = cube2.IOSState.from_numpy(st)
    ctx.force(p0)
    loss, gx, gp = cube2.loss_gradient(ctx, p0, torch.from_numpy(target.astype(np.float32)).cuda(), a)
    ctx.check()
    x0 = M.positions(st["off"], st["count"], w.n_ios, w.box)
    v0 = np.asarray(st["vel"], dtype=np.float32).astype(np.float64)
    lo, ox, op = A.loss_gradient(x0, v0, w, greens, a, target, ios=True)
    print(f"differentiation schedule at 32^3: loss GPU {loss:.6e} oracle {lo:.6e}")
    assert abs(loss - lo) <= 3e-3 * lo
    for name, got, ref in (("dL/dx0", gx.cpu().numpy().astype(np.float64), ox),
                           ("dL/dp0", gp.cpu().numpy().astype(np.float64), op)):
        cos = float((got * ref).sum() / np.sqrt((got ** 2).sum() * (ref ** 2).sum()))
        l2 = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        mag = np.linalg.norm(ref, axis=0)
        rel = np.linalg.norm(got - ref, axis=0) / np.maximum(mag, 1e-3 * np.sqrt(np.mean(mag ** 2)))
        print(f"{name}: cosine {cos:.6f}, relative L2 difference {l2:.3e}, per particle median {np.median(rel):.2e}, "
              f"p99 {np.quantile(rel, 0.99):.2e}")
        assert cos >= 0.99 and l2 <= 0.1, (name, cos, l2)
