"""The adaptive third PM level on the GPU (Sec. 2.1.1 Eq. PM3, Sec. 2.2.3)
against the oracle's (oracle/pm3.py), at the force bar.

Cases:
* SMALL: the oracle pin's layout (32 Mpc/h, 8^3 IOS cells, 8^3 + 32^3 meshes,
  the paper's softening of 3.5 cells on every level), subtiles of 2^3 IOS
  cells refined 2x (48^3 local meshes), a clustered random set; the subtiles
  whose densest IOS cell reaches the median are refined.  Also with a capacity
  below the number of subtiles that ask, so that the later ones stay two-level.
* C2LIKE: the 256^3 run's layout at 64^3 particles (32^3 + 128^3 meshes,
  fine softening 2 cells), subtiles of 8^3 IOS cells refined 2x (48^3 local
  meshes, b_3 = 2 local cells = half the PP range), the Zel'dovich
  displacement grown to z = 0; the densest quarter of the subtiles refined.
Checked: the geometry, the refinement map, the local Green's table (FP32
rounding of the oracle's), the total force (median relative error <= 1e-5,
99.9th percentile <= 1e-3), a KDK step (bitwise reproducible, particles
conserved), and that the adjoint refuses a context with the third level."""
import numpy as np
import pytest

from inputs import C2_SMALL
from inputs.workloads import Level, PM3Spec, Workload
from inputs.zeldovich import random_ios, zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import kdk as okdk  # noqa: E402
from oracle import pm3 as opm3  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402

SMALL = Workload(name="pm3-8c-8x32mesh", n_p=10, box=32.0, n_ios=8, levels=(Level(8, 3.5), Level(32, 3.5)),
                 b_pp=0.3)


def _rho_max(count, n_ios, T):
    ns = n_ios // T
    return count.reshape(n_ios, n_ios, n_ios).reshape(ns, T, ns, T, ns, T).max(axis=(1, 3, 5))


def _expected_slots(rho_max, rho_min, max_tiles):
    flag = (rho_max >= rho_min).ravel().astype(np.int64)
    slot = np.cumsum(flag) - flag
    return np.where((flag == 1) & (slot < max_tiles), slot, -1)


def _case(name, capacity=None):
    if name == "SMALL":
        st = random_ios(1000, SMALL.n_ios, SMALL.box, seed=83, clustered=0.6)
        T, r, beta3 = 2, 2, 3.5
        rho_max = _rho_max(st["count"], SMALL.n_ios, T)
        rho_min = int(np.median(rho_max))
        w = SMALL.with_(pm3=PM3Spec(T, r, beta3, rho_min, capacity or 64))
    else:
        w0 = C2_SMALL.with_(displace_to_a=1.0)
        st = zeldovich_ios(w0)
        T, r, beta3 = 8, 2, 2.0
        rho_max = _rho_max(st["count"], w0.n_ios, T)
        rho_min = max(2, int(np.quantile(rho_max, 0.75)))
        w = w0.with_(pm3=PM3Spec(T, r, beta3, rho_min, capacity or 512))
    return w, st, rho_max


def _ctx(w, n_part):
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    for l in range(len(w.levels)):
        ctx.set_green(l)
    ctx.set_green(cube2.LEVEL_PM3)
    return ctx


def _force_bar(got, ref):
    err = np.linalg.norm(got - ref, axis=0)
    floor = 1e-3 * np.sqrt(np.mean((ref ** 2).sum(axis=0)))
    rel = err / np.maximum(np.linalg.norm(ref, axis=0), floor)
    return float(np.median(rel)), float(np.quantile(rel, 0.999))


@pytest.mark.parametrize("name,capacity", [("SMALL", None), ("SMALL", 5), ("C2LIKE", None)])
def test_pm3_force_matches_oracle(name, capacity):
    w, st, rho_max = _case(name, capacity)
    n_part = int(st["count"].sum())
    ctx = _ctx(w, n_part)
    spec = w.pm3
    # geometry as the oracle derives it
    info = ctx.pm3_info()
    h3, b3, B, m = opm3.local_mesh(w, spec.tile, spec.refine, spec.beta)
    assert (info["B"], info["m"], info["ns"]) == (B, m, w.n_ios // spec.tile)
    assert info["H3"] == pytest.approx(h3, rel=1e-14) and info["b3"] == pytest.approx(b3, rel=1e-14)
    # the local Green's table: FP32 rounding of Eq. (Gk) with b_3 and the finest truncation
    g = ctx.get_green(cube2.LEVEL_PM3).cpu().numpy().astype(np.float64) * float(m) ** 3
    ref_g = opm3.pm3_green(w, spec.tile, spec.refine, spec.beta)
    assert np.all(np.abs(g - ref_g) <= 2.0 ** -23 * np.abs(ref_g) + 1e-7 * np.abs(ref_g).max())
    # force and the refinement map it used
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    ctx.check()
    got = p.acc.cpu().numpy().astype(np.float64)
    slots = _expected_slots(rho_max, spec.rho_min, spec.max_tiles)
    assert np.array_equal(ctx.pm3_map().cpu().numpy(), slots)
    used, asked = ctx.pm3_stats()
    assert asked == int((rho_max >= spec.rho_min).sum()) and used == min(asked, spec.max_tiles) and used > 0
    refine = np.where(slots.reshape(rho_max.shape) >= 0, spec.refine, 1)
    ref = opm3.adaptive_force(st["off"], st["count"], st["start"], w, spec.tile, refine, spec.beta)
    med, p999 = _force_bar(got, ref)
    print(f"{name} (capacity {spec.max_tiles}): {used} of {asked} subtiles refined, force median rel {med:.2e}, "
          f"p99.9 {p999:.2e}")
    assert med <= 1e-5 and p999 <= 1e-3
    # the third level changes the force (it is not a no-op at this bar)
    f2 = okdk.total_force(st["off"], st["count"], st["start"], w)
    assert _force_bar(f2, ref)[1] > 1e-3
    ctx.close()


def test_pm3_kdk_step_is_reproducible_and_conserves_particles():
    w, st, _ = _case("C2LIKE")
    n_part = int(st["count"].sum())
    ctx = _ctx(w, n_part)
    a = w.scale_factors()
    outs = []
    for _ in range(2):
        p = cube2.IOSState.from_numpy(st)
        ctx.force(p)
        ctx.kdk_step(p, a[40], a[41])
        ctx.check()
        outs.append(p)
    assert int(outs[0].count.sum().item()) == n_part
    for x, y in zip((outs[0].off, outs[0].count, outs[0].vel, outs[0].acc),
                    (outs[1].off, outs[1].count, outs[1].vel, outs[1].acc)):
        assert torch.equal(x, y)
    assert torch.isfinite(outs[0].acc).all()
    ctx.close()


def test_adjoint_refuses_the_third_level():
    w, st, _ = _case("SMALL")
    ctx = _ctx(w, int(st["count"].sum()))
    with pytest.raises(cube2.Cube2Error) as e:
        ctx.adjoint_init()
    assert e.value.code == cube2.ERR_STATE
    ctx.close()
