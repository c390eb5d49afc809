"""The TSC assignment (cube2_config.assign_order = 3, the paper's Eq. filter)
through the C ABI against the FP64 oracle: Green's tables with W = sinc^3,
the FP32 overdensity (FP32 atomic sums: within 1e-5 (1 + |delta|)), the total
force at the force bar (median <= 1e-5, 99.9th percentile <= 1e-3) and, for
the Zel'dovich states, a KDK step (particles conserved, state finite)."""
import numpy as np
import pytest

from inputs import C1
from inputs.workloads import C2_SMALL_TSC
from inputs.workloads import Level
from inputs.zeldovich import random_ios, zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import kdk as okdk  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402

C1_TSC = C1.with_(name="pm1-32c-64mesh-tsc", assign_order=3)
CLUSTER_TSC = C1.with_(name="clustered-tsc", n_ios=16, levels=(Level(32, 2.0),), b_pp=0.4, assign_order=3)
# the brick deposit's other mesh-to-IOS ratios: mesh cell = IOS cell, and a quarter of it
CLUSTER_TSC0 = C1.with_(name="clustered-tsc-16mesh", n_ios=16, levels=(Level(16, 1.0),), b_pp=0.4, assign_order=3)
CLUSTER_TSC2 = C1.with_(name="clustered-tsc-64mesh", n_ios=16, levels=(Level(64, 2.0),), b_pp=0.4, assign_order=3)
# 12^3 IOS cells: bricks of 8 and 4 cells (a partial brick on every axis)
RAGGED_TSC = C1.with_(name="ragged-tsc", box=48.0, n_ios=12, levels=(Level(24, 2.0),), b_pp=0.4, assign_order=3)


def _case(name):
    if name == "C1_TSC":
        return C1_TSC, zeldovich_ios(C1_TSC)
    if name == "C2_SMALL_TSC":
        return C2_SMALL_TSC, zeldovich_ios(C2_SMALL_TSC)
    if name == "RAGGED_TSC":
        return RAGGED_TSC, random_ios(12 ** 3, 12, RAGGED_TSC.box, seed=31, clustered=0.3)
    w = {"CLUSTER_TSC": CLUSTER_TSC, "CLUSTER_TSC0": CLUSTER_TSC0, "CLUSTER_TSC2": CLUSTER_TSC2}[name]
    return w, random_ios(5000, 16, w.box, seed=32, clustered=0.8)


@pytest.mark.parametrize("name", ["C1_TSC", "C2_SMALL_TSC", "CLUSTER_TSC", "CLUSTER_TSC0", "CLUSTER_TSC2",
                                  "RAGGED_TSC"])
def test_tsc_path_matches_oracle(name):
    w, st = _case(name)
    n_part = int(st["count"].sum())
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
    for l in range(len(w.levels)):
        ctx.set_green(l)
    greens = omesh.green_tables(w)
    p = cube2.IOSState.from_numpy(st)
    for l, lev in enumerate(w.levels):
        n = lev.n_mesh
        g = ctx.get_green(l).cpu().numpy().astype(np.float64) * float(n) ** 3
        assert np.all(np.abs(g - greens[l]) <= 2.0 ** -23 * np.abs(greens[l]) + 1e-7 * np.abs(greens[l]).max())
        ctx.deposit(l, p)
        rho = ctx.get_density(l).cpu().numpy().astype(np.float64)
        ref = omesh.density_tsc(st["off"], st["count"], w.n_ios, n)
        assert np.all(np.abs(rho - ref) <= 1e-5 * (1.0 + np.abs(ref))), np.abs(rho - ref).max()
    ctx.force(p)
    ctx.check()
    f = p.acc.cpu().numpy().astype(np.float64)
    ref = okdk.total_force(st["off"], st["count"], st["start"], w, greens)
    err = np.linalg.norm(f - ref, axis=0)
    mag = np.linalg.norm(ref, axis=0)
    rel = err / np.maximum(mag, 1e-3 * np.sqrt(np.mean(mag ** 2)))
    assert np.median(rel) <= 1e-5 and np.quantile(rel, 0.999) <= 1e-3, (np.median(rel), np.quantile(rel, 0.999))
    if not name.startswith(("CLUSTER", "RAGGED")):   # a Zel'dovich state: one KDK step of its schedule
        a = w.scale_factors()
        ctx.kdk_step(p, a[0], a[1])
        ctx.check()
        assert int(p.count.sum().item()) == n_part
        assert bool(torch.isfinite(p.vel).all()) and bool(torch.isfinite(p.acc).all())
    # the exact-integer accumulator and the adjoint are CIC-only
    with pytest.raises(cube2.Cube2Error):
        ctx.deposit_u64(0, p)
    ctx.adjoint_init()
    with pytest.raises(cube2.Cube2Error):
        ctx.force_vjp(p, torch.zeros_like(p.acc))
    ctx.close()
