"""Parity of the solve path bench.py times, at its own size: the 256^3-particle
workload with its 128^3 and 512^3 meshes (the N = 512 and N = 128 template
instantiations of every FFT pass, the reduced-table z pass included), against
the FP64 oracle computed in full on the host.

Two particle states run through the same context:
* the workload's initial conditions (Zel'dovich displacement at z = 49);
* a clustered state: the same Gaussian field with its Zel'dovich displacement
  grown to z = 0 (shell-crossed sheets and filaments, cells of up to a few
  dozen particles), made by the seeded generator alone.

Checked, per state: the 512^3 forward FFT of the deposited grid against
numpy's rfftn over the whole spectrum; both potentials over the whole mesh;
the force of each PM level, the PP force and the total force at 2000 random
particles plus the first particle of the five densest cells, at the force
bar (median relative error <= 1e-5, 99.9th percentile <= 1e-3, floor 1e-3
of the rms force).  The oracle's Green's tables are evaluated once per sorted
mode triple (``oracle.kernels.green_by_symmetry``) in a spawned process pool.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from inputs import C2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from inputs.zeldovich import zeldovich_ios  # noqa: E402
from oracle import kdk as okdk  # noqa: E402
from oracle import kernels as okern  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from oracle import pp as opp  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402

W = C2
STATES = {"ics-z49": W, "zeldovich-to-z0": W.with_(displace_to_a=1.0)}
N_SAMPLE = 2000


def _rel(got, ref):
    err = np.linalg.norm(got - ref, axis=0)
    floor = 1e-3 * np.sqrt(np.mean((ref ** 2).sum(axis=0)))
    return err / np.maximum(np.linalg.norm(ref, axis=0), floor)


def _assert_force_bar(name, got, ref):
    rel = _rel(got, ref)
    med, p999 = float(np.median(rel)), float(np.quantile(rel, 0.999))
    print(f"{name}: median rel {med:.2e}, p99.9 {p999:.2e}, max {rel.max():.2e} ({rel.size} particles)")
    assert med <= 1e-5 and p999 <= 1e-3, (name, med, p999)


@pytest.fixture(scope="module")
def greens():
    """Oracle Green's tables of both levels (FP64, rfftn layout)."""
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return [okern.green_by_symmetry(n, bs, bt, mapper=pool.map)
                for (n, _h, bs, bt) in omesh.level_params(W)]


@pytest.fixture(scope="module")
def ctx():
    c = cube2.init_mesh(cube2.make_config(W))
    for l in range(len(W.levels)):
        c.set_green(l)
    yield c
    c.close()


@pytest.fixture(scope="module", params=list(STATES))
def case(request, greens, ctx):
    w = STATES[request.param]
    st = zeldovich_ios(w)
    n_part = W.n_particles
    assert int(st["count"].sum()) == n_part
    p = cube2.IOSState.from_numpy(st)
    rng = np.random.default_rng(21)
    dense = np.argsort(-st["count"], kind="stable")[:5]
    targets = np.concatenate([rng.integers(0, n_part, N_SAMPLE), st["start"][dense].astype(np.int64)])
    # GPU: deposit both levels, the 512^3 forward spectrum, both solves and potentials
    ctx.deposit(-1, p)
    spec_gpu = ctx.debug_forward_fft(1).cpu().numpy()
    phis_gpu, level_f_gpu = [], []
    for l in range(len(W.levels)):
        ctx.solve_pm(l)
        phis_gpu.append(ctx.get_potential(l).cpu().numpy())
        ctx.interp_force(l, p, accumulate=False)
        level_f_gpu.append(p.acc[:, torch.from_numpy(targets).cuda()].cpu().numpy().astype(np.float64))
    ctx.pp_force(p, accumulate=False)
    pp_gpu = p.acc[:, torch.from_numpy(targets).cuda()].cpu().numpy().astype(np.float64)
    ctx.force(p)
    total_gpu = p.acc[:, torch.from_numpy(targets).cuda()].cpu().numpy().astype(np.float64)
    ctx.check()
    # oracle
    phis, level_f, spec_ref = [], [], None
    for l, ((n, h, _bs, _bt), g) in enumerate(zip(omesh.level_params(W), greens)):
        acc = omesh.deposit_u64(st["off"], st["count"], W.n_ios, n)
        if l == 1:
            spec_ref = np.fft.rfftn(omesh.density_fp32(acc, n_part).astype(np.float64))
        phi = omesh.solve_potential(omesh.density(acc, n_part), g)
        phis.append(phi)
        level_f.append(omesh.pm_force_level_at(phi, st["off"], st["count"], st["start"], W.n_ios, h, targets))
        del acc
    b_pp, b_cut = okdk.pp_params(W)
    pp_ref = opp.pp_force_at(st["off"], st["count"], st["start"], W.n_ios, W.box, b_pp, b_cut, targets)
    return dict(name=request.param, st=st, targets=targets, spec_gpu=spec_gpu, spec_ref=spec_ref,
                phis_gpu=phis_gpu, phis=phis, level_f_gpu=level_f_gpu, level_f=level_f, pp_gpu=pp_gpu,
                pp_ref=pp_ref, total_gpu=total_gpu, b_cut=b_cut)


def test_forward_fft_512_whole_spectrum(case):
    got, ref = case["spec_gpu"], case["spec_ref"]
    assert got.shape == ref.shape == (512, 512, 257)
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"{case['name']}: 512^3 forward FFT rel L2 {l2:.2e}, max {mx:.2e}")
    assert l2 < 2e-7 * np.log2(512) and mx < 1e-5


def test_potentials_whole_mesh(case):
    for l, (got, ref) in enumerate(zip(case["phis_gpu"], case["phis"])):
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print(f"{case['name']}: level {l} ({ref.shape[0]}^3) potential max error {err:.2e} of max |phi|")
        assert err < 1e-5


def test_level_pp_and_total_forces_at_sampled_particles(case):
    for l, (got, ref) in enumerate(zip(case["level_f_gpu"], case["level_f"])):
        _assert_force_bar(f"{case['name']} level {l} PM force", got, ref)
    # PP: FP32 rounding of a sum of pair terms, each at most the pair scale
    pair_scale = W.box ** 3 / W.n_particles / (4 * np.pi * case["b_cut"] ** 2)
    err = np.linalg.norm(case["pp_gpu"] - case["pp_ref"], axis=0)
    assert np.all(err <= 1e-5 * (pair_scale + np.linalg.norm(case["pp_ref"], axis=0)))
    total_ref = case["level_f"][0] + case["level_f"][1] + case["pp_ref"]
    _assert_force_bar(f"{case['name']} total force", case["total_gpu"], total_ref)
    counts = case["st"]["count"]
    print(f"{case['name']}: densest IOS cell {counts.max()} particles, occupied cells {np.mean(counts > 0):.3f}")
