"""The large workload: 1024^3 particles in a 1000 Mpc/h box, coarse 512^3 and
fine 2048^3 meshes, 1024^3 IOS cells, Zel'dovich displacement to z = 0 (one
force evaluation), velocities stored as FP16 codes with a per-IOS-cell FP32
scale.  Its initial conditions come from the device generator
(``inputs.zeldovich_gpu``); the oracle checks sampled outputs one by one: the
FP32 density of both levels at sampled cells (bit-exact against the oracle's
exact accumulator and conversion), both Green's tables at sampled modes, the
velocity codes and scales of sampled cells (bit-exact against the oracle's
codec), and the PP force of a 10^5-particle subsample (and of the first
particle of the densest cells); the total force must be finite and conserve
momentum.  About 215 GB of device memory."""
import numpy as np
import pytest

from inputs import C5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from inputs.zeldovich_gpu import zeldovich_ios_torch  # noqa: E402
from oracle import kdk as okdk  # noqa: E402
from oracle import kernels as okern  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from oracle import pp as opp  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402


def test_large_workload_sampled_parity():
    w = C5
    st = zeldovich_ios_torch(w, momenta=True)
    torch.cuda.empty_cache()
    n_part = w.n_particles
    assert int(st["count"].sum().item()) == n_part
    p = cube2.IOSState(st["off"], st["count"], st["start"], torch.zeros((3, 1), device="cuda"),
                       torch.zeros((3, n_part), device="cuda"))
    ctx = cube2.init_mesh(cube2.make_config(w.with_(vel_fp16=True), n_particles=n_part))
    for l in range(2):
        ctx.set_green(l)
    # host copies for the oracle
    off = st["off"].cpu().numpy().view(np.uint16)
    count = st["count"].cpu().numpy()
    start = st["start"].cpu().numpy()
    rng = np.random.default_rng(55)
    # 0. FP16 velocity storage: codes and scales of sampled occupied cells
    #    bit-exact against the oracle's codec on those cells' FP32 momenta
    ctx.vel_encode(p, st["vel"])
    occupied = np.nonzero(count)[0]
    cells = np.sort(rng.choice(occupied, 200, replace=False))
    cells[-1] = int(np.argmax(count))
    idx = np.concatenate([np.arange(start[c], start[c] + count[c]) for c in cells])
    it = torch.from_numpy(idx).cuda()
    v_host = st["vel"][:, it].cpu().numpy()
    codes, scale = okdk.encode_velocities(v_host, count[cells])
    assert np.array_equal(p.vscale[torch.from_numpy(cells).cuda()].cpu().numpy().view(np.uint32), scale.view(np.uint32))
    assert np.array_equal(p.vel16[:, it].cpu().numpy().view(np.uint16), codes.view(np.uint16))
    del st["vel"], it
    torch.cuda.empty_cache()
    print(f"large workload: stored velocity bytes {6 * n_part + 4 * count.size:.3e} (FP16 + per-cell scale) "
          f"vs FP32 {12 * n_part:.3e}")
    # 1. total force: finite, momentum conserved
    ctx.force(p)
    ctx.check()
    f = p.acc
    assert bool(torch.isfinite(f).all())
    tot = f.double().sum(dim=1).abs().max().item()
    assert tot <= 1e-4 * f.double().abs().sum().item()
    # 2. FP32 density per level at sampled cells (bit-exact)
    for l, lev in enumerate(w.levels):
        n = lev.n_mesh
        ctx.deposit(l, p)
        rho = ctx.get_density(l).view(-1)
        cells = rng.integers(0, n ** 3, 100)
        acc = omesh.deposit_u64_at(off, count, start, w.n_ios, n, cells)
        want = omesh.density_fp32(np.vstack([acc[None, :], np.zeros((n - 1, len(cells)), np.uint64)]), n_part)[0]
        got = rho[torch.from_numpy(cells).cuda()].cpu().numpy()
        assert np.array_equal(got, want)
        del rho
        torch.cuda.empty_cache()
    # 3. Green's tables at sampled modes
    for l, (n, _h, bs, bt) in enumerate(omesh.level_params(w)):
        g = ctx.get_green(l)
        modes = np.stack([rng.integers(0, n // 2 + 1, 64), rng.integers(0, n, 64), rng.integers(0, n, 64)], 1)
        modes[0] = [n // 2, n // 2, n // 2]
        got = g[torch.from_numpy(modes[:, 2]).cuda(), torch.from_numpy(modes[:, 1]).cuda(),
                torch.from_numpy(modes[:, 0]).cuda()].cpu().numpy().astype(np.float64) * float(n) ** 3
        ref = okern.green_at(n, modes, bs, bt)
        assert np.all(np.abs(got - ref) <= 2.0 ** -23 * np.abs(ref) + 1e-7 * np.abs(ref).max())
        del g
        torch.cuda.empty_cache()
    # 4. PP on a 10^5-particle subsample (seeded) and the densest cells' first particles
    ctx.pp_force(p, accumulate=False)
    ctx.check()
    dense = np.argsort(-count)[:3]
    targets = np.concatenate([rng.choice(n_part, 100000, replace=False), [int(start[c]) for c in dense]])
    got = p.acc[:, torch.from_numpy(targets).cuda()].cpu().numpy().astype(np.float64)
    b_pp, b_cut = okdk.pp_params(w)
    ref = opp.pp_force_at_many(off, count, start, w.n_ios, w.box, b_pp, b_cut, targets, n_particles=n_part)
    pair_scale = w.box ** 3 / n_part / (4 * np.pi * b_cut ** 2)
    err = np.linalg.norm(got - ref, axis=0)
    assert np.all(err <= 1e-5 * (pair_scale + np.linalg.norm(ref, axis=0)))
    nz = np.linalg.norm(ref, axis=0) > 0
    rel = err[nz] / np.linalg.norm(ref[:, nz], axis=0)
    print(f"large workload PP, {len(targets)} particles ({nz.sum()} with PP partners): relative error median "
          f"{np.median(rel):.2e}, 99.9th percentile {np.quantile(rel, 0.999):.2e}")
    ctx.close()
