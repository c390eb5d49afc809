"""GPU (CUDA path through the C ABI) against the FP64 oracle, element by element.

Tolerances: integer work (deposit accumulators, IOS counts) bit-exact; the FP32
density grid bit-exact against its stated conversion of the exact integers; the
Green's table to FP32 rounding of the FP64 value; forces with the relative error
rel_i = |F_gpu - F_or| / max(|F_or|, 1e-3 rms|F_or|): median <= 1e-5 and 99.9th
percentile <= 1e-3 (the precision targets of this project for FP32 forces).
"""
import numpy as np
import pytest

from inputs import C1, C2_SMALL
from inputs.workloads import Level
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

MEDIAN_TOL, P999_TOL = 1e-5, 1e-3

# ragged: 12^3 IOS cells (a full and a partial 8-cell deposit brick per axis),
# 12^3 (IOS/mesh = 1) and 24^3 (1/2) meshes, radix-3 FFTs
RAGGED = C1.with_(name="ragged-12", n_p=12, box=24.0, n_ios=12,
                  levels=(Level(12, 3.0), Level(24, 2.0)), b_pp=0.2)
# clustered random particles in a C1-like box (uneven cell counts)
CLUSTER = C1.with_(name="clustered", n_ios=16, levels=(Level(32, 2.0),), b_pp=0.4)
# a coarse mesh at half and a fine mesh at four times the IOS resolution: 4-cell
# bricks, whose coarse tiles start off the 4-cell alignment of the 16-byte
# tile copies in half of the bricks (the gather's 4-byte staging path)
MIXED = C1.with_(name="mixed-8-64", n_ios=16, levels=(Level(8, 3.5), Level(64, 2.0)), b_pp=0.2)


def rel_err(f_gpu, f_or):
    err = np.linalg.norm(f_gpu - f_or, axis=0)
    mag = np.linalg.norm(f_or, axis=0)
    floor = 1e-3 * np.sqrt(np.mean(mag ** 2))
    return err / np.maximum(mag, floor)


def assert_force_close(f_gpu, f_or, what=""):
    rel = rel_err(np.asarray(f_gpu, np.float64), f_or)
    med, p999 = np.median(rel), np.quantile(rel, 0.999)
    print(f"\n  force error {what}: median {med:.2e}, 99.9th percentile {p999:.2e} (N = {rel.size})")
    assert med <= MEDIAN_TOL and p999 <= P999_TOL, f"{what}: median {med:.3e}, p99.9 {p999:.3e}"


def _state(name):
    if name == "C1":
        return C1, zeldovich_ios(C1)
    if name == "C2_SMALL":
        return C2_SMALL, zeldovich_ios(C2_SMALL)
    if name == "RAGGED":
        return RAGGED, random_ios(12 ** 3, 12, RAGGED.box, seed=31, clustered=0.3)
    if name == "CLUSTER":
        return CLUSTER, random_ios(5000, 16, CLUSTER.box, seed=32, clustered=0.8)
    if name == "MIXED":
        return MIXED, random_ios(5000, 16, MIXED.box, seed=34, clustered=0.5)
    if name == "C4_24":
        # an ensemble box with a radix-3 mesh: 24^3 particles, 48^3 mesh
        from inputs.workloads import c4_ensemble
        w = c4_ensemble(n_boxes=1, seed=41, sizes=(24,))[0]
        return w, zeldovich_ios(w)
    if name == "DENSE":
        # a 4500-particle clump: cells of hundreds of particles (the PP kernel's
        # sub-cell ordering of dense cells and its shared-stream path, the
        # deposit's heavily loaded bricks)
        from inputs.zeldovich import ios_from_positions
        rng = np.random.Generator(np.random.Philox(33))
        clump = 32.0 + rng.normal(0.0, 2.0, size=(3, 4500))
        pos = np.concatenate([clump, rng.uniform(0.0, CLUSTER.box, size=(3, 1500))], axis=1) % CLUSTER.box
        return CLUSTER, ios_from_positions(pos, rng.normal(0.0, 1.0, size=pos.shape), 16, CLUSTER.box)
    raise KeyError(name)


_CACHE = {}


def case(name):
    """(workload, numpy state, oracle green tables, gpu context) cached per module."""
    if name not in _CACHE:
        w, st = _state(name)
        n_part = int(st["count"].sum())
        greens = omesh.green_tables(w)
        ctx = cube2.init_mesh(cube2.make_config(w, n_particles=n_part))
        for l in range(len(w.levels)):
            ctx.set_green(l)
        _CACHE[name] = (w, st, greens, ctx)
    return _CACHE[name]


ALL = ["C1", "C2_SMALL", "RAGGED", "CLUSTER", "DENSE", "C4_24", "MIXED"]


@pytest.mark.parametrize("name", ALL)
def test_green_table_is_fp32_rounding_of_fp64(name):
    w, st, greens, ctx = case(name)
    for l, lev in enumerate(w.levels):
        n = lev.n_mesh
        g = ctx.get_green(l).cpu().numpy().astype(np.float64) * float(n) ** 3
        ref = greens[l]
        tol = 2.0 ** -23 * np.abs(ref) + 1e-7 * np.abs(ref).max()
        assert np.all(np.abs(g - ref) <= tol), (l, np.abs(g - ref).max())


@pytest.mark.parametrize("name", ALL)
def test_deposit_is_bit_exact(name):
    w, st, _, ctx = case(name)
    n_part = int(st["count"].sum())
    p = cube2.IOSState.from_numpy(st)
    for l, lev in enumerate(w.levels):
        acc = omesh.deposit_u64(st["off"], st["count"], w.n_ios, lev.n_mesh)
        got = ctx.deposit_u64(l, p).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, acc), f"level {l}: {np.count_nonzero(got != acc)} cells differ"
        ctx.deposit(l, p)
        d32 = ctx.get_density(l).cpu().numpy()
        assert np.array_equal(d32.view(np.uint32), omesh.density_fp32(acc, n_part).view(np.uint32))
    # every level in one particle pass gives the same grids
    ctx.deposit(-1, p)
    for l, lev in enumerate(w.levels):
        acc = omesh.deposit_u64(st["off"], st["count"], w.n_ios, lev.n_mesh)
        d32 = ctx.get_density(l).cpu().numpy()
        assert np.array_equal(d32.view(np.uint32), omesh.density_fp32(acc, n_part).view(np.uint32))
    ctx.check()


@pytest.mark.parametrize("name", ALL)
def test_forward_fft_matches_library_fft(name):
    w, st, _, ctx = case(name)
    n_part = int(st["count"].sum())
    p = cube2.IOSState.from_numpy(st)
    for l, lev in enumerate(w.levels):
        ctx.deposit(l, p)
        d32 = ctx.get_density(l).cpu().numpy()
        spec = ctx.debug_forward_fft(l).cpu().numpy().astype(np.complex128)
        ref = np.fft.rfftn(d32.astype(np.float64))
        err = np.linalg.norm(spec - ref) / np.linalg.norm(ref)
        assert err < 2e-7 * np.log2(lev.n_mesh) + 1e-7, (l, err)


@pytest.mark.parametrize("name", ALL)
def test_potential_matches_oracle(name):
    w, st, greens, ctx = case(name)
    n_part = int(st["count"].sum())
    p = cube2.IOSState.from_numpy(st)
    for l, lev in enumerate(w.levels):
        ctx.deposit(l, p)
        ctx.solve_pm(l)
        phi = ctx.get_potential(l).cpu().numpy().astype(np.float64)
        acc = omesh.deposit_u64(st["off"], st["count"], w.n_ios, lev.n_mesh)
        ref = omesh.solve_potential(omesh.density(acc, n_part), greens[l])
        err = np.abs(phi - ref)
        assert err.max() <= 1e-5 * np.abs(ref).max(), (l, err.max() / np.abs(ref).max())
        assert np.linalg.norm(phi - ref) <= 2e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", ALL)
def test_pm_and_pp_forces_match_oracle(name):
    w, st, greens, ctx = case(name)
    p = cube2.IOSState.from_numpy(st)
    params = omesh.level_params(w)
    for l in range(len(w.levels)):
        ctx.deposit(l, p)
        ctx.solve_pm(l)
        ctx.interp_force(l, p, accumulate=False)
        n, h, _, _ = params[l]
        ref, _ = omesh.pm_force_level(st["off"], st["count"], w.n_ios, n, h, greens[l])
        assert_force_close(p.acc.cpu().numpy(), ref, f"{name} PM level {l}")
    b_pp, b_cut = okdk.pp_params(w)
    ctx.pp_force(p, accumulate=False)
    ref = opp.pp_force(st["off"], st["count"], st["start"], w.n_ios, w.box, b_pp, b_cut)
    got = p.acc.cpu().numpy().astype(np.float64)
    # absolute error against the pair-force scale V_p / (4 pi b_cut^2): the PP sum
    # of a particle is a handful of such terms, most of them near the cutoff
    # plus an FP32 summation term relative to the particle's own PP force
    pair_scale = w.box ** 3 / int(st["count"].sum()) / (4 * np.pi * b_cut ** 2)
    err = np.linalg.norm(got - ref, axis=0)
    bound = 1e-5 * (pair_scale + np.linalg.norm(ref, axis=0))
    assert np.all(err <= bound), (err / bound).max()
    assert_force_close(got, ref, f"{name} PP")
    ctx.check()


@pytest.mark.parametrize("name", ALL)
def test_total_force_matches_oracle(name):
    w, st, greens, ctx = case(name)
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    ctx.check()
    ref = okdk.total_force(st["off"], st["count"], st["start"], w, greens)
    assert_force_close(p.acc.cpu().numpy(), ref, f"{name} total force")


def test_force_conserves_momentum_and_is_deterministic():
    w, st, _, ctx = case("CLUSTER")
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    f1 = p.acc.clone()
    ctx.force(p)
    assert torch.equal(f1, p.acc)
    f = f1.cpu().numpy().astype(np.float64)
    assert np.abs(f.sum(axis=1)).max() < 1e-5 * np.abs(f).sum()


def _oracle_drift_units(st, w, greens, a0, a1, f0_gpu):
    """Unrounded oracle drift in fixed-point units and a bound on how far the
    GPU's FP32 displacement can sit from it, both in the re-binned order.

    The bound covers the first kick's force difference (GPU F(x0) against the
    oracle's) and FP32 rounding of the momentum and of p * Dr."""
    f0 = okdk.total_force(st["off"], st["count"], st["start"], w, greens)
    ah = 0.5 * (a0 + a1)
    k1 = 1.5 * w.omega_m * okdk.kick_integral(a0, ah, w.omega_m, w.omega_l)
    v1 = st["vel"].astype(np.float64) + k1 * f0
    dfac = okdk.drift_integral(a0, a1, w.omega_m, w.omega_l) * 65536 / (w.box / w.n_ios)
    disp = v1 * dfac
    slack = np.abs(k1 * (f0_gpu - f0)) * dfac + 4e-7 * (np.abs(disp) + np.abs(k1 * f0 * dfac)) + 1e-3
    X = (omesh.fixed_coords(st["off"], st["count"], w.n_ios) + np.rint(disp).astype(np.int64)) % (w.n_ios * 65536)
    c3 = X >> 16
    order = np.argsort((c3[2] * w.n_ios + c3[1]) * w.n_ios + c3[0], kind="stable")
    return disp[:, order], slack[:, order]


@pytest.mark.parametrize("name", ["C1", "C2_SMALL", "CLUSTER", "DENSE"])
def test_kdk_step_matches_oracle(name):
    w, st, greens, ctx = case(name)
    a = w.scale_factors()
    a0, a1 = a[0], a[1]
    if name in ("CLUSTER", "DENSE"):
        a0, a1 = 0.5, 0.52
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    f0_gpu = p.acc.cpu().numpy().astype(np.float64)
    ctx.kdk_step(p, a0, a1)
    ctx.check()
    got = p.to_numpy()
    ref = okdk.kdk_step(dict(off=st["off"], count=st["count"], start=st["start"],
                             vel=st["vel"].astype(np.float64), acc=None), w, a0, a1, greens)
    assert np.array_equal(got["count"], ref["count"])
    assert np.array_equal(got["start"], ref["start"])
    # offsets: equal, except by one fixed-point unit where the oracle's FP64
    # displacement lies within FP32 reach of a rounding boundary
    disp, slack = _oracle_drift_units(st, w, greens, a0, a1, f0_gpu)
    d = np.abs(got["off"].astype(np.int64) - ref["off"].astype(np.int64))
    d = np.minimum(d, 65536 - d)
    assert d.max() <= 1
    frac = disp - np.floor(disp)
    near = np.abs(frac - 0.5) <= slack
    assert np.all(near[d == 1]), np.count_nonzero(d == 1) - np.count_nonzero(near[d == 1])
    assert np.mean(d == 0) >= 0.99
    assert_force_close(got["vel"], ref["vel"], "velocity")
    assert_force_close(got["acc"], ref["acc"], "force after step")


def test_kdk_far_movers_take_the_general_rebin_path():
    # momenta large enough that many particles cross more than one IOS cell
    w, st, greens, ctx = case("CLUSTER")
    st = dict(st)
    st["vel"] = (st["vel"] * 60.0).astype(np.float32)
    a0, a1 = 0.5, 0.52
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    ctx.kdk_step(p, a0, a1)
    ctx.check()
    got = p.to_numpy()
    ref = okdk.kdk_step(dict(off=st["off"], count=st["count"], start=st["start"],
                             vel=st["vel"].astype(np.float64), acc=None), w, a0, a1, greens)
    assert np.array_equal(got["count"], ref["count"])
    d = np.abs(got["off"].astype(np.int64) - ref["off"].astype(np.int64))
    assert np.minimum(d, 65536 - d).max() <= 1
    assert_force_close(got["vel"], ref["vel"], "velocity")


@pytest.mark.parametrize("n", [33, 1000, 1024, 1025, 20000])
def test_rebin_sorts_huge_cells_stably(n):
    # n particles packed into one IOS cell: the atomic slots scramble the cell,
    # and the sort must restore the old order exactly (a vanishing step moves
    # nobody): one warp per cell up to 1024 particles, one CTA above (runs of
    # 8192 merged through scratch for 20000)
    w = CLUSTER
    rng = np.random.default_rng(5)
    cell = np.array([5.3, 9.1, 13.7])
    pos = (np.floor(cell / 4.0) * 4.0)[:, None] + rng.uniform(0.0, 4.0, size=(3, n))
    pos = np.concatenate([pos, rng.uniform(0, w.box, size=(3, 3000))], axis=1)
    from inputs.zeldovich import ios_from_positions
    st = ios_from_positions(pos, np.zeros_like(pos), w.n_ios, w.box)
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=pos.shape[1]))
    ctx.set_green(0)
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    ctx.kdk_step(p, 0.5, 0.5 + 1e-12)
    ctx.check()
    got = p.to_numpy()
    assert np.array_equal(got["count"], st["count"]) and np.array_equal(got["off"], st["off"])
    assert got["count"].max() >= n


def test_kdk_is_deterministic_and_stable_order():
    w, st, _, ctx = case("CLUSTER")
    outs = []
    for _ in range(2):
        p = cube2.IOSState.from_numpy(st)
        ctx.force(p)
        for k in range(3):
            ctx.kdk_step(p, 0.5 + 0.02 * k, 0.52 + 0.02 * k)
        outs.append(p.to_numpy())
    for key in ("off", "count", "start", "vel", "acc"):
        assert np.array_equal(outs[0][key], outs[1][key]), key


def test_call_order_and_argument_errors():
    w, st, _, _ = case("C1")
    ctx = cube2.init_mesh(cube2.make_config(w))
    p = cube2.IOSState.from_numpy(st)
    with pytest.raises(cube2.Cube2Error) as e:
        ctx.solve_pm(0)                      # no Green's table, no density
    assert e.value.code == cube2.ERR_STATE
    with pytest.raises(cube2.Cube2Error) as e:
        ctx.force(p)                         # no Green's table
    assert e.value.code == cube2.ERR_STATE
    with pytest.raises(cube2.Cube2Error) as e:
        ctx.deposit(3, p)
    assert e.value.code == cube2.ERR_BAD_ARG
    ctx.close()


def test_single_particle_and_empty_box():
    w = C1.with_(n_ios=8, levels=(Level(16, 2.0),), box=16.0, b_pp=0.2)
    from inputs.zeldovich import ios_from_positions
    st = ios_from_positions(np.array([[3.3], [7.9], [12.2]]), np.zeros((3, 1)), 8, 16.0)
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=1))
    ctx.set_green(0)
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    ctx.check()
    f = p.acc.cpu().numpy()
    assert np.abs(f).max() < 1e-6 * 16.0 ** 3 / (4 * np.pi * 2.0 ** 2)
    # empty box: every call is a no-op on zero particles
    st0 = dict(off=np.zeros((3, 0), np.uint16), count=np.zeros(8 ** 3, np.int32),
               start=np.zeros(8 ** 3, np.int32), vel=np.zeros((3, 0), np.float32))
    ctx0 = cube2.init_mesh(cube2.make_config(w, n_particles=0))
    ctx0.set_green(0)
    p0 = cube2.IOSState.from_numpy(st0)
    ctx0.force(p0)
    ctx0.kdk_step(p0, 0.5, 0.6)
    ctx0.check()
    assert int(p0.count.sum()) == 0
    # ... and so is the adjoint chain
    ctx0.adjoint_init()
    assert ctx0.force_vjp(p0, torch.zeros(3, 0, device="cuda")).shape == (3, 0)
    loss, g = ctx0.density_mse_vjp(0, p0, torch.zeros(16, 16, 16, device="cuda"))
    assert loss == 0.0 and g.shape == (3, 0)
    loss, gx, gv = cube2.loss_gradient(ctx0, p0, torch.zeros(16, 16, 16, device="cuda"), [0.5, 0.6, 0.7])
    ctx0.check()
    assert loss == 0.0 and gx.shape == (3, 0) and gv.shape == (3, 0)


def test_host_buffer_step_equals_device_step():
    """cube2_kdk_step_host (pinned host state, uploads, step, overlapped
    downloads) leaves the host arrays bitwise equal to a device-side step; the
    host's start array is not read (the device forms it from count)."""
    w, st, _, ctx = case("C2_SMALL")
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    a = w.scale_factors()
    host = cube2.IOSState(*(x.cpu().pin_memory() for x in (p.off, p.count, p.start, p.vel, p.acc)))
    host.start.fill_(-7)          # not read: formed on the device from count
    dev = p.clone()
    ctx.kdk_step(p, a[0], a[1])
    ctx.kdk_step_host(dev, host, a[0], a[1])
    ctx.check()
    for x, y in zip((host.off, host.count, host.start, host.vel, host.acc), (p.off, p.count, p.start, p.vel, p.acc)):
        assert torch.equal(x, y.cpu())
