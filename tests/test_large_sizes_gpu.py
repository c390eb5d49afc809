"""The largest meshes the library takes, on a sparse particle set that the
oracle can check exactly at sampled points: with a handful of particles the
density is a constant background plus a few nonzero cells, so its DFT at any
mode is a short direct sum.  Checks the deposit (bit-exact at the occupied
cells, exact total), the Green's table at sampled modes, and the forward FFT
at sampled modes, for a radix-3 mesh (768^3), 1024^3 and the largest
supported mesh, 2048^3 (about 180 GB of device memory at its peak)."""
import numpy as np
import pytest

from inputs import C1
from inputs.workloads import Level
from inputs.zeldovich import ios_from_positions

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import kernels as okern  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402


@pytest.mark.parametrize("n", [768, 1024, 2048])
def test_large_mesh_deposit_green_and_fft(n):
    n_ios = n // 2
    w = C1.with_(name=f"large-{n}", n_p=16, box=float(n_ios), n_ios=n_ios, levels=(Level(n, 2.0),), b_pp=0.1)
    rng = np.random.default_rng(n)
    npart = 12
    pos = rng.uniform(0.0, w.box, size=(3, npart))
    st = ios_from_positions(pos, np.zeros((3, npart)), n_ios, w.box)
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=npart))
    ctx.set_green(0)
    p = cube2.IOSState.from_numpy(st)
    # deposit: the FP32 density grid, bit-exact at every occupied cell against
    # the oracle's exact accumulator and its FP32 conversion; empty cells hold
    # the conversion of 0 (the 64-bit grid itself is not copied out: 8 n^3 bytes)
    ctx.deposit(0, p)
    rho = ctx.get_density(0).view(-1)
    # the oracle's FP32 conversion reads the mesh size from the first axis:
    # convert a zero and the sampled accumulators on an (n, k) stand-in grid
    conv = lambda a: omesh.density_fp32(np.vstack([a, np.zeros((n - 1, a.shape[1]), np.uint64)]), npart)[0]
    empty = float(conv(np.zeros((1, 1), np.uint64))[0])
    dev = torch.nonzero(rho != empty).view(-1)
    cells = dev.cpu().numpy()
    assert 0 < len(cells) <= 8 * npart
    acc = omesh.deposit_u64_at(st["off"], st["count"], st["start"], n_ios, n, cells)
    assert int(sum(int(x) for x in acc)) == npart << 48
    assert np.array_equal(rho[dev].cpu().numpy(), conv(acc[None, :]))
    vals = (rho[dev].double() - empty).cpu().numpy()
    del rho
    torch.cuda.empty_cache()
    # Green's table at sampled modes
    g = ctx.get_green(0)
    modes = np.stack([rng.integers(0, n // 2 + 1, 64), rng.integers(0, n, 64), rng.integers(0, n, 64)], 1)
    modes[0] = [n // 2, n // 2, n // 2]
    modes[1] = [1, 0, 0]
    gg = g[torch.from_numpy(modes[:, 2]).cuda(), torch.from_numpy(modes[:, 1]).cuda(),
           torch.from_numpy(modes[:, 0]).cuda()].cpu().numpy().astype(np.float64) * float(n) ** 3
    gr = okern.green_at(n, modes, 2.0, None)
    assert np.all(np.abs(gg - gr) <= 2.0 ** -23 * np.abs(gr) + 1e-7 * np.abs(gr).max())
    del g
    torch.cuda.empty_cache()
    # forward FFT of the FP32 density at sampled modes against a direct sum
    # over the occupied cells (the background is constant: k = 0 only)
    ctx.deposit(0, p)
    idx = cells
    cx, cy, cz = idx % n, (idx // n) % n, idx // (n * n)
    spec = ctx.debug_forward_fft(0)
    km = modes[2:]
    km = km[(km != 0).any(axis=1)]          # k = 0 carries the background
    got = spec[torch.from_numpy(km[:, 2]).cuda(), torch.from_numpy(km[:, 1]).cuda(),
               torch.from_numpy(km[:, 0]).cuda()].cpu().numpy().astype(np.complex128)
    ph = -2j * np.pi / n * (np.outer(km[:, 0], cx) + np.outer(km[:, 1], cy) + np.outer(km[:, 2], cz))
    ref = (np.exp(ph) * vals[None, :]).sum(axis=1)
    scale = np.abs(vals).sum()
    assert np.abs(got - ref).max() <= 1e-5 * scale, np.abs(got - ref).max() / scale
    ctx.check()
    ctx.close()
