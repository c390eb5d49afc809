"""Allocation-free Poisson solve against the context-based one, through the C ABI.

cube2_solve_pm_noalloc serves callers that cannot allocate device memory where
they need a solve; it keeps its working memory in a fixed device array instead.
Each case calls it twice in a row (the second call reuses what the first left
in that array) and compares each result with cube2_solve_pm on the same density
and Green's table, to the potential tolerance of the other parity tests, for a
radix-2 mesh, a radix-3 mesh and the 128^3 limit that fills the array; a
sequence 128 -> 48 -> 128 checks that what a larger mesh leaves behind does
not leak into a smaller one.  The file is collected last and builds everything
it needs itself, so it runs the same alone in a fresh process and after the
other tests.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from inputs import C1  # noqa: E402
from inputs.workloads import Level, Workload  # noqa: E402
from inputs.zeldovich import random_ios, zeldovich_ios  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402

_CASES = {}


def _case(n):
    """(rho, green, phi from cube2_solve_pm) for an n^3 mesh, built once."""
    if n in _CASES:
        return _CASES[n]
    if n == 64:
        w, st = C1, zeldovich_ios(C1)
    else:
        w = Workload(name=f"noalloc-{n}", n_p=n // 2, box=float(n // 2), n_ios=n // 2, levels=(Level(n, 2.0),),
                     b_pp=0.1)
        st = random_ios(20000, n // 2, w.box, seed=n, clustered=0.5)
    ctx = cube2.init_mesh(cube2.make_config(w, n_particles=int(st["count"].sum())))
    ctx.set_green(0)
    p = cube2.IOSState.from_numpy(st)
    ctx.deposit(0, p)
    rho = ctx.get_density(0)
    green = ctx.get_green(0)
    ctx.solve_pm(0)
    ref = ctx.get_potential(0)
    ctx.check()
    ctx.close()
    _CASES[n] = (rho, green, ref)
    return _CASES[n]


def _noalloc(rho, green, n):
    lib = cube2.library()
    out = torch.full_like(rho, float("nan"))
    rc = lib.cube2_solve_pm_noalloc(ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(green.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), n,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == cube2.OK, lib.cube2_last_error(None)
    torch.cuda.synchronize()
    return out


def _check(n, out):
    ref = _CASES[n][2]
    assert torch.isfinite(out).all()
    err = (out - ref).abs().max().item() / ref.abs().max().item()
    assert err <= 1e-5, (n, err)


@pytest.mark.parametrize("n", [64, 48, 128])
def test_noalloc_solve_matches_context_solve_on_two_calls(n):
    rho, green, _ref = _case(n)
    for _ in range(2):
        _check(n, _noalloc(rho, green, n))


def test_noalloc_solve_after_a_larger_mesh():
    for n in (128, 48, 128):
        rho, green, _ref = _case(n)
        _check(n, _noalloc(rho, green, n))


def test_noalloc_wrapper_validates_before_calling_the_library():
    rho, green, ref = _case(48)
    phi = torch.empty_like(rho)
    cube2.solve_pm_noalloc(rho, green, phi)
    torch.cuda.synchronize()
    _check(48, phi)
    with pytest.raises(ValueError):
        cube2.solve_pm_noalloc(rho.double(), green, phi)
    with pytest.raises(ValueError):
        cube2.solve_pm_noalloc(rho, green[:, :, :-1], phi)
    with pytest.raises(ValueError):
        cube2.solve_pm_noalloc(rho.transpose(0, 2), green, phi)
    with pytest.raises(ValueError):
        cube2.solve_pm_noalloc(rho, green, phi.cpu())


def test_noalloc_solve_rejects_meshes_beyond_its_array():
    lib = cube2.library()
    dummy = torch.zeros(8, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.cube2_solve_pm_noalloc(p, p, p, 256, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == cube2.ERR_UNSUPPORTED_SIZE
    assert b"not supported" in lib.cube2_last_error(None)
