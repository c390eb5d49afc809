"""Allocation-free Poisson solve against the context-based one, through the C ABI.

cube2_solve_pm_noalloc serves callers that cannot allocate device memory where
they need a solve; it keeps its working memory in a fixed device array instead.
This test calls it twice in a row (the second call reuses what the first left
in that array) and compares each result with cube2_solve_pm on the same density
and Green's table, to the potential tolerance of the other parity tests.  It
lives in its own file, collected last, and builds everything it needs itself,
so it runs the same alone in a fresh process and after the other tests.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from inputs import C1  # noqa: E402
from inputs.zeldovich import zeldovich_ios  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402


def test_noalloc_solve_matches_context_solve_on_two_calls():
    w = C1
    n = w.levels[0].n_mesh
    st = zeldovich_ios(w)
    ctx = cube2.init_mesh(cube2.make_config(w))
    ctx.set_green(0)
    p = cube2.IOSState.from_numpy(st)
    ctx.deposit(0, p)
    rho = ctx.get_density(0)
    green = ctx.get_green(0)
    ctx.solve_pm(0)
    ref = ctx.get_potential(0)
    ctx.check()
    lib = cube2.library()
    stream = torch.cuda.current_stream().cuda_stream
    scale = ref.abs().max().item()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        rc = lib.cube2_solve_pm_noalloc(ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(green.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), n, ctypes.c_void_p(stream))
        assert rc == cube2.OK, lib.cube2_last_error(None)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= 1e-5 * scale
    ctx.close()


def test_noalloc_solve_rejects_meshes_beyond_its_array():
    lib = cube2.library()
    dummy = torch.zeros(8, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = lib.cube2_solve_pm_noalloc(p, p, p, 256, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == cube2.ERR_UNSUPPORTED_SIZE
    assert b"not supported" in lib.cube2_last_error(None)
