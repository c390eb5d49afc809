"""The kernel-detected error words, triggered by host-built inputs (no GPU
fault is involved: every index stays in bounds, the kernels record the
condition in the context's sticky status word and cube2_check reports it).

* CUBE2_ERR_CAPACITY: 65 536 particles on one mesh-cell centre put 2^16 x 2^48
  = 2^64 into one uint64 accumulator cell; 65 535 of them fit exactly.
* CUBE2_ERR_NONFINITE: a NaN momentum reaches the kick.
* CUBE2_ERR_DISPLACEMENT: a finite momentum that drifts a particle by half
  the box or more in one step.
After each error the status is cleared and the context keeps working."""
import numpy as np
import pytest

from inputs import C1
from inputs.workloads import Level, Workload
from inputs.zeldovich import zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2512_12629_gb300 import cube2  # noqa: E402

# 8^3 IOS cells of 1 Mpc/h, one 16^3 mesh (half an IOS cell per mesh cell)
SMALL = Workload(name="err-8c-16mesh", n_p=8, box=8.0, n_ios=8, levels=(Level(16, 2.0),), b_pp=0.1)


def _stacked(n_part):
    """n_part particles at the centre of mesh cell (0, 0, 0): IOS cell 0,
    offsets 1/4 cell on every axis (mesh coordinate 1/2)."""
    off = np.full((3, n_part), 16384, dtype=np.uint16)
    count = np.zeros(SMALL.n_ios ** 3, dtype=np.int32)
    count[0] = n_part
    start = np.zeros_like(count)
    start[1:] = n_part
    return dict(off=off, count=count, start=start, vel=np.zeros((3, n_part), np.float32))


def test_capacity_word_at_2_to_the_64():
    ok = _stacked(65535)
    ctx = cube2.init_mesh(cube2.make_config(SMALL, n_particles=65535))
    acc = ctx.deposit_u64(0, cube2.IOSState.from_numpy(ok)).cpu().numpy().view(np.uint64).ravel()
    ctx.check()
    assert int(acc[0]) == 65535 << 48 and not acc[1:].any()
    ctx.close()
    bad = _stacked(65536)
    ctx = cube2.init_mesh(cube2.make_config(SMALL, n_particles=65536))
    ctx.deposit(0, cube2.IOSState.from_numpy(bad))
    with pytest.raises(cube2.Cube2Error) as e:
        ctx.check()
    assert e.value.code == cube2.ERR_CAPACITY
    ctx.check()                      # cleared
    ctx.close()


@pytest.fixture(scope="module")
def c1():
    st = zeldovich_ios(C1)
    ctx = cube2.init_mesh(cube2.make_config(C1))
    ctx.set_green(0)
    return st, ctx


def _step(ctx, st, mutate):
    p = cube2.IOSState.from_numpy(st)
    ctx.force(p)
    mutate(p)
    a = C1.scale_factors()
    ctx.kdk_step(p, a[0], a[1])
    return p


def test_nonfinite_word_on_a_nan_momentum(c1):
    st, ctx = c1

    def nan(p):
        p.vel[0, 5] = float("nan")
    _step(ctx, st, nan)
    with pytest.raises(cube2.Cube2Error) as e:
        ctx.check()
    assert e.value.code == cube2.ERR_NONFINITE
    _step(ctx, st, lambda p: None)
    ctx.check()


def test_displacement_word_on_an_oversized_momentum(c1):
    st, ctx = c1
    a = C1.scale_factors()
    _k1, dr, _k2 = cube2.kdk_factors(cube2.make_config(C1), a[0], a[1])
    # a momentum that drifts the particle by 0.6 of the box in this step
    v = 0.6 * C1.box / dr

    def big(p):
        p.vel[1, 7] = v
    _step(ctx, st, big)
    with pytest.raises(cube2.Cube2Error) as e:
        ctx.check()
    assert e.value.code == cube2.ERR_DISPLACEMENT
    # just below half the box is a legal (if absurd) drift
    def under(p):
        p.vel[1, 7] = 0.45 * C1.box / dr
    _step(ctx, st, under)
    ctx.check()
