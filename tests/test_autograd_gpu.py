"""Differentiation through torch.autograd (cube2.FinalDensity) and the IOS
placement it starts from (cube2_ios_from_positions), through the C ABI:

1. placement of arbitrary positions (inside and outside the box) into IOS is
   bit-exact against the input generator's quantiser (offsets, counts,
   starts and the stable order, ties in input order), momenta permuted along;
2. the autograd gradient of a density loss with respect to the initial
   positions and momenta equals the adjoint sweep's (cube2.loss_gradient,
   itself checked against the FP64 oracle in test_adjoint_gpu) put back into
   the input order, to FP32 rounding of the cotangent;
3. the chain to the Zel'dovich displacement field psi (x0 = q + D psi,
   p0 = a^2 E f D psi) through torch: dL/dpsi = D dL/dx0 + a^2 E f D dL/dp0."""
import numpy as np
import pytest

from inputs import C1
from inputs.zeldovich import gaussian_displacement, growth_d, growth_f, hubble_e, quantise_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2512_12629_gb300 import cube2  # noqa: E402

# C1's box and mesh, three steps z = 9 -> 4 (past the linear regime's start)
W = C1.with_(z_init=9.0, z_final=4.0, n_steps=3)


@pytest.fixture(scope="module")
def ctx():
    c = cube2.init_mesh(cube2.make_config(W))
    c.set_green(0)
    c.adjoint_init()
    yield c
    c.close()


def _lagrangian(w):
    n, box = w.n_p, w.box
    psi = gaussian_displacement(n, box, w.omega_m, w.h, w.sigma8, w.seed).reshape(3, -1)
    g = (np.arange(n) + 0.5) * (box / n)
    q = np.stack(np.meshgrid(g, g, g, indexing="ij")[::-1]).reshape(3, -1)
    a = w.a_init
    d = growth_d(a, w.omega_m, w.omega_l)
    c = a ** 2 * float(hubble_e(a, w.omega_m, w.omega_l)) * growth_f(a, w.omega_m, w.omega_l) * d
    return q, psi, d, c


def test_placement_matches_the_quantiser(ctx):
    rng = np.random.Generator(np.random.Philox(71))
    n = W.n_particles
    pos = rng.uniform(-W.box, 2.0 * W.box, size=(3, n))
    pos[:, :200] = np.floor(pos[:, :200])          # exact cell edges and ties
    mom = rng.normal(0.0, 3.0, size=(3, n)).astype(np.float32)
    st = quantise_ios(pos, W.n_ios, W.box)
    p, perm = ctx.ios_from_positions(torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda())
    ctx.check()
    np.testing.assert_array_equal(p.off.cpu().numpy().view(np.uint16), st["off"])
    np.testing.assert_array_equal(p.count.cpu().numpy(), st["count"])
    np.testing.assert_array_equal(p.start.cpu().numpy(), st["start"])
    np.testing.assert_array_equal(perm.cpu().numpy(), st["perm"])
    np.testing.assert_array_equal(p.vel.cpu().numpy(), mom[:, st["perm"]])


def test_autograd_gradient_equals_the_adjoint_sweep(ctx):
    q, psi, d, c = _lagrangian(W)
    a = W.scale_factors()
    gen = torch.Generator(device="cuda").manual_seed(5)
    target = torch.randn((64, 64, 64), device="cuda", generator=gen) * 0.5
    x0 = torch.tensor(q + d * psi, device="cuda", requires_grad=True)
    v0 = torch.tensor((c * psi).astype(np.float32), device="cuda", requires_grad=True)
    delta = cube2.final_density(ctx, x0, v0, a)
    loss = ((delta - target) ** 2).mean()
    loss.backward()
    ctx.check()
    # the same through the adjoint sweep, in IOS order, mapped back
    p0, perm = ctx.ios_from_positions(x0.detach(), v0.detach())
    ctx.force(p0)
    l_ref, gx, gv = cube2.loss_gradient(ctx, p0, target, a)
    idx = perm.long()
    gx_in = torch.zeros_like(x0)
    gv_in = torch.zeros_like(v0)
    gx_in[:, idx] = gx.double()
    gv_in[:, idx] = gv
    assert float(loss.detach()) == pytest.approx(l_ref, rel=1e-6)
    for got, ref in ((x0.grad, gx_in), (v0.grad, gv_in)):
        err = (got.double() - ref.double()).norm() / ref.double().norm()
        assert float(err) < 1e-5, float(err)
    assert float(x0.grad.abs().max()) > 0 and float(v0.grad.abs().max()) > 0


def test_displacement_field_gradient(ctx):
    q, psi_np, d, c = _lagrangian(W)
    a = W.scale_factors()
    gen = torch.Generator(device="cuda").manual_seed(6)
    target = torch.randn((64, 64, 64), device="cuda", generator=gen) * 0.5
    qt = torch.tensor(q, device="cuda")
    psi = torch.tensor(psi_np, device="cuda", requires_grad=True)
    x0 = qt + d * psi
    v0 = (c * psi).float()
    loss = ((cube2.final_density(ctx, x0, v0, a) - target) ** 2).mean()
    (g_psi,) = torch.autograd.grad(loss, psi)
    # the two leaves separately, composed by hand
    x0l = (qt + d * psi.detach()).requires_grad_(True)
    v0l = (c * psi.detach()).float().requires_grad_(True)
    loss2 = ((cube2.final_density(ctx, x0l, v0l, a) - target) ** 2).mean()
    gx, gv = torch.autograd.grad(loss2, (x0l, v0l))
    ref = d * gx + c * gv.double()
    err = (g_psi - ref).norm() / ref.norm()
    assert float(err) < 1e-6, float(err)
    ctx.check()
