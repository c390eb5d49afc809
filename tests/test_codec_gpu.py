"""FP16 velocity storage with a per-IOS-cell FP32 scale (Sec. 2.3 reading; the
large workload's velocity format) on the GPU against the oracle's codec.

* The codes and scales of the GPU encoder equal the oracle's bit for bit on
  the same FP32 momenta (the scale is a maximum, order-free; the code is one
  correctly rounded FP32 division and one binary16 rounding), and the decoder
  gives the oracle's FP32 values exactly.
* One KDK step with FP16 storage (decode in the kick, FP32 working copy
  through the re-bin and the second kick, encode at the end) against the
  oracle's FP64 step from the decoded initial momenta, encoded the same way:
  counts exact, offsets within one fixed-point unit, decoded momenta within
  one binary16 ulp of the cell scale plus the force bar.
* The stored velocity state is 6 bytes per particle plus 4 per IOS cell,
  against 12 bytes per particle in FP32."""
import numpy as np
import pytest

from inputs import C1, C2_SMALL
from inputs.zeldovich import zeldovich_ios

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import kdk as okdk  # noqa: E402
from oracle import mesh as omesh  # noqa: E402
from paper_2512_12629_gb300 import cube2  # noqa: E402


def _ctx(w):
    ctx = cube2.init_mesh(cube2.make_config(w.with_(vel_fp16=True)))
    for l in range(len(w.levels)):
        ctx.set_green(l)
    return ctx


@pytest.mark.parametrize("w", [C1, C2_SMALL.with_(displace_to_a=1.0)], ids=["C1", "C2_SMALL-z0"])
def test_codec_is_bit_exact_against_the_oracle(w):
    st = zeldovich_ios(w)
    ctx = _ctx(w)
    p = cube2.IOSState.from_numpy(st)
    v = torch.from_numpy(np.ascontiguousarray(st["vel"], dtype=np.float32)).cuda()
    ctx.vel_encode(p, v)
    back = ctx.vel_decode(p)
    ctx.check()
    codes, scale = okdk.encode_velocities(st["vel"], st["count"])
    assert np.array_equal(p.vscale.cpu().numpy().view(np.uint32), scale.view(np.uint32))
    assert np.array_equal(p.vel16.cpu().numpy().view(np.uint16), codes.view(np.uint16))
    ref = okdk.decode_velocities(codes, scale, st["count"])
    assert np.array_equal(back.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    n, c = st["off"].shape[1], st["count"].size
    print(f"{w.name}: stored velocity bytes {6 * n + 4 * c} vs FP32 {12 * n}; "
          f"max relative round-trip error {np.abs(ref - st['vel']).max() / np.abs(st['vel']).max():.2e}")
    ctx.close()


def test_kdk_step_with_fp16_storage_matches_oracle():
    w = C1
    st = zeldovich_ios(w)
    greens = omesh.green_tables(w)
    ctx = _ctx(w)
    p = cube2.IOSState.from_numpy(st)
    ctx.vel_encode(p, torch.from_numpy(np.ascontiguousarray(st["vel"], dtype=np.float32)).cuda())
    a = w.scale_factors()
    ctx.force(p)
    ctx.kdk_step(p, a[0], a[1])
    ctx.check()
    got_v = ctx.vel_decode(p).cpu().numpy().astype(np.float64)
    got = p.to_numpy()
    codes0, scale0 = okdk.encode_velocities(st["vel"], st["count"])
    v0 = okdk.decode_velocities(codes0, scale0, st["count"]).astype(np.float64)
    ref = okdk.kdk_step(dict(off=st["off"], count=st["count"], start=st["start"], vel=v0, acc=None), w, a[0], a[1],
                        greens)
    assert np.array_equal(got["count"], ref["count"])
    d = np.abs(got["off"].astype(np.int64) - ref["off"].astype(np.int64))
    d = np.minimum(d, 65536 - d)
    assert d.max() <= 1 and np.mean(d == 0) >= 0.99
    codes1, scale1 = okdk.encode_velocities(ref["vel"], ref["count"])
    ref_v = okdk.decode_velocities(codes1, scale1, ref["count"]).astype(np.float64)
    cell = np.repeat(np.arange(ref["count"].size), ref["count"])
    # beyond one binary16 ulp of the cell scale (codes of values that straddle
    # a rounding boundary), the difference is the force bar's
    quant = 2.0 ** -10 * scale1[cell].astype(np.float64)
    resid = np.maximum(np.abs(got_v - ref_v) - quant[None, :], 0.0)
    vnorm = np.linalg.norm(ref_v, axis=0)
    rel = np.linalg.norm(resid, axis=0) / np.maximum(vnorm, 1e-3 * np.sqrt(np.mean(vnorm ** 2)))
    print(f"FP16 step: decoded momenta beyond the quantisation: median {np.median(rel):.2e}, "
          f"p99.9 {np.quantile(rel, 0.999):.2e}")
    assert np.median(rel) <= 1e-5 and np.quantile(rel, 0.999) <= 1e-3
    # the GPU's stored scales are those of its own working momenta: within FP32 reach of the oracle's
    gs = p.vscale.cpu().numpy().astype(np.float64)
    assert np.allclose(gs, scale1, rtol=1e-4, atol=0)
    ctx.close()
