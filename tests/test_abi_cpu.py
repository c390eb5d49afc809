"""CPU-only checks of the C-ABI library: it loads, exports every declared symbol,
validates configs on the host, and its host-side KDK factors match the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cube2.h")


@pytest.fixture(scope="module")
def binding():
    from paper_2512_12629_gb300 import build
    build.build()
    from paper_2512_12629_gb300 import cube2
    return cube2


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cube2_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(binding):
    names = declared_functions()
    assert len(names) >= 18
    lib = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_structs_match_header_layout(binding, tmp_path):
    # compile a probe against the header with the host C compiler and compare
    # sizeof/offsetof with the ctypes mirrors
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "probe.c"
    fields = {"cube2_config": [f for f, _ in binding.Config._fields_],
              "cube2_particles": [f for f, _ in binding.Particles._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cube2.h"', "int main(void){"]
    for st, fl in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({st}));')
        lines += [f'printf("%zu\\n", offsetof({st}, {f}));' for f in fl]
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = []
    for cls in (binding.Config, binding.Particles):
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert got == want


@pytest.mark.parametrize("field,value,code", [
    ("n_ios", 2, -1), ("n_levels", 3, -1), ("b_pp", 0.0, -1),
])
def test_init_mesh_rejects_bad_config_on_host(binding, field, value, code):
    from inputs import C1
    cfg = binding.make_config(C1)
    setattr(cfg, field, value)
    ptr = ctypes.c_void_p()
    assert binding.library().cube2_init_mesh(ctypes.byref(ptr), ctypes.byref(cfg), None) == code
    assert binding.library().cube2_last_error(None)


def test_init_mesh_rejects_unsupported_meshes(binding):
    from inputs import C1
    lib = binding.library()
    for n_mesh, n_ios in ((80, 32), (64, 8), (100, 50)):   # 5 | 80; ratio 8; 5^2 | 100
        cfg = binding.make_config(C1)
        cfg.n_mesh[0] = n_mesh
        cfg.n_ios = n_ios
        ptr = ctypes.c_void_p()
        assert lib.cube2_init_mesh(ctypes.byref(ptr), ctypes.byref(cfg), None) == -6
    cfg = binding.make_config(C1)
    cfg.beta[0] = 3.0            # PP range 3 Mpc/h > IOS cell 2 Mpc/h
    assert lib.cube2_init_mesh(ctypes.byref(ctypes.c_void_p()), ctypes.byref(cfg), None) == -1


def test_kdk_factors_match_oracle(binding):
    from inputs import C2
    from oracle import kdk as okdk
    cfg = binding.make_config(C2)
    a = C2.scale_factors()
    for i in (0, 17, 49):
        k1, dr, k2 = binding.kdk_factors(cfg, a[i], a[i + 1])
        ah = 0.5 * (a[i] + a[i + 1])
        assert k1 == pytest.approx(okdk.kick_integral(a[i], ah, 0.3, 0.7), rel=1e-13)
        assert dr == pytest.approx(okdk.drift_integral(a[i], a[i + 1], 0.3, 0.7), rel=1e-13)
        assert k2 == pytest.approx(okdk.kick_integral(ah, a[i + 1], 0.3, 0.7), rel=1e-13)


def test_third_level_config_is_validated_on_host(binding):
    from inputs import C2_SMALL
    from inputs.workloads import Level, PM3Spec, Workload
    lib = binding.library()
    small = Workload(name="pm3-8c-8x32mesh", n_p=10, box=32.0, n_ios=8, levels=(Level(8, 3.5), Level(32, 3.5)),
                     b_pp=0.3)
    # refinement not a power of two, tile not dividing n_ios, b_3 beyond the PP range, no capacity
    for field, value in (("pm3_refine", 3), ("pm3_tile", 3), ("pm3_beta", 28.0), ("pm3_max_tiles", 0)):
        cfg = binding.make_config(small.with_(pm3=PM3Spec(2, 2, 3.5, 2, 8)), n_particles=1000)
        setattr(cfg, field, value)
        ptr = ctypes.c_void_p()
        assert lib.cube2_init_mesh(ctypes.byref(ptr), ctypes.byref(cfg), None) == -1, field
    # a local mesh the FFT passes do not take: 16^3 IOS-cell subtiles need 64 + 2 x 8 cells -> 81 = 3^4
    cfg = binding.make_config(C2_SMALL.with_(pm3=PM3Spec(16, 2, 2.0, 2, 8)))
    assert lib.cube2_init_mesh(ctypes.byref(ctypes.c_void_p()), ctypes.byref(cfg), None) == -6
    # TSC with the third level
    cfg = binding.make_config(small.with_(pm3=PM3Spec(2, 2, 3.5, 2, 8), assign_order=3), n_particles=1000)
    assert lib.cube2_init_mesh(ctypes.byref(ctypes.c_void_p()), ctypes.byref(cfg), None) == -1
