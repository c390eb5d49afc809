"""Python binding of libcube2gb (include/cube2.h): argument marshalling only.

Every function forwards to the C entry point of the same name
(``cube2_<name>``); all arithmetic runs in the library's CUDA kernels.  Torch
tensors own the device memory of the particle arrays and give the stream.
There is no CPU fallback: importing this module without the built library,
or calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcube2gb.so")

OK = 0
ERR_BAD_ARG = -1
ERR_CUDA = -2
ERR_CAPACITY = -3
ERR_TIMEOUT = -4
ERR_NONFINITE = -5
ERR_UNSUPPORTED_SIZE = -6
ERR_STATE = -7
ERR_DISPLACEMENT = -8
MAX_LEVELS = 2
PROFILE_CLASSES = 27
LEVEL_PM3 = 2


class Cube2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cube2 error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double),
        ("n_ios", ctypes.c_int32),
        ("n_levels", ctypes.c_int32),
        ("n_mesh", ctypes.c_int32 * MAX_LEVELS),
        ("beta", ctypes.c_double * MAX_LEVELS),
        ("b_pp", ctypes.c_double),
        ("omega_m", ctypes.c_double),
        ("omega_l", ctypes.c_double),
        ("n_particles", ctypes.c_int64),
        ("alias_max", ctypes.c_int32),
        ("assign_order", ctypes.c_int32),
        ("iso_length", ctypes.c_double),
        ("pm3_tile", ctypes.c_int32),
        ("pm3_refine", ctypes.c_int32),
        ("pm3_beta", ctypes.c_double),
        ("pm3_rho_min", ctypes.c_int32),
        ("pm3_max_tiles", ctypes.c_int32),
        ("vel_fp16", ctypes.c_int32),
    ]


class EnsembleOpts(ctypes.Structure):
    _fields_ = [
        ("n_streams", ctypes.c_int32),
        ("persistent_pp", ctypes.c_int32),
        ("pp_ctas_per_sm", ctypes.c_int32),
        ("pp_wmax", ctypes.c_int32),
        ("timeout_ms", ctypes.c_double),
    ]


def ensemble_opts(n_streams=16, persistent_pp=False, pp_ctas_per_sm=16, pp_wmax=0, timeout_ms=1000.0):
    return EnsembleOpts(int(n_streams), int(bool(persistent_pp)), int(pp_ctas_per_sm), int(pp_wmax), float(timeout_ms))


class Particles(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("off", ctypes.c_void_p * 3),
        ("count", ctypes.c_void_p),
        ("start", ctypes.c_void_p),
        ("vel", ctypes.c_void_p * 3),
        ("acc", ctypes.c_void_p * 3),
        ("vel16", ctypes.c_void_p * 3),
        ("vscale", ctypes.c_void_p),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2512_12629_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "cube2_init_mesh": (I, [ctypes.POINTER(P), ctypes.POINTER(Config), P]),
        "cube2_set_green": (I, [P, I, ctypes.c_char_p]),
        "cube2_deposit": (I, [P, I, ctypes.POINTER(Particles)]),
        "cube2_deposit_u64": (I, [P, I, ctypes.POINTER(Particles), P]),
        "cube2_solve_pm": (I, [P, I]),
        "cube2_interp_force": (I, [P, I, ctypes.POINTER(Particles), I]),
        "cube2_pp_force": (I, [P, ctypes.POINTER(Particles), I]),
        "cube2_force": (I, [P, ctypes.POINTER(Particles)]),
        "cube2_kdk_step": (I, [P, ctypes.POINTER(Particles), D, D]),
        "cube2_ios_from_positions": (I, [P, P, P, ctypes.POINTER(Particles), P]),
        "cube2_kdk_step_host": (I, [P, ctypes.POINTER(Particles), ctypes.POINTER(Particles), D, D]),
        "cube2_get_density": (I, [P, I, P]),
        "cube2_get_potential": (I, [P, I, P]),
        "cube2_get_green": (I, [P, I, P]),
        "cube2_debug_forward_fft": (I, [P, I, P]),
        "cube2_kdk_factors": (I, [ctypes.POINTER(Config), D, D, ctypes.POINTER(D)]),
        "cube2_check": (I, [P]),
        "cube2_last_error": (ctypes.c_char_p, [P]),
        "cube2_launch_count": (ctypes.c_int64, [P]),
        "cube2_profile": (I, [P, I]),
        "cube2_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_int64)]),
        "cube2_profile_class_name": (ctypes.c_char_p, [I]),
        "cube2_pp_stats": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "cube2_pp_count": (I, [P, ctypes.c_int]),
        "cube2_pp_stats_paths": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "cube2_solve_pm_noalloc": (I, [P, P, P, ctypes.c_int32, P]),
        "cube2_fma_probe": (I, [P, I, I, I, P]),
        "cube2_pm3_info": (I, [P, ctypes.POINTER(D)]),
        "cube2_pm3_stats": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "cube2_pm3_map": (I, [P, P]),
        "cube2_vel_encode": (I, [P, ctypes.POINTER(Particles), P]),
        "cube2_vel_decode": (I, [P, ctypes.POINTER(Particles), P]),
        "cube2_adjoint_init": (I, [P]),
        "cube2_force_vjp": (I, [P, ctypes.POINTER(Particles), P, P]),
        "cube2_kdk_permutation": (I, [P, P]),
        "cube2_density_mse_vjp": (I, [P, I, ctypes.POINTER(Particles), P, P, ctypes.POINTER(D)]),
        "cube2_density_vjp": (I, [P, I, ctypes.POINTER(Particles), P, P]),
        "cube2_kdk_adjoint_step": (I, [P, ctypes.POINTER(Particles), ctypes.POINTER(Particles), P, P, P, D, D]),
        "cube2_kdk_adjoint": (I, [P, P, P, I, ctypes.POINTER(D), P, P]),
        "cube2_lpt_partition": (I, [ctypes.POINTER(D), I, I, ctypes.POINTER(I)]),
        "cube2_config_cost": (I, [ctypes.POINTER(Config), ctypes.POINTER(D)]),
        "cube2_ensemble_create": (I, [ctypes.POINTER(P), P, P, I, ctypes.POINTER(D), I, I]),
        "cube2_ensemble_launch": (I, [P, P]),
        "cube2_ensemble_create_ex": (I, [ctypes.POINTER(P), P, P, I, ctypes.POINTER(D), I, ctypes.POINTER(EnsembleOpts)]),
        "cube2_ensemble_check": (I, [P, P]),
        "cube2_ensemble_publish": (I, [P, I]),
        "cube2_ensemble_autotune": (I, [P, P, I, ctypes.POINTER(D), I, I, P, ctypes.POINTER(EnsembleOpts),
                                        ctypes.POINTER(D)]),
        "cube2_ensemble_info": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "cube2_ensemble_destroy": (None, [P]),
        "cube2_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def library():
    return _lib


def make_config(w, n_particles=None, alias_max=2) -> Config:
    """Config from an ``inputs.workloads.Workload`` record."""
    c = Config()
    c.box = w.box
    c.n_ios = w.n_ios
    c.n_levels = len(w.levels)
    for i, lev in enumerate(w.levels):
        c.n_mesh[i] = lev.n_mesh
        c.beta[i] = lev.beta
    c.b_pp = w.b_pp
    c.omega_m = w.omega_m
    c.omega_l = w.omega_l
    c.n_particles = w.n_particles if n_particles is None else n_particles
    c.alias_max = alias_max
    c.assign_order = getattr(w, "assign_order", 2)
    c.iso_length = getattr(w, "iso_length", 0.0)
    c.vel_fp16 = 1 if getattr(w, "vel_fp16", False) else 0
    pm3 = getattr(w, "pm3", None)
    if pm3 is not None:
        c.pm3_tile, c.pm3_refine, c.pm3_beta = pm3.tile, pm3.refine, pm3.beta
        c.pm3_rho_min, c.pm3_max_tiles = pm3.rho_min, pm3.max_tiles
    return c


@dataclass
class IOSState:
    """Particle set in IOS form as torch tensors (device or pinned host).

    vel16 / vscale (optional): FP16 velocity storage for contexts made with
    vel_fp16 (then ``vel`` is unused and may be a placeholder)."""
    off: torch.Tensor     # (3, N) int16 storage of the uint16 offsets
    count: torch.Tensor   # (n_ios^3,) int32
    start: torch.Tensor   # (n_ios^3,) int32
    vel: torch.Tensor     # (3, N) float32
    acc: torch.Tensor     # (3, N) float32
    vel16: torch.Tensor = None   # (3, N) int16 storage of IEEE binary16 codes
    vscale: torch.Tensor = None  # (n_ios^3,) float32 per-cell scale

    @property
    def n(self):
        return self.off.shape[1]

    @staticmethod
    def from_numpy(st, device="cuda", pin=False):
        def t(a, dtype=None):
            x = torch.from_numpy(np.ascontiguousarray(a))
            if dtype is not None:
                x = x.to(dtype)
            if device == "cpu":
                return x.pin_memory() if pin else x
            return x.to(device)
        off = np.ascontiguousarray(st["off"]).view(np.int16)
        n = off.shape[1]
        vel = st.get("vel")
        vel = np.zeros((3, n), np.float32) if vel is None else np.asarray(vel, np.float32)
        acc = np.zeros((3, n), np.float32)
        return IOSState(t(off), t(st["count"].astype(np.int32)), t(st["start"].astype(np.int32)),
                        t(vel), t(acc))

    def to_numpy(self):
        return dict(off=self.off.cpu().numpy().view(np.uint16), count=self.count.cpu().numpy(),
                    start=self.start.cpu().numpy(), vel=self.vel.cpu().numpy(), acc=self.acc.cpu().numpy())

    def clone(self):
        extra = (None, None) if self.vel16 is None else (self.vel16.clone(), self.vscale.clone())
        return IOSState(*(x.clone() for x in (self.off, self.count, self.start, self.vel, self.acc)), *extra)

    def struct(self) -> Particles:
        p = Particles()
        p.n = self.n
        for d in range(3):
            p.off[d] = self.off[d].data_ptr()
            p.vel[d] = self.vel[d].data_ptr()
            p.acc[d] = self.acc[d].data_ptr()
        p.count = self.count.data_ptr()
        p.start = self.start.data_ptr()
        if self.vel16 is not None:
            for d in range(3):
                p.vel16[d] = self.vel16[d].data_ptr()
            p.vscale = self.vscale.data_ptr()
        return p


class Context:
    """Owner of a cube2_ctx (meshes, Green's tables, scratch) on one device/stream."""

    def __init__(self, cfg: Config, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("cube2 needs a CUDA device (no CPU fallback)")
        self.cfg = cfg
        self.stream = torch.cuda.current_stream() if stream is None else stream
        ptr = ctypes.c_void_p()
        code = _lib.cube2_init_mesh(ctypes.byref(ptr), ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream))
        if code != OK:
            raise Cube2Error(code, _lib.cube2_last_error(None).decode())
        self.ptr = ptr

    def _chk(self, code):
        if code != OK:
            raise Cube2Error(code, _lib.cube2_last_error(self.ptr).decode())

    def close(self):
        if getattr(self, "ptr", None):
            _lib.cube2_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # same names as the C ABI ------------------------------------------------
    def set_green(self, level, cache_path=None):
        self._chk(_lib.cube2_set_green(self.ptr, level, cache_path.encode() if cache_path else None))

    def deposit(self, level, p: IOSState):
        self._chk(_lib.cube2_deposit(self.ptr, level, ctypes.byref(p.struct())))

    def deposit_u64(self, level, p: IOSState):
        n = self.cfg.n_mesh[level]
        out = torch.empty((n, n, n), dtype=torch.int64, device=p.off.device)
        self._chk(_lib.cube2_deposit_u64(self.ptr, level, ctypes.byref(p.struct()), out.data_ptr()))
        return out

    def solve_pm(self, level):
        self._chk(_lib.cube2_solve_pm(self.ptr, level))

    def interp_force(self, level, p: IOSState, accumulate=False):
        self._chk(_lib.cube2_interp_force(self.ptr, level, ctypes.byref(p.struct()), int(accumulate)))

    def pp_force(self, p: IOSState, accumulate=False):
        self._chk(_lib.cube2_pp_force(self.ptr, ctypes.byref(p.struct()), int(accumulate)))

    def force(self, p: IOSState):
        self._chk(_lib.cube2_force(self.ptr, ctypes.byref(p.struct())))

    def adjoint_init(self):
        self._chk(_lib.cube2_adjoint_init(self.ptr))

    def force_vjp(self, p: IOSState, v: torch.Tensor, out: torch.Tensor = None):
        """w = d<v, F>/dx for a cotangent v (3, N) FP32 on the device; returns w (3, N)."""
        if out is None:
            out = torch.empty_like(v)
        vp = (ctypes.c_void_p * 3)(*[v[d].data_ptr() for d in range(3)])
        wp = (ctypes.c_void_p * 3)(*[out[d].data_ptr() for d in range(3)])
        self._chk(_lib.cube2_force_vjp(self.ptr, ctypes.byref(p.struct()), vp, wp))
        return out

    def kdk_permutation(self, out: torch.Tensor = None):
        """Map of the last re-bin: out[new] = old index (int32, device)."""
        if out is None:
            out = torch.empty(self.cfg.n_particles, dtype=torch.int32, device="cuda")
        self._chk(_lib.cube2_kdk_permutation(self.ptr, out.data_ptr()))
        return out

    def density_mse_vjp(self, level, p: IOSState, target: torch.Tensor, out: torch.Tensor = None):
        """(L, dL/dx) for L = mean((delta - target)^2) on `level`; dL/dx (3, N) FP32."""
        if out is None:
            out = torch.empty_like(p.vel)
        wp = (ctypes.c_void_p * 3)(*[out[d].data_ptr() for d in range(3)])
        loss = ctypes.c_double()
        self._chk(_lib.cube2_density_mse_vjp(self.ptr, int(level), ctypes.byref(p.struct()), target.data_ptr(), wp,
                                             ctypes.byref(loss)))
        return loss.value, out

    def density_vjp(self, level, p: IOSState, g: torch.Tensor, out: torch.Tensor = None):
        """d<g, delta>/dx (3, N) FP32 for a cotangent g ([n][n][n] FP32, device) on the level's overdensity."""
        if out is None:
            out = torch.empty((3, p.n), dtype=torch.float32, device=p.off.device)
        g = g.contiguous()
        wp = (ctypes.c_void_p * 3)(*[out[d].data_ptr() for d in range(3)])
        self._chk(_lib.cube2_density_vjp(self.ptr, int(level), ctypes.byref(p.struct()), g.data_ptr(), wp))
        return out

    def kdk_adjoint_step(self, pre: IOSState, post: IOSState, perm: torch.Tensor, xbar: torch.Tensor,
                         pbar: torch.Tensor, a0, a1):
        """Reverse of kdk_step(a0, a1): xbar, pbar (3, N) are updated in place."""
        xp = (ctypes.c_void_p * 3)(*[xbar[d].data_ptr() for d in range(3)])
        pp = (ctypes.c_void_p * 3)(*[pbar[d].data_ptr() for d in range(3)])
        self._chk(_lib.cube2_kdk_adjoint_step(self.ptr, ctypes.byref(pre.struct()), ctypes.byref(post.struct()),
                                              perm.data_ptr(), xp, pp, float(a0), float(a1)))

    def kdk_adjoint(self, states, perms, a, xbar: torch.Tensor, pbar: torch.Tensor):
        """Reverse of len(a) - 1 KDK steps (cube2_kdk_adjoint); xbar, pbar updated in place."""
        n = len(a) - 1
        structs = [st.struct() for st in states]
        sp = (ctypes.c_void_p * (n + 1))(*[ctypes.addressof(x) for x in structs])
        pp = (ctypes.c_void_p * n)(*[q.data_ptr() for q in perms])
        av = np.ascontiguousarray(a, dtype=np.float64)
        xp = (ctypes.c_void_p * 3)(*[xbar[d].data_ptr() for d in range(3)])
        bp = (ctypes.c_void_p * 3)(*[pbar[d].data_ptr() for d in range(3)])
        self._chk(_lib.cube2_kdk_adjoint(self.ptr, sp, pp, n, av.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         xp, bp))

    def kdk_step(self, p: IOSState, a0, a1):
        self._chk(_lib.cube2_kdk_step(self.ptr, ctypes.byref(p.struct()), float(a0), float(a1)))

    def ios_from_positions(self, pos: torch.Tensor, mom: torch.Tensor = None, out: IOSState = None,
                           perm: torch.Tensor = None):
        """IOS state of positions pos (3, N) FP64 [Mpc/h] and momenta mom (3, N)
        FP32 (None: zero), on the device: (state, perm) with perm[j] (int32) the
        input index of IOS slot j; the state's acc is zero."""
        n, nc = int(self.cfg.n_particles), int(self.cfg.n_ios) ** 3
        if pos.dtype != torch.float64 or pos.shape != (3, n) or not pos.is_cuda:
            raise ValueError("pos must be a (3, N) float64 CUDA tensor")
        pos = pos.contiguous()
        if mom is not None:
            if mom.dtype != torch.float32 or mom.shape != (3, n) or not mom.is_cuda:
                raise ValueError("mom must be a (3, N) float32 CUDA tensor")
            mom = mom.contiguous()
        if out is None:
            dev = pos.device
            out = IOSState(torch.empty((3, n), dtype=torch.int16, device=dev), torch.empty(nc, dtype=torch.int32, device=dev),
                           torch.empty(nc, dtype=torch.int32, device=dev), torch.empty((3, n), dtype=torch.float32, device=dev),
                           torch.zeros((3, n), dtype=torch.float32, device=dev))
        if perm is None:
            perm = torch.empty(n, dtype=torch.int32, device=pos.device)
        pp = (ctypes.c_void_p * 3)(*[pos[d].data_ptr() for d in range(3)])
        mp = None if mom is None else (ctypes.c_void_p * 3)(*[mom[d].data_ptr() for d in range(3)])
        self._chk(_lib.cube2_ios_from_positions(self.ptr, pp, mp, ctypes.byref(out.struct()), perm.data_ptr()))
        return out, perm

    def kdk_step_host(self, dev: IOSState, host: IOSState, a0, a1):
        self._chk(_lib.cube2_kdk_step_host(self.ptr, ctypes.byref(dev.struct()), ctypes.byref(host.struct()),
                                           float(a0), float(a1)))

    def _grid(self, fn, level, shape, dtype, device):
        out = torch.empty(shape, dtype=dtype, device=device)
        self._chk(fn(self.ptr, level, out.data_ptr()))
        return out

    def get_density(self, level, device="cuda"):
        n = self.cfg.n_mesh[level]
        return self._grid(_lib.cube2_get_density, level, (n, n, n), torch.float32, device)

    def get_potential(self, level, device="cuda"):
        n = self.cfg.n_mesh[level]
        return self._grid(_lib.cube2_get_potential, level, (n, n, n), torch.float32, device)

    def get_green(self, level, device="cuda"):
        n = self.pm3_info()["m"] if level == LEVEL_PM3 else self.cfg.n_mesh[level]
        return self._grid(_lib.cube2_get_green, level, (n, n, n // 2 + 1), torch.float32, device)

    def debug_forward_fft(self, level, device="cuda"):
        n = self.cfg.n_mesh[level]
        out = self._grid(_lib.cube2_debug_forward_fft, level, (n, n, n // 2 + 1, 2), torch.float32, device)
        return torch.view_as_complex(out)

    def check(self):
        self._chk(_lib.cube2_check(self.ptr))

    def vel_encode(self, p: IOSState, v: torch.Tensor):
        """Fill p.vel16 / p.vscale (allocated here if absent) from FP32 momenta v (3, N)."""
        if p.vel16 is None:
            p.vel16 = torch.empty(p.off.shape, dtype=torch.int16, device=p.off.device)
            p.vscale = torch.empty(p.count.shape, dtype=torch.float32, device=p.off.device)
        vp = (ctypes.c_void_p * 3)(*[v[d].data_ptr() for d in range(3)])
        self._chk(_lib.cube2_vel_encode(self.ptr, ctypes.byref(p.struct()), vp))
        return p

    def vel_decode(self, p: IOSState, out: torch.Tensor = None):
        """FP32 momenta (3, N) = half(p.vel16) * p.vscale of each particle's cell."""
        if out is None:
            out = torch.empty(p.off.shape, dtype=torch.float32, device=p.off.device)
        vp = (ctypes.c_void_p * 3)(*[out[d].data_ptr() for d in range(3)])
        self._chk(_lib.cube2_vel_decode(self.ptr, ctypes.byref(p.struct()), vp))
        return out

    def pm3_info(self):
        """Geometry of the adaptive third level: dict(tile, ns, refine, B, m, H3, b3, max_tiles)."""
        out = (ctypes.c_double * 8)()
        self._chk(_lib.cube2_pm3_info(self.ptr, out))
        keys = ("tile", "ns", "refine", "B", "m", "H3", "b3", "max_tiles")
        return {k: (out[i] if k in ("H3", "b3") else int(out[i])) for i, k in enumerate(keys)}

    def pm3_stats(self):
        """(local meshes in use, subtiles that asked for refinement) of the last force/PP call."""
        out = (ctypes.c_int64 * 2)()
        self._chk(_lib.cube2_pm3_stats(self.ptr, out))
        return int(out[0]), int(out[1])

    def pm3_map(self):
        """Local mesh index of every subtile (device int32, -1 = unrefined) of the last force/PP call."""
        ns = self.pm3_info()["ns"]
        out = torch.empty(ns ** 3, dtype=torch.int32, device="cuda")
        self._chk(_lib.cube2_pm3_map(self.ptr, out.data_ptr()))
        return out

    def launch_count(self):
        return int(_lib.cube2_launch_count(self.ptr))

    def pp_count(self, on=True):
        """Switch the PP work counters on (or off, the default) for later PP evaluations."""
        self._chk(_lib.cube2_pp_count(self.ptr, int(bool(on))))

    def pp_stats(self):
        """(in-range ordered pairs, candidate pairs) counted since the last call (see pp_count)."""
        out = (ctypes.c_int64 * 2)()
        self._chk(_lib.cube2_pp_stats(self.ptr, out))
        return int(out[0]), int(out[1])

    def pp_stats_paths(self):
        """(pairs, candidates) of all targets and of the per-lane path, since the last call."""
        out = (ctypes.c_int64 * 4)()
        self._chk(_lib.cube2_pp_stats_paths(self.ptr, out))
        return tuple(int(v) for v in out)

    def profile(self, capacity):
        """Start (capacity > 0) or stop (0) per-kernel-class CUDA-event timing."""
        self._chk(_lib.cube2_profile(self.ptr, int(capacity)))

    def profile_read(self):
        """{(class_name, level): (milliseconds, launch_groups)} since the last read."""
        n = PROFILE_CLASSES * MAX_LEVELS
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self._chk(_lib.cube2_profile_read(self.ptr, ms, cnt))
        out = {}
        for c in range(PROFILE_CLASSES):
            name = _lib.cube2_profile_class_name(c).decode()
            for l in range(MAX_LEVELS):
                k = c * MAX_LEVELS + l
                if cnt[k]:
                    out[(name, l)] = (ms[k], int(cnt[k]))
        return out


def solve_pm_noalloc(rho: torch.Tensor, green: torch.Tensor, phi: torch.Tensor, stream=None):
    """Context-free Poisson solve that allocates no device memory.

    For callers that cannot allocate where they need a solve; the library keeps
    its working memory in a fixed device array (meshes up to 128^3).  rho and
    phi are contiguous FP32 [n][n][n], green the contiguous FP32 [n][n][n/2+1]
    table of ``get_green``, all on one CUDA device; the call runs on that
    device's current stream (or ``stream``).  Raises ValueError before calling
    into the library when a tensor does not match."""
    if rho.dim() != 3 or len(set(rho.shape)) != 1:
        raise ValueError("rho must be an (n, n, n) tensor")
    n = int(rho.shape[0])
    for name, t, shape in (("rho", rho, (n, n, n)), ("phi", phi, (n, n, n)), ("green", green, (n, n, n // 2 + 1))):
        if t.dtype != torch.float32 or tuple(t.shape) != shape or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape {shape}")
    if not (rho.device == phi.device == green.device):
        raise ValueError("rho, green and phi must be on one device")
    with torch.cuda.device(rho.device):
        st = torch.cuda.current_stream(rho.device) if stream is None else stream
        code = _lib.cube2_solve_pm_noalloc(rho.data_ptr(), green.data_ptr(), phi.data_ptr(), n,
                                           ctypes.c_void_p(st.cuda_stream))
    if code != OK:
        raise Cube2Error(code, _lib.cube2_last_error(None).decode())


def fma_probe(out: torch.Tensor, blocks, threads, iters, stream=None):
    """Launch the FP32 FMA probe (cube2_fma_probe) on ``stream``; returns the
    FP32 operations it performs (2 * 8 * 16 * iters * blocks * threads)."""
    st = torch.cuda.current_stream() if stream is None else stream
    code = _lib.cube2_fma_probe(out.data_ptr(), int(blocks), int(threads), int(iters), ctypes.c_void_p(st.cuda_stream))
    if code != OK:
        raise Cube2Error(code, "fma_probe")
    return 2 * 8 * 16 * int(iters) * int(blocks) * int(threads)


def config_cost(cfg: Config):
    """Work estimate of one KDK step of a box (cube2_config_cost); host only."""
    out = ctypes.c_double()
    code = _lib.cube2_config_cost(ctypes.byref(cfg), ctypes.byref(out))
    if code != OK:
        raise Cube2Error(code, "config_cost")
    return out.value


def lpt_partition(costs, bins):
    """Bin of each task by cube2_lpt_partition (largest cost first, to the least loaded bin)."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    out = np.zeros(len(c), dtype=np.int32)
    code = _lib.cube2_lpt_partition(c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(c), int(bins),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if code != OK:
        raise Cube2Error(code, "lpt_partition")
    return out


def _ensemble_arrays(ctxs, states, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    nb = a.shape[0]
    if nb != len(ctxs) or nb != len(states):
        raise ValueError("one context, state and schedule per box")
    structs = [st.struct() for st in states]
    cp = (ctypes.c_void_p * nb)(*[c.ptr.value for c in ctxs])
    pp = (ctypes.c_void_p * nb)(*[ctypes.addressof(x) for x in structs])
    return a, structs, cp, pp


class Ensemble:
    """n_steps KDK steps of many boxes recorded as one CUDA graph (cube2_ensemble_*).

    ctxs / states: one Context and IOSState per box, forces current.  a: array
    (n_boxes, n_steps + 1) of scale factors.  opts: an EnsembleOpts
    (``ensemble_opts``); without it, n_streams branches of per-box launches.
    The states' tensors are used in place by every launch and must stay alive
    (this object keeps them)."""

    def __init__(self, ctxs, states, a, n_streams=8, opts=None):
        self.ctxs, self.states = list(ctxs), list(states)
        a, self._structs, cp, pp = _ensemble_arrays(self.ctxs, self.states, a)
        nb, ns = a.shape[0], a.shape[1] - 1
        self.opts = opts if opts is not None else ensemble_opts(n_streams=n_streams)
        ptr = ctypes.c_void_p()
        code = _lib.cube2_ensemble_create_ex(ctypes.byref(ptr), cp, pp, nb,
                                             a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ns,
                                             ctypes.byref(self.opts))
        if code != OK:
            msgs = [_lib.cube2_last_error(c.ptr).decode() for c in self.ctxs]
            raise Cube2Error(code, "; ".join(m for m in msgs if m) or "ensemble_create")
        self.ptr = ptr

    def launch(self, stream=None):
        st = torch.cuda.current_stream() if stream is None else stream
        code = _lib.cube2_ensemble_launch(self.ptr, ctypes.c_void_p(st.cuda_stream))
        if code != OK:
            raise Cube2Error(code, "ensemble_launch")

    def check(self, stream=None):
        """Synchronise; raise Cube2Error(ERR_TIMEOUT) if a persistent kernel gave up waiting."""
        st = torch.cuda.current_stream() if stream is None else stream
        code = _lib.cube2_ensemble_check(self.ptr, ctypes.c_void_p(st.cuda_stream))
        if code != OK:
            raise Cube2Error(code, "ensemble_check")

    def publish(self, on=True):
        """Host control of the persistent queue's publication (False withholds it)."""
        code = _lib.cube2_ensemble_publish(self.ptr, int(bool(on)))
        if code != OK:
            raise Cube2Error(code, "ensemble_publish")

    def info(self):
        """(kernel nodes in the graph, particle-steps per launch)."""
        out = (ctypes.c_int64 * 2)()
        code = _lib.cube2_ensemble_info(self.ptr, out)
        if code != OK:
            raise Cube2Error(code, "ensemble_info")
        return int(out[0]), int(out[1])

    def close(self):
        if getattr(self, "ptr", None):
            _lib.cube2_ensemble_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ensemble_autotune(ctxs, states, a, start=None, trials=2, stream=None):
    """cube2_ensemble_autotune: (fastest EnsembleOpts, its ms per launch); the
    boxes' states are left as they were."""
    a, _structs, cp, pp = _ensemble_arrays(list(ctxs), list(states), a)
    best = start if start is not None else ensemble_opts()
    best = EnsembleOpts(best.n_streams, best.persistent_pp, best.pp_ctas_per_sm, best.pp_wmax, best.timeout_ms)
    ms = ctypes.c_double()
    st = torch.cuda.current_stream() if stream is None else stream
    code = _lib.cube2_ensemble_autotune(cp, pp, a.shape[0], a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        a.shape[1] - 1, int(trials), ctypes.c_void_p(st.cuda_stream),
                                        ctypes.byref(best), ctypes.byref(ms))
    if code != OK:
        raise Cube2Error(code, "ensemble_autotune")
    return best, ms.value


def kdk_factors(cfg: Config, a0, a1):
    out = (ctypes.c_double * 3)()
    code = _lib.cube2_kdk_factors(ctypes.byref(cfg), float(a0), float(a1), out)
    if code != OK:
        raise Cube2Error(code, "kdk_factors")
    return tuple(out)


# module-level functions with the C names -------------------------------------
def init_mesh(cfg: Config, stream=None) -> Context:
    return Context(cfg, stream)


def set_green(ctx: Context, level, cache_path=None):
    ctx.set_green(level, cache_path)


def deposit(ctx: Context, level, p: IOSState):
    ctx.deposit(level, p)


def solve_pm(ctx: Context, level):
    ctx.solve_pm(level)


def interp_force(ctx: Context, level, p: IOSState, accumulate=False):
    ctx.interp_force(level, p, accumulate)


def pp_force(ctx: Context, p: IOSState, accumulate=False):
    ctx.pp_force(p, accumulate)


def force(ctx: Context, p: IOSState):
    ctx.force(p)


def kdk_step(ctx: Context, p: IOSState, a0, a1):
    ctx.kdk_step(p, a0, a1)


def adjoint_init(ctx: Context):
    ctx.adjoint_init()


def loss_gradient(ctx: Context, p0: IOSState, target: torch.Tensor, a, level=-1):
    """Gradient of L = mean((delta_final - target)^2) through len(a) - 1 KDK
    steps with respect to the initial positions and velocities.

    p0: the initial state with current forces (unchanged).  Runs the steps
    with a checkpoint and re-bin map per step, then cube2_density_mse_vjp and
    cube2_kdk_adjoint_step backwards.  Returns (L, dL/dx0, dL/dv0), the
    gradients (3, N) in p0's particle order."""
    level = ctx.cfg.n_levels - 1 if level < 0 else level
    states, perms = [p0], []
    p = p0.clone()
    for k in range(len(a) - 1):
        ctx.kdk_step(p, a[k], a[k + 1])
        perms.append(ctx.kdk_permutation())
        states.append(p.clone())
    loss, xbar = ctx.density_mse_vjp(level, states[-1], target)
    pbar = torch.zeros_like(xbar)
    ctx.kdk_adjoint(states, perms, a, xbar, pbar)
    return loss, xbar, pbar


def force_vjp(ctx: Context, p: IOSState, v, out=None):
    return ctx.force_vjp(p, v, out)


def ios_from_positions(ctx: Context, pos, mom=None, out=None, perm=None):
    return ctx.ios_from_positions(pos, mom, out, perm)


class FinalDensity(torch.autograd.Function):
    """The final overdensity of one level after len(a) - 1 KDK steps as a
    differentiable function of the initial positions x0 ((3, N) FP64, Mpc/h)
    and momenta v0 ((3, N) FP32), in the caller's particle order.

    Forward: cube2_ios_from_positions, the force, the steps (a checkpoint and
    re-bin map kept per step), cube2_deposit of the final state.  Backward, for
    a cotangent g on the density: cube2_density_vjp (the position gradient of
    <g, delta>), the reverse sweep cube2_kdk_adjoint, and the gradients put
    back into the input order through the placement's permutation.  The IOS quantisation of x0 and
    the drift's rounding are taken as the identity (the gradient of the
    continuous map at the stored positions)."""

    @staticmethod
    def forward(fctx, x0, v0, ctx, a, level):
        ctx.adjoint_init()
        p, perm = ctx.ios_from_positions(x0.detach(), v0.detach())
        ctx.force(p)
        states, perms = [p], []
        q = p.clone()
        for k in range(len(a) - 1):
            ctx.kdk_step(q, a[k], a[k + 1])
            perms.append(ctx.kdk_permutation())
            states.append(q.clone())
        ctx.deposit(level, states[-1])
        delta = ctx.get_density(level).clone()
        fctx.sim = (ctx, list(a), level, states, perms, perm, delta)
        fctx.dtypes = (x0.dtype, v0.dtype)
        return delta

    @staticmethod
    def backward(fctx, g):
        ctx, a, level, states, perms, perm, delta = fctx.sim
        xbar = ctx.density_vjp(level, states[-1], g.to(delta.dtype))
        pbar = torch.zeros_like(xbar)
        ctx.kdk_adjoint(states, perms, a, xbar, pbar)
        idx = perm.long()
        gx = torch.zeros(xbar.shape, dtype=fctx.dtypes[0], device=xbar.device)
        gv = torch.zeros(pbar.shape, dtype=fctx.dtypes[1], device=pbar.device)
        gx[:, idx] = xbar.to(gx.dtype)
        gv[:, idx] = pbar.to(gv.dtype)
        return gx, gv, None, None, None


def final_density(ctx: Context, x0, v0, a, level=-1):
    """Differentiable final overdensity (FinalDensity.apply)."""
    level = ctx.cfg.n_levels - 1 if level < 0 else level
    return FinalDensity.apply(x0, v0, ctx, a, level)
