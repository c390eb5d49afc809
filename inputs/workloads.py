"""Workload definitions (pure data, no arithmetic of the method).

Each workload fixes the box, the particle lattice, the Information Optimized
Storage (IOS) mesh, the PM levels (coarsest first, each with its softening
factor beta in its own mesh cells), the PP softening b_PP, the cosmology and
the time span.  Both the CUDA path and the FP64 oracle read these records;
each derives its own softening/truncation lengths from them.

Cosmology and spectrum follow the workload recipe of this project: flat
LCDM with Omega_m = 0.3, Omega_L = 0.7, h = 0.7, sigma_8 = 0.8, a BBKS
transfer function and Zel'dovich initial conditions.  The paper's own runs
(Sec. 3.2) use CAMB spectra at z_i = 200; those inputs are not reproduced.
"""
from __future__ import annotations

import numpy as np
from dataclasses import dataclass, field, replace


@dataclass(frozen=True)
class Level:
    n_mesh: int      # mesh cells per dimension
    beta: float      # softening length b = beta * H in this level's cells


@dataclass(frozen=True)
class PM3Spec:
    """Adaptive third PM level: subtiles of ``tile``^3 IOS cells; a subtile
    whose densest IOS cell holds >= ``rho_min`` particles gets a local mesh of
    spacing H_finest / ``refine`` with softening ``beta`` local cells (its PP
    range); at most ``max_tiles`` refined subtiles per force evaluation."""
    tile: int
    refine: int
    beta: float
    rho_min: int
    max_tiles: int = 4096


@dataclass(frozen=True)
class Workload:
    name: str
    n_p: int                     # particles per dimension on the Lagrangian lattice
    box: float                   # comoving box side L [Mpc/h]
    n_ios: int                   # IOS cells per dimension (cell = PP cell)
    levels: tuple                # tuple[Level], coarsest first
    b_pp: float                  # PP softening [Mpc/h]
    z_init: float = 49.0
    z_final: float = 0.0
    n_steps: int = 1
    seed: int = 1
    omega_m: float = 0.3
    omega_l: float = 0.7
    h: float = 0.7
    sigma8: float = 0.8
    # growth factor used for the displacement: None -> D(a_init);
    # a float -> D at that scale factor (e.g. 1.0 for a z=0-like state)
    displace_to_a: float | None = None
    assign_order: int = 2        # mass assignment: 2 = CIC (the workload's), 3 = TSC (the paper's)
    iso_length: float = 0.0      # > 0: isolated boundary conditions, force truncated at this r [Mpc/h]
    pm3: PM3Spec | None = None   # adaptive third PM level (None: the global levels only)
    vel_fp16: bool = False       # velocities stored as FP16 with a per-IOS-cell FP32 scale

    @property
    def n_particles(self) -> int:
        return self.n_p ** 3

    @property
    def a_init(self) -> float:
        return 1.0 / (1.0 + self.z_init)

    @property
    def a_final(self) -> float:
        return 1.0 / (1.0 + self.z_final)

    def scale_factors(self):
        """Constant-Delta-a schedule a_0 < a_1 < ... < a_{n_steps}."""
        a0, a1 = self.a_init, self.a_final
        return [a0 + (a1 - a0) * i / self.n_steps for i in range(self.n_steps + 1)]

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# 32^3 particles, 64 Mpc/h, one 64^3 PM level with a 2-cell softening (= PP
# cutoff), 1 force evaluation + 1 KDK step from z = 49.
C1 = Workload(
    name="pm1-32c-64mesh", n_p=32, box=64.0, n_ios=32,
    levels=(Level(64, 2.0),), b_pp=0.2,
    z_init=49.0, z_final=0.0, n_steps=50, seed=1,
)

# 256^3 particles, 256 Mpc/h, coarse 128^3 (beta 3.5) + fine 512^3 (beta 2),
# FP32 velocities, 50 constant-Delta-a KDK steps z = 49 -> 0.
C2 = Workload(
    name="pm2-256c-128x512mesh", n_p=256, box=256.0, n_ios=256,
    levels=(Level(128, 3.5), Level(512, 2.0)), b_pp=0.1,
    z_init=49.0, z_final=0.0, n_steps=50, seed=2,
)

# Same recipe as C2 at 1/64 of the volume (64^3 particles, 32^3 + 128^3
# meshes): the size used for element-wise parity of the two-level path.
C2_SMALL = C2.with_(name="pm2-64c-32x128mesh", n_p=64, box=64.0, n_ios=64,
                    levels=(Level(32, 3.5), Level(128, 2.0)), seed=12)

# The two-level recipe at 64^3 particles with the paper's TSC assignment
# (Eq. filter) instead of CIC.
C2_SMALL_TSC = C2_SMALL.with_(name="pm2-64c-32x128mesh-tsc", assign_order=3)
# The 256^3 workload with TSC assignment.
C2_TSC = C2.with_(name="pm2-256c-128x512mesh-tsc", assign_order=3)

# Pairwise force accuracy under isolated boundary conditions (Sec. 3.1,
# Appendix A): two particles at a time in a 64 Mpc/h box with the force
# truncated at L = 32 Mpc/h (the doubled box of the paper's test), the paper's
# softening of 3.5 cells on both levels (coarse mesh n_ios/2, fine mesh
# 4 n_ios so that the PP range 1.75 Mpc/h fits the 2 Mpc/h IOS cell),
# b_pp = 0.1 IOS cell.  Separations below L - b_coarse = 18 Mpc/h are exactly
# isolated.  n_p is unused: the pairs are placed explicitly.
ISO_PAIRS = Workload(
    name="pm2-iso-pairs-32c-16x128mesh", n_p=2, box=64.0, n_ios=32,
    levels=(Level(16, 3.5), Level(128, 3.5)), b_pp=0.2, iso_length=32.0, seed=31,
)

# Same recipe as C2 at 27/64 of the volume (192^3 particles, 96^3 + 384^3
# meshes, the same IOS/mesh ratios): every array larger than L2, a working
# set of about 1.5 GB; the size used for multi-pass profiler captures.
C2_MID = C2.with_(name="pm2-192c-96x384mesh", n_p=192, box=192.0, n_ios=192,
                  levels=(Level(96, 3.5), Level(384, 2.0)), seed=22)

# Differentiation workload: 128^3 particles, 128 Mpc/h, one 256^3 level,
# 10 KDK steps z = 9 -> 0.
C3 = Workload(
    name="pm1-128c-256mesh", n_p=128, box=128.0, n_ios=128,
    levels=(Level(256, 2.0),), b_pp=0.1,
    z_init=9.0, z_final=0.0, n_steps=10, seed=3,
)

# 1024^3 particles, 1 Gpc/h, coarse 512^3 + fine 2048^3, one force
# evaluation on a z=0-like Zel'dovich state.
C5 = Workload(
    name="pm2-1024c-512x2048mesh", n_p=1024, box=1000.0, n_ios=1024,
    levels=(Level(512, 3.5), Level(2048, 2.0)), b_pp=0.1 * 1000.0 / 1024,
    z_init=49.0, z_final=0.0, n_steps=1, seed=5, displace_to_a=1.0,
)

def c4_ensemble(n_boxes=64, seed=100, n_steps=20, sizes=(32, 48, 64, 96)):
    """Ensemble of independent boxes at C1's resolution: box b has
    n_p ~ U(sizes) particles per side, L = 2 n_p Mpc/h, one PM level of
    2 n_p cells (2-cell softening = the IOS cell), n_p^3 IOS cells,
    sigma_8 ~ U(0.7, 0.9), seed ``seed + b``, n_steps constant-Delta-a KDK
    steps from z = 49 to 0.  Sizes and sigma_8 come from one Philox stream
    seeded with ``seed``."""
    rng = np.random.Generator(np.random.Philox(seed))
    n_ps = rng.choice(np.asarray(sizes), size=n_boxes)
    s8 = rng.uniform(0.7, 0.9, size=n_boxes)
    return [Workload(name=f"c4-box{b}-n{int(n)}", n_p=int(n), box=2.0 * int(n), n_ios=int(n),
                     levels=(Level(2 * int(n), 2.0),), b_pp=0.2, z_init=49.0, z_final=0.0,
                     n_steps=n_steps, seed=seed + b, sigma8=float(sg))
            for b, (n, sg) in enumerate(zip(n_ps, s8))]


# The 256^3 run with the adaptive third PM level: subtiles of 8^3 IOS cells
# (8 Mpc/h) whose densest IOS cell holds >= 512 particles get a local mesh of
# 0.25 Mpc/h cells (48^3 with its buffer) and softening 2 local cells, which
# halves their PP range.  The threshold balances a local mesh (about 2 us of
# deposit and FFT) against the PP pairs it removes (about 2.4 ps each) at the
# densities this run reaches (a few hundred subtiles by z = 0: 392 at the
# last step).  The capacity bounds the batched FFT grids (blocks of unused
# meshes return at once, but are still scheduled), so it is sized to the run.
C2_PM3 = C2.with_(name="pm2-256c-128x512mesh-pm3", pm3=PM3Spec(tile=8, refine=2, beta=2.0, rho_min=512,
                                                                max_tiles=512))

WORKLOADS = {w.name: w for w in (C1, C2, C2_SMALL, C2_MID, C3, C5, C2_SMALL_TSC, C2_TSC, ISO_PAIRS, C2_PM3)}
