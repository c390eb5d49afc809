"""FP64 CPU oracle of the CUBE2 multi-level PM + PP force step and its KDK update.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2512_12629_gb300``) never imports, calls or links
anything here, and nothing here imports the product path: the two share only
the seeded input generator in ``inputs/``.

Written from the paper (CUBE2, Yu et al., Sci. China PMA 2026) in plain
numpy FP64, following its steps in order:

* kernels.py  Eqs. (denprofile), (refforce), (Sk), (Rk), (diff), (Gk)
* mesh.py     Sec. 2.1.2 PM steps: CIC deposit (integer), Poisson solve,
              4-point FD in real space, CIC interpolation
* pp.py       Sec. 2.2.3 and Eq. (PP): cell-list PP over IOS order
* kdk.py      total force and the kick-drift-kick step with IOS re-binning
* ewald.py    periodic direct summation, used only to pin the oracle

numpy.fft (rfftn/irfftn) is used as the FFT primitive.

Pins (tests/test_oracle_*.py): closed forms of S, R and S(k); quadrature of
S(r) -> S(k) and S^2(k)/k^2 -> R(r); D(k) against the DFT of the stencil;
the CIC alias sum against its closed form; the symmetry and continuum limit
of G; exact-rational brute-force CIC; Ewald direct summation; Newton's law
for two bodies; the Zel'dovich pancake; momentum conservation; EdS closed
forms of the KDK integrals.
"""
from . import ewald, kdk, kernels, mesh, pp  # noqa: F401
