"""GB300-native (sm_103a) multi-level PM + PP gravity step of CUBE2 (Yu et al. 2026).

The compute path is libcube2gb.so (C ABI in include/cube2.h, CUDA sources in
csrc/); ``cube2`` is its thin Python binding.  ``build`` compiles the library.
Touching any binding name (``Context``, ``init_mesh``, ...) without the built
library raises ImportError: there is no CPU fallback.
"""
_BINDING = {"Config", "Context", "Cube2Error", "IOSState", "Particles", "deposit", "force",
            "init_mesh", "interp_force", "kdk_factors", "kdk_step", "make_config", "pp_force",
            "set_green", "solve_pm"}


def __getattr__(name):
    if name in _BINDING:
        from . import cube2
        return getattr(cube2, name)
    raise AttributeError(name)
