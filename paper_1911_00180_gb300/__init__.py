"""GB300-native worm lattice Boltzmann method for gray phonon transport
(Hammer, Fritz, Bedoya-Martinez, arXiv 1911.00180).

The compute path is libwlbm.so (CUDA for sm_103a, C ABI in include/wlbm.h); this package
is its Python binding.  The library is loaded on first use of any binding name, and
that raises ImportError when it is not built: there is no fallback path.  The build
module (``paper_1911_00180_gb300.build``) imports without the library.
"""
_EXPORTS = ("WormLBM", "WlbmError", "wlbm_lattice", "wlbm_schedule", "lib", "LIB_PATH",
            "wlbm_reduce_state_noalloc", "WormLBMBatch",
            "BC_PERIODIC", "BC_ISOTHERMAL", "BC_ADIABATIC_DIFFUSE", "BC_ADIABATIC_SPECULAR",
            "REDUCE_N",
            "STORE_FP32_DEV", "STORE_BF16_DEV")


def __getattr__(name):
    if name in _EXPORTS or name == "wlbm":
        import importlib
        mod = importlib.import_module(".wlbm", __name__)
        return mod if name == "wlbm" else getattr(mod, name)
    raise AttributeError(name)
