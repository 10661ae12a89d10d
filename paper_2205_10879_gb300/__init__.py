"""GB300-native FastMuyGPs posterior-mean engine.

The compute path is the CUDA library libfmgp.so (sources in csrc/, C ABI in
include/fmgp.h); this package holds its build step, a ctypes binding with the
same entry-point names, the serving loop and the seeded workload generators.
Submodules are imported lazily so that `workloads` can be used without
loading the CUDA library."""
import importlib

__all__ = ["fmgp_build_knn", "fmgp_precompute", "fmgp_predict", "fmgp_loocv_objective",
           "make_kernel", "PREC_FP64", "PREC_MIXED", "FmgpError"]


def __getattr__(name):
    if name in __all__ or name in ("load", "version", "coeff_shape", "Kernel"):
        mod = importlib.import_module("._binding", __name__)
        return getattr(mod, name)
    raise AttributeError(name)
