"""GB300 (sm_103a) hot path of NysADMM: Nystrom-preconditioned CG for the
ADMM x-subproblem (A^T D A + rho I) x = r, with the sketch, the FP64 Nystrom
core, the preconditioner apply, the fused A/A^T pass and the prox/dual steps,
behind the C ABI of include/nysadmm.h.

The binding (paper_2202_11599_gb300.nysadmm) is imported lazily so that the
package can be inspected without a GPU; it raises if libnysadmm.so is missing.
"""
import importlib

__all__ = ["nysadmm", "build_lib"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
