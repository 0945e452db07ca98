"""GB300 (sm_103a) library for the exact self-gravity field of thin,
Gaussian-stratified gas + dust discs on a log-polar grid (Rendon Restrepo
et al. 2025, "Self-gravity in thin protoplanetary discs 1").

    from paper_2506_10812_gb300 import Plan
    plan = Plan(nr, nphi, r_in, r_out, h_g, h_d=None, G=1.0)
    out = plan.solve(sigma_g)          # {"phi_g", "gr_g", "gphi_g"} on the GPU

The computation lives in ``libsg.so`` (C ABI in ``include/sg.h``); this
package only marshals torch tensors into it.  ``inputs`` draws seeded
synthetic discs and can be imported without the CUDA library.
"""

__all__ = ["Plan", "Batch", "inputs"]


def __getattr__(name):
    import importlib
    if name == "Plan":
        return importlib.import_module(".plan", __name__).Plan
    if name == "Batch":
        return importlib.import_module(".batch", __name__).Batch
    if name in ("inputs", "build"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
