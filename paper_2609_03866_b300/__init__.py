"""ncf: kernel-weighted auto/cross-correlation of irregularly sampled series
on one B300 GPU (sm_103a), after the Wiener-Khinchin NUFFT estimator of
arXiv 2609.03866.

The compute path is the C-ABI library ``libncf.so`` (hand-written CUDA); this
package only marshals arguments to it.  Importing the package does not load
the library; the first call does, and fails loudly if it is missing.
"""
__all__ = ["corr", "corr_batch", "Context"]


def __getattr__(name):
    if name in ("corr", "corr_batch", "Context", "NcfError", "lib"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
