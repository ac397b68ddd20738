"""GB300-native per-time-step solver of the coupled heart-and-torso bidomain
model (block-LU / monodomain preconditioned CG with hierarchical Cholesky
factors), exposed through the C ABI in include/bid.h.

The binding lives in ``paper_1711_08708_gb300.bid``; it is imported lazily so
that ``build`` can run before the shared library exists.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name == "bid":
        import importlib
        return importlib.import_module(".bid", __name__)
    raise AttributeError(name)
