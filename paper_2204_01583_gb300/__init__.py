"""GB300 (sm_103a) contour-integral overlap operator.

sgn(H_W) b and D_ov(m_q) b from a trapezoid-rule quadrature of resolvents
(Nagai & Tomiya, arXiv:2204.01583, Eqs. 1, 5-7), computed by a CUDA library
behind the C ABI of ``include/ov.h``.  ``lib`` is its ctypes binding; ``ops``
adds torch-facing helpers (canonical tensor layouts, autograd).
"""
from .build import build  # noqa: F401

__all__ = ["build", "lib", "ops"]


def __getattr__(name):
    if name in ("lib", "ops"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
