"""VATE (arXiv 1812.00282) on B300: sliding-window host cardinality with
asynchronous timestamps, as hand-written CUDA for sm_103a behind a C ABI.

``paper_1812_00282_b300.vate`` is the ctypes binding of ``include/vate.h``.
The binding is loaded on first use of any of its names (so that
``paper_1812_00282_b300.build`` can run before the library exists); loading
fails with ImportError if ``libvate.so`` is missing -- there is no fallback.
"""
import importlib

_BINDING = "paper_1812_00282_b300.vate"


_SUBMODULES = ("build", "vate", "learned", "serving", "sharded", "probe")


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    if name in _SUBMODULES:               # `from paper_1812_00282_b300 import build` before the library exists
        return importlib.import_module(__name__ + "." + name)
    mod = importlib.import_module(_BINDING)
    try:
        return getattr(mod, name)
    except AttributeError:
        raise AttributeError("module %r has no attribute %r" % (__name__, name)) from None


def __dir__():
    return sorted(set(globals()) | set(dir(importlib.import_module(_BINDING))))
