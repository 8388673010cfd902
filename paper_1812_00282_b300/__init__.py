"""VATE (arXiv 1812.00282) on B300: sliding-window host cardinality with
asynchronous timestamps, as hand-written CUDA for sm_103a behind a C ABI.

``paper_1812_00282_b300.vate`` is the ctypes binding of ``include/vate.h``;
importing this package loads ``libvate.so`` and fails if it is not built.
"""
from .vate import *  # noqa: F401,F403
from .vate import Vate, VateError, make_params, vate_info, vate_params  # noqa: F401
