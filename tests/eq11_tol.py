"""The tolerance of Eq. 11 estimates: FP32 on the device against the FP64
oracle.

The device evaluates g * log1p(x), x = (N0*g - V0*P) / (V0*P), from an exact
integer numerator: three FP32 roundings of x and log1pf's own error, a few
1e-7 relative wherever log1p is well conditioned.  Two checks:
  - |dev - oracle| <= 1e-5 * max(|oracle|, 1) for every host;
  - pure relative error |dev - oracle| <= 1e-5 * |oracle| wherever the
    oracle's own value is meaningful to that precision (|oracle| >= 1e-3: its
    g ln Z_p - g ln Z_v form cancels to ~1e-11 absolute) and log1p is well
    conditioned (Z_p / Z_v = exp(oracle / g) >= 0.1, condition number <= 4),
    so that the absolute floor cannot hide relative drift of small estimates.
"""
import numpy as np

RTOL = 1e-5


def eq11_errors(dev, ora, g):
    """(floor-relative errors, pure relative errors on the conditioned set, that set)."""
    dev = np.asarray(dev, np.float64)
    ora = np.asarray(ora, np.float64)
    floor = np.abs(dev - ora) / np.maximum(np.abs(ora), 1.0)
    well = (np.abs(ora) >= 1e-3) & (ora / float(g) >= np.log(0.1))
    rel = np.zeros_like(ora)
    rel[well] = np.abs(dev[well] - ora[well]) / np.abs(ora[well])
    return floor, rel, well


def assert_eq11_close(dev, ora, g, what=""):
    floor, rel, well = eq11_errors(dev, ora, g)
    if floor.size:
        i = int(floor.argmax())
        assert floor[i] <= RTOL, "%s: error %.3g (floor 1) at %d: dev %r, oracle %r" % (
            what, floor[i], i, float(np.asarray(dev)[i]), float(np.asarray(ora)[i]))
        j = int(rel.argmax())
        assert rel[j] <= RTOL, "%s: relative error %.3g at %d: dev %r, oracle %r" % (
            what, rel[j], j, float(np.asarray(dev)[j]), float(np.asarray(ora)[j]))
