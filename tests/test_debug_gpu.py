"""The checked build (VATE_DEBUG, libvate_debug.so), which stands in for a
memory checker: its kernels check every computed pool position, every AT
value they read and every block index, and record a violation in the handle's
status words instead of trapping.

  - On clean data it computes exactly what the release library computes (pool,
    census, estimates, flags) and records nothing.
  - A deliberately corrupted stored value (vate_debug_poke, checked build
    only) is reported by the next kernel that reads it -- the gather of an
    estimate -- with the VALUE bit and the 16-byte chunk that holds it;
    nothing traps and the handle keeps working.
  - The release library has the checks compiled out.
"""
import numpy as np
import pytest
import torch

from traffic import SMALL, Traffic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def as_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def run(V, params, slices=5):
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    d = V.Vate(*params[:6], counter=params[6] if len(params) > 6 else 0)
    hosts = as_i32(tr.aips[:2000])
    out = []
    for s in range(slices):
        d.ingest(as_i32(tr.slice_pairs(s)), s)
        d.close_slice(s)
        pool = torch.empty(1 << params[0], dtype=torch.uint8 if params[1] <= 63 else torch.int16, device="cuda")
        hist = torch.empty(2 * params[1] + 1, dtype=torch.int64, device="cuda")
        e = torch.empty(hosts.numel(), dtype=torch.float32, device="cuda")
        f = torch.empty(hosts.numel(), dtype=torch.uint8, device="cuda")
        d.copy_pool(pool)
        d.census(hist)
        d.estimate(hosts, params[1], e, f)
        out.append([t.cpu().numpy() for t in (pool, hist, e, f)])
    status = V.vate_debug_status(d.h)
    d.close()
    return out, status


@pytest.mark.parametrize("params", [(16, 5, 512, 32, 0, 1), (16, 5, 512, 2, 1, 2), (17, 100, 256, 1, 0, 3),
                                    (16, 4, 512, 32, 0, 4, 1)],
                         ids=["L32", "L2-lowdev", "16bit-L1", "recorders"])
def test_checked_build_equals_release_and_reports_nothing(V, params):
    ref, st0 = run(V, params)
    assert st0 == (0, 0)
    with V.use_library(V.DEBUG_LIB_PATH):
        assert V.vate_debug_checks()
        chk, st = run(V, params)
    assert st == (0, 0), "the checked build reported %r on clean data" % (st,)
    for s, (a, b) in enumerate(zip(ref, chk)):
        for name, x, y in zip(("pool", "census", "estimates", "flags"), a, b):
            assert np.array_equal(x, y), "slice %d: %s differs between the builds" % (s, name)


def test_checked_build_reports_a_corrupted_value_and_keeps_going(V):
    c, k, g, L = 16, 5, 512, 32
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    with V.use_library(V.DEBUG_LIB_PATH):
        d = V.Vate(c, k, g, L, 0, 7)
        hosts = as_i32(tr.aips[:500])
        e = torch.empty(hosts.numel(), dtype=torch.float32, device="cuda")
        for s in range(3):
            d.ingest(as_i32(tr.slice_pairs(s)), s)
            d.close_slice(s)
        d.estimate(hosts, k, e)
        assert V.vate_debug_status(d.h) == (0, 0)
        pid = V.vate_host_h(d.params, int(tr.aips[0]), 5)   # a VAT of the first host
        V.vate_debug_poke(d.h, pid, 2 * k + 9)              # above 2k: out of range
        d.estimate(hosts, k, e)
        torch.cuda.synchronize()
        bits, first = V.vate_debug_status(d.h)
        assert bits & V.VATE_DBG_VALUE
        assert first >> 63 == 1 and (first >> 56) & 0x7F == V.VATE_DBG_VALUE
        assert first & ((1 << 56) - 1) == pid >> 4           # the 16-byte chunk the gather read it from
        # nothing trapped: the handle keeps working
        V.vate_debug_status(d.h, clear=True)
        d.ingest(as_i32(tr.slice_pairs(3)), 3)
        d.close_slice(3)
        d.estimate(hosts, k, e)
        torch.cuda.synchronize()
        assert torch.isfinite(e).all()
        d.close()


def test_release_build_has_no_checks(V):
    assert not V.vate_debug_checks()
    d = V.Vate(14, 2, 64, 1, 0, 1)
    with pytest.raises(V.VateError) as e:
        V.vate_debug_poke(d.h, 0, 200)
    assert e.value.code == V.VATE_EINVAL
    d.close()
