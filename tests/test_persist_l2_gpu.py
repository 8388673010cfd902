"""VATE_OPT_PERSIST_L2 (include/vate.h): the handles and monitor groups that ask
for it hold the device's process-wide persisting-L2 limit; the last one
destroyed puts back the limit it found, and a handle without the option
touches no process-wide setting.  Read with cudaDeviceGetLimit."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def persisting_limit():
    from cuda.bindings import runtime as rt
    err, value = rt.cudaDeviceGetLimit(rt.cudaLimit.cudaLimitPersistingL2CacheSize)
    assert err == rt.cudaError_t.cudaSuccess
    return int(value)


def device_maximum():
    from cuda.bindings import runtime as rt
    err, value = rt.cudaDeviceGetAttribute(rt.cudaDeviceAttr.cudaDevAttrMaxPersistingL2CacheSize,
                                           torch.cuda.current_device())
    assert err == rt.cudaError_t.cudaSuccess
    return int(value)


def test_the_last_persisting_handle_restores_the_limit(V):
    pytest.importorskip("cuda.bindings")
    torch.cuda.synchronize()
    before = persisting_limit()
    plain = V.Vate(16, 4, 256, 2, 0, 1)
    assert persisting_limit() == before                    # no option: nothing process-wide
    a = V.Vate(16, 4, 256, 2, 0, 2, options=V.VATE_OPT_PERSIST_L2)
    b = V.Vate(16, 4, 256, 2, 0, 3, options=V.VATE_OPT_PERSIST_L2)
    held = persisting_limit()
    if device_maximum() > 0:
        assert held >= min(device_maximum(), max(before, 1))
    a.close()
    assert persisting_limit() == held                      # b still holds it
    b.close()
    assert persisting_limit() == before                    # put back
    plain.close()
    assert persisting_limit() == before


def test_a_persisting_group_restores_the_limit(V):
    pytest.importorskip("cuda.bindings")
    torch.cuda.synchronize()
    before = persisting_limit()
    prm = [V.vate_params(log2_pool=16, k=4, g=256, seg_len=2, partition=0, counter=0, at_bits=0,
                         options=V.VATE_OPT_PERSIST_L2 if s == 1 else 0, seed=s) for s in range(2)]
    g = V.vate_group_create(prm)
    if device_maximum() > 0:
        assert persisting_limit() >= min(device_maximum(), max(before, 1))
    V.vate_group_destroy(g)
    assert persisting_limit() == before
