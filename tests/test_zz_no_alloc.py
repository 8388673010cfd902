"""The allocation-free census entry point, vate_census_noalloc.

It is meant for callers that cannot let a library call cudaMalloc (a
latency-bound packet loop, or an application whose device memory belongs to
its own allocator).  Its result must equal the regular census of the same pool
(vate_census) bit for bit -- the counts are integers -- on two calls in a row,
which also shows that the shared static scratch is reset between calls.
This file is collected last, so that a failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


@pytest.mark.parametrize("c,k,L,partition,counter", [(20, 5, 32, 0, 0), (26, 10, 32, 0, 0), (16, 63, 1, 1, 0),
                                                      (14, 1, 8, 1, 0), (20, 10, 32, 0, 1), (16, 63, 1, 1, 1)])
def test_census_noalloc_matches_regular_census(V, c, k, L, partition, counter):
    from traffic import SMALL, Traffic
    tr = Traffic(SMALL, pkts_per_slice=30_000)
    d = V.Vate(c, k, 64, L, partition, seed=c * 100 + k, counter=counter)
    pool = torch.empty(1 << c, dtype=torch.uint8, device="cuda")
    ref = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
    for s in range(3):
        pairs = torch.from_numpy(tr.slice_pairs(s).view(np.int32)).cuda()
        d.ingest(pairs, 2 * s)          # every other slice: the window slides twice
        d.close_slice(2 * s)
        d.census(ref)
        d.copy_pool(pool)
        info = d.info()
        for call in range(2):           # two calls in a row on the shared scratch
            out = torch.full((2 * k + 1,), -1, dtype=torch.int64, device="cuda")
            V.vate_census_noalloc(d.params, pool, info.bact0, out)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (s, call, out.cpu().numpy(), ref.cpu().numpy())
        assert int(ref.sum().item()) == 1 << c
    d.close()


def test_census_noalloc_rejects_bad_arguments(V):
    k = 5
    params = V.make_params(16, k, 64, 1, 0, 1)
    pool = torch.full((1 << 16,), 2 * k, dtype=torch.uint8, device="cuda")
    hist = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(V.VateError) as e:
        V.vate_census_noalloc(params, pool, 2 * k, hist)                          # bact0 must be below 2k
    assert e.value.code == V.VATE_EINVAL
    big = torch.empty(129, dtype=torch.int64, device="cuda")
    with pytest.raises(V.VateError) as e:
        V.vate_census_noalloc(V.make_params(16, 64, 64, 1, 0, 1), pool, 0, big)   # 129 bins: beyond the maximum
    assert e.value.code == V.VATE_EINVAL
    V.vate_census_noalloc(params, pool, 3, hist)
    torch.cuda.synchronize()
    expect = np.zeros(2 * k + 1, np.int64)
    expect[2 * k] = 1 << 16
    np.testing.assert_array_equal(hist.cpu().numpy(), expect)


@pytest.mark.parametrize("counter", [0, 1])
def test_census_noalloc_counts_out_of_range_values_as_inactive(V, counter):
    """Bytes above the counter's range (a caller's pool is not checked) are
    counted as inactive by both forms of the census -- the timestamp bins of
    the paper's per-block values and the stored-value count of recorders,
    which clamps every byte to the inactive value before it indexes the
    block's histogram."""
    c, k = 16, 5
    params = V.make_params(c, k, 64, 1, 0, 1, counter)
    g = torch.Generator().manual_seed(5)
    top = k if counter else 2 * k                  # the inactive value
    pool = torch.randint(0, top + 1, (1 << c,), generator=g, dtype=torch.int32)
    wild = torch.randint(0, 1 << c, (4096,), generator=g)
    pool[wild] = torch.randint(top + 1, 256, (4096,), generator=g, dtype=torch.int32)
    pool_u8 = pool.to(torch.uint8)
    hist = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
    V.vate_census_noalloc(params, pool_u8.cuda(), 3, hist)
    torch.cuda.synchronize()
    v = pool.numpy()
    want = np.zeros(2 * k + 1, np.int64)
    want[2 * k] = int((v >= top).sum())
    active = v[v < top]
    if counter:                                    # a recorder's value is its distance
        np.add.at(want, active, 1)
    else:                                          # Eq. 5 with the ACT of each AT's block
        from oracle import Oracle
        o = Oracle(c=c, k=k, g=64, seg_len=1, partition=0, seed=1)
        pid = np.nonzero(v < top)[0]
        act = np.array([(3 + o.block(int(p))) % (2 * k) for p in pid])
        np.add.at(want, (act - active) % (2 * k), 1)
    np.testing.assert_array_equal(hist.cpu().numpy(), want)


def test_census_noalloc_takes_no_device_memory(V):
    """The promise itself: after the first call on the device (which looks up
    the static scratch array's address), further calls leave the device's free
    memory (cudaMemGetInfo) unchanged -- no cudaMalloc, no library pool."""
    c, k = 20, 10
    params = V.make_params(c, k, 64, 32, 0, 3)
    pool = torch.randint(0, 2 * k + 1, (1 << c,), dtype=torch.uint8, device="cuda")
    hist = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
    ref = torch.empty_like(hist)
    V.vate_census_noalloc(params, pool, 1, ref)          # first call on this device: the set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(8):
        V.vate_census_noalloc(params, pool, 1, hist)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(hist, ref)
