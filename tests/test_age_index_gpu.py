"""The age index (include/vate_hostset.h, vate_hostset_create_ages): one
pass over a host list's index in the pool's 4-bit age map gives every host's
per-age counts.  Compared bit for bit with the per-host gathers, which
test_parity_gpu.py and test_learned_gpu.py check against the oracle:
  - vate_age_counts_hostset against vate_age_counts: every L the index
    serves, both partitions, k from 1 to 15, distance recorders, pools of one,
    several and many regions, host lists with repeats and hosts never seen;
  - vate_estimate_hostset on an age index against vate_estimate and
    vate_active_counts, for several k';
  - vate_estimate_learned_hostset against vate_estimate_learned, values and
    flags (FALLBACK and GATED among them), with a trained model, the Glorot
    initialisation, and a gate that takes part;
  - the learned estimator's configuration at full size: the 2^24-AT pool, all
    2^20 hosts of the 40 Gb/s traffic, k = 10, g = 4096, L = 1 and 2;
  - the calls it must refuse.
"""
import numpy as np
import pytest
import torch

from traffic import LINK40G, SMALL, Traffic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def as_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def host_list(tr, rng, extra=37):
    absent = rng.integers(1, 1 << 32, extra, dtype=np.uint64).astype(np.uint32)
    absent = absent[~np.isin(absent, tr.aips)]
    return np.concatenate([tr.aips, absent, rng.choice(tr.aips, 50)])


def compare_counts(V, d, s, hosts, k):
    n = len(hosts)
    dh = as_i32(hosts)
    c1 = torch.empty(n * k, dtype=torch.int16, device="cuda")
    c2 = torch.full((n * k,), -1, dtype=torch.int16, device="cuda")
    V.vate_age_counts(d.h, dh, c1)
    V.vate_age_counts_hostset(d.h, s, c2)
    torch.cuda.synchronize()
    assert torch.equal(c1, c2), "per-age counts"
    return c1


def compare_estimates(V, d, s, hosts, kp):
    n = len(hosts)
    dh = as_i32(hosts)
    e1 = torch.empty(n, dtype=torch.float32, device="cuda")
    f1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    a1 = torch.empty(n, dtype=torch.int32, device="cuda")
    e2, f2, a2 = torch.empty_like(e1), torch.empty_like(f1), torch.empty_like(a1)
    d.estimate(dh, kp, e1, f1)
    V.vate_active_counts(d.h, dh, kp, a1)
    V.vate_estimate_hostset(d.h, s, kp, e2, f2, a2)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2), "A, k'=%d" % kp
    assert torch.equal(f1, f2), "flags, k'=%d" % kp
    assert torch.equal(e1.view(torch.int32), e2.view(torch.int32)), "estimates, k'=%d" % kp


def compare_learned(V, d, s, hosts, params):
    n = len(hosts)
    o1 = torch.empty(n, dtype=torch.float32, device="cuda")
    f1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    o2, f2 = torch.empty_like(o1), torch.full_like(f1, 0xAA)
    V.vate_estimate_learned(d.h, as_i32(hosts), params, o1, f1)
    V.vate_estimate_learned_hostset(d.h, s, params, o2, f2)
    torch.cuda.synchronize()
    assert torch.equal(f1, f2), "flags"
    assert torch.equal(o1.view(torch.int32), o2.view(torch.int32)), "learned estimates"
    return f1


@pytest.mark.parametrize("L", [1, 2, 4, 8])
@pytest.mark.parametrize("c,k", [(16, 5), (22, 15), (20, 1)])
@pytest.mark.parametrize("part", [0, 1])
def test_age_index_equals_per_host_gathers(V, L, c, k, part):
    g = 512
    tr = Traffic(SMALL, pkts_per_slice=30_000)
    rng = np.random.default_rng(c * 10 + L + k)
    hosts = host_list(tr, rng)
    d = V.Vate(c, k, g, L, part, 51 + L)
    s = V.vate_hostset_create_ages(d.h, as_i32(hosts))
    _, nh, nr = V.vate_hostset_info(s)
    assert nh == len(hosts) and nr == -(-(1 << c) // 393216)
    for sl in range(2 * k + 4):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        if sl in (0, k, 2 * k + 3):
            cnt = compare_counts(V, d, s, hosts, k)
            assert int(cnt.sum()) > 0
            for kp in sorted({1, (k + 1) // 2, k}):
                compare_estimates(V, d, s, hosts, kp)
    V.vate_hostset_destroy(s)
    d.close()


@pytest.mark.parametrize("L", [1, 4])
def test_age_index_with_distance_recorders(V, L):
    k, c, g = 4, 20, 256
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    hosts = tr.aips
    d = V.Vate(c, k, g, L, 0, 43, counter=V.VATE_COUNTER_DR)
    s = V.vate_hostset_create_ages(d.h, as_i32(hosts))
    for sl in (0, 1, 2, 5, 6, 14):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        compare_counts(V, d, s, hosts, k)
        for kp in (1, k):
            compare_estimates(V, d, s, hosts, kp)
    V.vate_hostset_destroy(s)
    d.close()


def trained_params(V, d, tr, hosts, slices, k, seed=5):
    """A model trained by the library's kernels on this handle's features with
    exact window counts as labels, so that its outputs look like a real model's."""
    from oracle.exact import window_cardinality
    from paper_1812_00282_b300 import learned
    n_in = 2 * k + 2
    x = torch.empty(len(hosts) * n_in, dtype=torch.float32, device="cuda")
    V.vate_features(d.h, as_i32(hosts), x)
    X = x.view(-1, n_in)
    cnt = window_cardinality([tr.slice_pairs(s) for s in slices], len(slices) - 1, k, hosts)
    n = torch.from_numpy(cnt.astype(np.float64)).cuda()
    T = ((torch.log1p(n) - 16.0 * X[:, n_in - 1].double()) / 8.0).float()
    return learned.train(V, X, T, n_in, epochs=3, batch=512, seed=seed)


@pytest.mark.parametrize("L", [1, 2, 8])
@pytest.mark.parametrize("scenario", ["steady", "sparse"])
def test_learned_through_the_age_index(V, L, scenario):
    # steady: 8 slices into a 2^16-AT pool, nearly every host active; sparse: a
    # 2^20-AT pool after a gap of more than 2k slices and one slice of 2,000
    # pairs, so that most hosts have no active VAT and fall back.  Trained,
    # Glorot-initialised and gated parameters.
    k, g = 5, 512
    c = 16 if scenario == "steady" else 20
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    rng = np.random.default_rng(7 + L)
    hosts = host_list(tr, rng, extra=29)
    d = V.Vate(c, k, g, L, 0, 7)
    s = V.vate_hostset_create_ages(d.h, as_i32(hosts))
    for sl in range(8):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
    d.close_slice(7)
    trained = trained_params(V, d, tr, tr.aips, list(range(8)), k)
    if scenario == "sparse":
        sl = 8 + 2 * k + 1
        d.ingest(as_i32(tr.slice_pairs(sl, 2000)), sl)
        d.close_slice(sl)
    glorot = torch.empty_like(trained)
    V.vate_mlp_init(glorot, 2 * k + 2, 99)
    plain = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
    d.estimate(as_i32(hosts), k, plain)
    gated = trained.clone()
    gated[-1] = float(torch.quantile(plain.double().clamp(min=0), 0.7)) + 0.5
    seen = 0
    for params in (trained, glorot, gated):
        f = compare_learned(V, d, s, hosts, params)
        seen |= int(np.bitwise_or.reduce(f.cpu().numpy()))
    assert seen & (V.VATE_FLAG_FALLBACK if scenario == "sparse" else V.VATE_FLAG_GATED)
    V.vate_hostset_destroy(s)
    d.close()


@pytest.mark.slow
@pytest.mark.parametrize("L", [1, 2])
def test_age_index_learned_configuration_full_size(V, L):
    # the learned estimator's configuration: the 40 Gb/s traffic on a 2^24-AT
    # pool, k = 10, g = 4096, all 2^20 hosts in one call; counts, A and the
    # learned estimate (Glorot parameters with a gate at the closed form's 80th
    # percentile) against the per-host gathers at three closes
    tr = Traffic(LINK40G)
    k = 10
    d = V.Vate(24, k, 4096, L, 0, 0xC3)
    s = V.vate_hostset_create_ages(d.h, as_i32(tr.aips))
    assert V.vate_hostset_info(s)[2] == 43
    params = torch.empty(V.vate_mlp_param_count(2 * k + 2), dtype=torch.float32, device="cuda")
    V.vate_mlp_init(params, 2 * k + 2, 17)
    for sl in range(2 * k + 3):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        if sl in (3, k + 1, 2 * k + 2):
            compare_counts(V, d, s, tr.aips, k)
            compare_estimates(V, d, s, tr.aips, k)
            plain = torch.empty(len(tr.aips), dtype=torch.float32, device="cuda")
            d.estimate(as_i32(tr.aips), k, plain)
            params[-1] = float(torch.quantile(plain[::64].double().clamp(min=0), 0.8)) + 0.5
            f = compare_learned(V, d, s, tr.aips, params)
            assert ((f & V.VATE_FLAG_GATED) != 0).any()
    V.vate_hostset_destroy(s)
    d.close()


@pytest.mark.parametrize("L", [1, 8])
def test_age_index_many_regions_and_tiny_lists(V, L):
    # a 2^28-AT pool (683 regions of 384 K ATs, most of them empty for a short
    # vector): a single host and a list of 300
    c, k, g = 28, 4, 64
    tr = Traffic(SMALL, pkts_per_slice=8_000)
    d = V.Vate(c, k, g, L, 0, 77)
    lists = [tr.aips[:1], tr.aips[:300]]
    sets = [V.vate_hostset_create_ages(d.h, as_i32(h)) for h in lists]
    assert V.vate_hostset_info(sets[0])[2] == 683
    for sl in range(4):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        for h, s in zip(lists, sets):
            compare_counts(V, d, s, h, k)
            compare_estimates(V, d, s, h, k)
    for s in sets:
        V.vate_hostset_destroy(s)
    d.close()


def test_age_index_refusals(V):
    tr = Traffic(SMALL, pkts_per_slice=5_000)
    hosts = as_i32(tr.aips[:100])
    wide_k = V.Vate(16, 16, 256, 2, 0, 1)
    d = V.Vate(16, 4, 256, 2, 0, 1)
    dr = V.Vate(16, 4, 256, 2, 0, 1, counter=V.VATE_COUNTER_DR)
    with pytest.raises(V.VateError) as e:                     # k > 15
        V.vate_hostset_create_ages(wide_k.h, hosts)
    assert e.value.code == V.VATE_EINVAL
    bits = V.vate_hostset_create(d.h, hosts)
    ages = V.vate_hostset_create_ages(d.h, hosts)
    ages_dr = V.vate_hostset_create_ages(dr.h, hosts)
    k, n_in = 4, 10
    params = torch.empty(V.vate_mlp_param_count(n_in), dtype=torch.float32, device="cuda")
    V.vate_mlp_init(params, n_in, 3)
    out = torch.empty(100, dtype=torch.float32, device="cuda")
    cnt = torch.empty(100 * k, dtype=torch.int16, device="cuda")
    d.ingest(as_i32(tr.slice_pairs(0)), 0)
    with pytest.raises(V.VateError) as e:                     # slice not closed
        V.vate_age_counts_hostset(d.h, ages, cnt)
    assert e.value.code == V.VATE_ESLICE
    d.close_slice(0)
    dr.ingest(as_i32(tr.slice_pairs(0)), 0)
    dr.close_slice(0)
    for call in (lambda: V.vate_age_counts_hostset(d.h, bits, cnt),            # not an age index
                 lambda: V.vate_estimate_learned_hostset(d.h, bits, params, out),
                 lambda: V.vate_estimate_learned_hostset(dr.h, ages_dr, params, out),   # recorders: no model
                 lambda: V.vate_estimate_learned_hostset(dr.h, ages, params, out)):     # another handle's index
        with pytest.raises(V.VateError) as e:
            call()
        assert e.value.code == V.VATE_EINVAL
    V.vate_age_counts_hostset(d.h, ages, cnt)
    V.vate_estimate_learned_hostset(d.h, ages, params, out)
    for s in (bits, ages, ages_dr):
        V.vate_hostset_destroy(s)
    for x in (wide_k, d, dr):
        x.close()
