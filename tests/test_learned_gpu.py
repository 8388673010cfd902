"""The learned estimator's kernels (include/vate_learned.h) against the FP64
reference of the model (oracle/mlp.py) and the oracle's features:
  - features: per-age counts and pool fractions exact, the Eq. 11 feature
    within the FP32 tolerance;
  - forward pass within FP32 accumulation tolerance;
  - one training step: gradient and loss within FP32 tolerance, Adam update
    recomputed from the returned gradient;
  - training is bit-reproducible;
  - the learned estimate (vate_estimate_learned, which serves closes: one
    fused kernel for L >= 16, two passes for L <= 8) against the oracle's
    output rule (oracle/mlp.py estimate) fed with the oracle's own features: flags bit-exact (FALLBACK included),
    fallback rows within the Eq. 11 tolerance, the others within the bound
    derived from the kernel's FP32 arithmetic (tests/learned_tol.py) -- on
    the small traffic (every host, a ragged count, hosts never seen) and at
    full size in the benchmark's launch configuration (all 2^20 hosts of the
    40 Gb/s traffic in one call on the 2^24-AT pool, k = 10, g = 4096, a
    seeded sample plus every super-spreader compared).
"""
import numpy as np
import pytest
import torch

from eq11_tol import assert_eq11_close
from learned_tol import learned_error_bound
from oracle import Oracle, mlp
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


def small_run(V, L=32, k=5, c=16, g=512, slices=8):
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    d = V.Vate(c, k, g, L, 0, 7)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=0, seed=7)
    for s in range(slices):
        p = tr.slice_pairs(s)
        if s:
            o.advance()
        o.ingest(p)
        d.ingest(as_i32(p), s)
    d.close_slice(slices - 1)
    return tr, d, o


@pytest.mark.parametrize("L", [1, 32])
def test_features_match_oracle(V, L):
    tr, d, o = small_run(V, L=L)
    hosts = tr.aips[:1500]
    k = o.k
    x = torch.empty(len(hosts) * (2 * k + 2), dtype=torch.float32, device="cuda")
    V.vate_features(d.h, as_i32(hosts), x)
    X = x.view(len(hosts), -1).cpu().numpy().astype(np.float64)
    Xo, _ = mlp.features(o, hosts)
    np.testing.assert_allclose(X[:, :2 * k + 1], Xo[:, :2 * k + 1], rtol=1e-6, atol=0)
    np.testing.assert_allclose(X[:, 2 * k + 1], Xo[:, 2 * k + 1], rtol=1e-5, atol=1e-6)
    d.close()


def test_forward_matches_reference(V):
    rng = np.random.default_rng(1)
    n_in = 22
    p = rng.normal(0, 0.2, mlp.n_params(n_in)).astype(np.float32)
    X = rng.normal(0, 1, (3000, n_in)).astype(np.float32)
    y = torch.empty(3000, dtype=torch.float32, device="cuda")
    V.vate_mlp_forward(torch.from_numpy(p).cuda(), n_in, torch.from_numpy(X).cuda(), y)
    ref = mlp.forward(p.astype(np.float64), n_in, X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)


def test_mlp_apply_matches_the_oracle_rule(V):
    # vate_mlp_apply (the rule the model selection scores) against the oracle's
    # rule on the same feature rows: rows with no active VAT, negative, small
    # and gated closed forms
    rng = np.random.default_rng(12)
    k, n_in, n = 5, 12, 5000
    p = rng.normal(0, 0.1, mlp.n_params(n_in)).astype(np.float32)
    p[-1] = 300.0
    X = rng.uniform(0, 0.05, (n, n_in)).astype(np.float32)
    X[::7, :k] = 0.0                                      # no active VAT
    plain = np.exp(rng.uniform(-1, 8, n)).astype(np.float32) * rng.choice([-1, 1, 1, 1], n).astype(np.float32)
    X[:, n_in - 1] = (np.log1p(np.maximum(plain, 0)) / 16).astype(np.float32)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    V.vate_mlp_apply(torch.from_numpy(p).cuda(), n_in, torch.from_numpy(X).cuda(), torch.from_numpy(plain).cuda(),
                     out, fl)
    est, flags, z = mlp.estimate(p.astype(np.float64), n_in, X.astype(np.float64), plain.astype(np.float64), k)
    with np.errstate(over="ignore"):
        amb = np.abs(np.expm1(z) - 300.0) <= 0.03            # either side of the gate in FP32
    np.testing.assert_array_equal(fl.cpu().numpy()[~amb], flags[~amb])
    assert (flags & mlp.GATED).any() and (flags & mlp.FALLBACK).any() and (flags == 0).any()
    dev = out.cpu().numpy().astype(np.float64)
    closed = (flags != 0) & ~amb
    assert np.array_equal(dev[closed], plain[closed].astype(np.float64))
    m = (flags == 0) & ~amb
    bound = learned_error_bound(p.astype(np.float64), n_in, X[m].astype(np.float64), plain[m].astype(np.float64),
                                z[m], est[m], plain_rtol=0.0)
    assert np.all(np.abs(dev[m] - est[m]) <= bound)


@pytest.mark.parametrize("kind", [0, 1])
def test_train_step_gradient_and_update(V, kind):
    rng = np.random.default_rng(2)
    n_in, n = 12, 1000
    npar = mlp.n_params(n_in)
    p = rng.normal(0, 0.2, npar).astype(np.float32)
    X = rng.normal(0, 1, (n, n_in)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    dp = torch.from_numpy(p.copy()).cuda()
    m = torch.zeros(npar, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    grad = torch.empty_like(m)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    scratch = torch.empty(V.vate_mlp_train_scratch(n_in, n), dtype=torch.float32, device="cuda")
    lr = 1e-3
    w = rng.uniform(0.2, 3.0, n).astype(np.float32)
    V.vate_mlp_train_step(dp, m, v, n_in, torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), lr, 1, scratch,
                          grad, loss, weight=torch.from_numpy(w).cuda(), loss_kind=kind)
    lref, gref = mlp.loss_and_grad(p.astype(np.float64), n_in, X.astype(np.float64), t.astype(np.float64),
                                   w.astype(np.float64), absolute=(kind == 1))
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - lref) <= 1e-5 * abs(lref)
    scale = np.abs(gref).max()
    assert np.abs(g - gref).max() <= 1e-4 * scale, np.abs(g - gref).max() / scale
    # Adam at t = 1 from zero moments: m = 0.1 g, v = 0.001 g^2, update lr * g / (|g| + eps)
    gf = grad.cpu().numpy()
    expect = p - lr * (0.1 * gf / 0.1) / (np.sqrt(0.001 * gf * gf / 0.001) + 1e-8)
    np.testing.assert_allclose(dp.cpu().numpy(), expect, rtol=1e-6, atol=1e-7)


def check_fused_against_oracle(V, d, o, hosts, params, out=None, fl=None, idx=None):
    """vate_estimate_learned on `hosts` (all of them in one call) against the
    oracle's output rule on its own features, for the rows `idx` (all when
    None).  Returns (max relative error, share of rows within 1e-5 * max(|o|, 1))."""
    k, n_in = o.k, 2 * o.k + 2
    n = len(hosts)
    out = torch.empty(n, dtype=torch.float32, device="cuda") if out is None else out
    fl = torch.empty(n, dtype=torch.uint8, device="cuda") if fl is None else fl
    V.vate_estimate_learned(d.h, as_i32(hosts), params, out, fl)
    idx = np.arange(n) if idx is None else idx
    sample = hosts[idx]
    X, plain = mlp.features(o, sample, k)
    _, _, pflags = o.estimate(sample, k)
    p64 = params.cpu().numpy().astype(np.float64)
    est, flags, z = mlp.estimate(p64, n_in, X, plain, k, pflags)
    dev = out.cpu().numpy()[idx].astype(np.float64)
    # a corrected value or a closed form within 1e-4 of the gate may fall on either side of it (FP32 on
    # the device, and the closed form there is within 1e-5 of the oracle's)
    tau = mlp.gate(p64)
    with np.errstate(invalid="ignore", over="ignore"):
        e_all = np.expm1(z)
        band = 1e-4 * max(abs(tau), 1.0)
        amb = np.isfinite(tau) & ((np.abs(e_all - tau) <= band) | (np.abs(plain - tau) <= band))
    assert amb.sum() <= max(2, len(idx) // 100), amb.sum()
    np.testing.assert_array_equal(fl.cpu().numpy()[idx][~amb], flags[~amb],
                                  err_msg="flags (SAT, POOLFULL, FALLBACK, GATED)")
    closed = ((flags & (mlp.FALLBACK | mlp.GATED)) != 0) & ~amb
    assert_eq11_close(dev[closed], est[closed], o.g, "rows given the closed form")
    fb = closed | amb
    m = ~fb
    bound = learned_error_bound(p64, n_in, X[m], plain[m], z[m], est[m])
    err = np.abs(dev[m] - est[m])
    worst = int(np.argmax(err / bound)) if m.any() else 0
    assert np.all(err <= bound), "row %d: |dev - oracle| %.3g above the derived bound %.3g (oracle %r)" % (
        worst, err[worst], bound[worst], est[m][worst])
    rel = err / np.maximum(np.abs(est[m]), 1.0)
    # and the estimates' 1e-5 rule (the derived bound above is the worst case of
    # the FP32 arithmetic; in practice the model's rounding stays ~10x inside it)
    assert rel.size == 0 or rel.max() <= 1e-5, "max error %.3g above 1e-5 * max(|oracle|, 1)" % rel.max()
    return (float(rel.max()) if rel.size else 0.0), (float((rel <= 1e-5).mean()) if rel.size else 1.0), \
        int(((flags & mlp.FALLBACK) != 0).sum())


def labelled_params(V, d, hosts, tr, slices, k, epochs=3, seed=5):
    """A model trained (by the library's kernels) on this handle's features with
    exact window counts as labels, so that its outputs look like a real model's."""
    from oracle.exact import window_cardinality
    from paper_1812_00282_b300 import learned
    n_in = 2 * k + 2
    x = torch.empty(len(hosts) * n_in, dtype=torch.float32, device="cuda")
    V.vate_features(d.h, as_i32(hosts), x)
    X = x.view(-1, n_in)
    sl = [tr.slice_pairs(s) for s in slices]
    cnt = window_cardinality(sl, len(sl) - 1, k, hosts)
    n = torch.from_numpy(cnt.astype(np.float64)).cuda()
    T = ((torch.log1p(n) - 16.0 * X[:, n_in - 1].double()) / 8.0).float()
    return learned.train(V, X, T, n_in, epochs=epochs, batch=512, seed=seed)


def test_training_is_reproducible(V):
    from paper_1812_00282_b300 import learned
    tr, d, o = small_run(V, L=32, k=5, c=16, g=512)
    k, n_in = 5, 12
    hosts = as_i32(tr.aips)
    x = torch.empty(hosts.numel() * n_in, dtype=torch.float32, device="cuda")
    V.vate_features(d.h, hosts, x)
    X = x.view(-1, n_in)
    T = torch.rand(X.shape[0], generator=torch.Generator(device="cuda").manual_seed(3), device="cuda")
    p1 = learned.train(V, X, T, n_in, epochs=2, batch=512, seed=5)
    p2 = learned.train(V, X, T, n_in, epochs=2, batch=512, seed=5)
    assert torch.equal(p1, p2)
    d.close()


@pytest.mark.parametrize("L", [1, 32])
@pytest.mark.parametrize("scenario", ["steady", "sparse"])
def test_fused_estimate_matches_oracle_small(V, L, scenario):
    # Every host of the small traffic plus up to 37 addresses never seen,
    # about 4,130 rows (not a multiple of 32), with a trained model and with
    # the Glorot initialisation.  steady: 8 slices into a 2^16-AT pool, where
    # nearly every host has active VATs.  sparse: a 2^20-AT pool after a gap
    # of more than 2k slices and one slice of 2,000 pairs, so that most hosts
    # have no active VAT and get the closed form with FALLBACK.
    c = 16 if scenario == "steady" else 20
    tr, d, o = small_run(V, L=L, k=5, c=c, g=512, slices=8)
    slices = list(range(8))
    if scenario == "sparse":
        s = 8 + 2 * 5 + 1
        p = tr.slice_pairs(s, 2000)
        for _ in range(s - 7):
            o.advance()
        o.ingest(p)
        d.ingest(as_i32(p), s)
        d.close_slice(s)
    rng = np.random.default_rng(17)
    absent = rng.integers(1, 1 << 32, 37, dtype=np.uint64).astype(np.uint32)
    absent = absent[~np.isin(absent, tr.aips)]
    hosts = np.concatenate([tr.aips, absent])
    trained = labelled_params(V, d, tr.aips, tr, slices, 5)
    glorot = torch.empty(V.vate_mlp_param_count(12), dtype=torch.float32, device="cuda")
    V.vate_mlp_init(glorot, 12, 99)
    assert torch.isinf(glorot[-1]) and torch.isinf(trained[-1])     # the gate starts (and trains) closed
    gated = trained.clone()
    plain = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
    d.estimate(as_i32(hosts), 5, plain)
    gated[-1] = float(torch.quantile(plain.double().clamp(min=0), 0.7)) + 0.5   # gates roughly the top 30 %
    for params in (trained, glorot, gated):
        rel, share, nfb = check_fused_against_oracle(V, d, o, hosts, params)
        if scenario == "sparse":
            assert nfb > len(hosts) // 4
        print("L=%d %s: max rel err %.3g, %.4f of rows within 1e-5, %d fallbacks" % (L, scenario, rel, share, nfb))
    d.close()


@pytest.mark.parametrize("L", [1, 2, 32])
def test_two_pass_form_equals_vate_estimate_learned(V, L):
    # vate_estimate_learned fuses features and model in one kernel for
    # L >= 16 and runs them in two passes through a scratch for L <= 8.  The
    # public two-pass form -- vate_features, Eq. 11 from vate_estimate,
    # vate_mlp_apply -- must give the same values bit for bit on either
    # placement, and the same FALLBACK / GATED bits (vate_mlp_apply reports
    # only those), with a trained model whose gate takes part.
    tr, d, o = small_run(V, L=L, k=5, c=16, g=512, slices=8)
    rng = np.random.default_rng(23)
    absent = rng.integers(1, 1 << 32, 29, dtype=np.uint64).astype(np.uint32)
    hosts = as_i32(np.concatenate([tr.aips, absent[~np.isin(absent, tr.aips)]]))
    n, n_in = hosts.numel(), 12
    params = labelled_params(V, d, tr.aips, tr, list(range(8)), 5)
    plain = torch.empty(n, dtype=torch.float32, device="cuda")
    d.estimate(hosts, 5, plain)
    params[-1] = float(torch.quantile(plain.double().clamp(min=0), 0.8)) + 0.5
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    V.vate_estimate_learned(d.h, hosts, params, out, fl)
    x = torch.empty(n * n_in, dtype=torch.float32, device="cuda")
    V.vate_features(d.h, hosts, x)
    out2 = torch.empty_like(out)
    fl2 = torch.empty_like(fl)
    V.vate_mlp_apply(params, n_in, x, plain, out2, fl2)
    assert torch.equal(out.view(torch.int32), out2.view(torch.int32))
    rule = V.VATE_FLAG_FALLBACK | V.VATE_FLAG_GATED
    assert torch.equal(fl & rule, fl2)
    assert ((fl2 & V.VATE_FLAG_GATED) != 0).any() and (fl2 == 0).any()
    d.close()


def test_fused_estimate_matches_oracle_full_size(V):
    # The learned-estimator configuration in the benchmark's launch
    # configuration: the 40 Gb/s traffic on a 2^24-AT pool, k = 10, g = 4096,
    # L = 2, every one of the 2^20 hosts estimated by one vate_estimate_learned
    # call after k + 2 slices of 5M pairs; the oracle computes a seeded sample
    # of 4,096 outputs plus every super-spreader one by one.  The model is
    # trained by the library on 20 generated slices of the same configuration
    # and its gate chosen on those training rows.
    from paper_1812_00282_b300 import learned
    from traffic import DeviceTraffic
    k, c, g = 10, 24, 4096
    tr = Traffic(LINK40G)
    X, T, P, N, _ = learned.collect(V, DeviceTraffic(tr), c, k, g, 2, 0xC4, 0, 20 + k, 8192)
    params = learned.train(V, X, T, 2 * k + 2, epochs=3, seed=0xC4, weight=learned.balance_weights(N))
    learned.choose_gate(V, params, X, P, N, 2 * k + 2)
    d = V.Vate(c, k, g, 2, 0, 0xC5)
    o = Oracle(c=c, k=k, g=g, seg_len=2, partition=0, seed=0xC5)
    for s in range(k + 2):
        if s:
            o.advance()
        p = tr.slice_pairs(s)
        o.ingest(p)
        d.ingest(torch.from_numpy(p.view(np.int32)).cuda(), s)
    d.close_slice(k + 1)
    rng = np.random.default_rng(23)
    idx = np.union1d(rng.choice(tr.spec.n_aips, 4096, replace=False), tr.super_hosts)
    rel, share, nfb = check_fused_against_oracle(V, d, o, tr.aips, params, idx=idx)
    print("full size: max rel err %.3g, %.4f of rows within 1e-5, %d fallbacks of %d" % (rel, share, nfb, len(idx)))
    d.close()


def test_learned_pipeline_small(V):
    # the whole train / held-out evaluation loop on the small traffic shape
    from paper_1812_00282_b300 import learned
    from traffic import SMALL
    r = learned.run(V, spec=SMALL, c=18, k=5, g=1024, train_slices=24, eval_slices=8, hosts_per_slice=2048,
                    eval_hosts_per_slice=2048, epochs=3)
    for pop in ("n>=1",):
        assert np.isfinite(r["mre"][pop]["learned"]) and np.isfinite(r["mre"][pop]["plain"])
        assert r["mre"][pop]["hosts"] > 1000
    assert r["params"].numel() == V.vate_mlp_param_count(12)


@pytest.mark.slow
def test_learned_full_configuration_no_worse_than_eq11(V):
    # The learned-estimator workload at full size: the 40 Gb/s traffic on a
    # 2^24-AT pool, k = 10, g = 4096, trained on 200 generated slices with
    # exact labels and evaluated on 100 held-out slices of another stream.
    # At equal AT memory its mean relative error must not exceed the closed
    # form's (Eq. 11), over all hosts active in the window and over the hosts
    # with at least 100 peers.
    from paper_1812_00282_b300 import learned
    r = learned.run(V)                      # 32-AT segments
    assert r["train_slices"] == 200 and r["eval_slices"] == 100 and r["log2_pool"] == 24
    assert r["accepted"]
    for pop in ("n>=1", "n>=100"):
        m = r["mre"][pop]
        assert m["hosts"] > 1000 and np.isfinite(m["learned"])
        assert m["learned"] <= m["plain"], (pop, m)


@pytest.mark.slow
@pytest.mark.parametrize("L", [2, 1])
def test_learned_at_short_segments_meets_its_acceptance(V, L):
    # The same workload at 2-AT segments and at the paper's placement (L = 1,
    # the 40 Gb/s workload's), where the closed form is far better than at 32
    # (mean relative error 0.28 / 0.25 instead of 0.61 over n >= 100): the
    # model, with its gate chosen on the training rows, beats it over all
    # hosts active in the window and stays within 5 % of it over the hosts with
    # n >= 100 (measured at L = 2, ungated: 5.63 vs 9.31 and 0.293 vs 0.282; at
    # L = 1, gated at 16: 7.27 vs 8.46 and 0.260 vs 0.254).
    from paper_1812_00282_b300 import learned
    r = learned.run(V, seg_len=L)
    m1, m100 = r["mre"]["n>=1"], r["mre"]["n>=100"]
    assert m1["hosts"] > 1000 and m100["hosts"] > 1000
    assert m1["learned"] <= m1["plain"], m1
    assert m100["learned"] <= learned.ACCEPT_LARGE * m100["plain"], m100
    assert r["accepted"]
