"""Learned active-block gating on the GPU (rac_predictor_*, rac_enforce_learned).

- the predictor's gradient (the library's backward kernels) and its logits
  (scalar and tensor-core routines) against the float64 reference MLP;
- the trace of the Proposition-2 recurrence against the oracle: the exact set
  of candidate (sweep, state, slab) pairs, each one's label and features;
- learned gating keeps D_ac and the status of the oracle exactly, for random,
  extreme and trained predictors, with pending-pair verification and with
  RAC_VERIFY_FULL.  At threshold -inf nothing is skipped: the pending mode
  runs exactly the Proposition-2 sweeps (K sweeps, the same evaluations) and
  RAC_VERIFY_FULL adds one full sweep (K + 1); at +inf every gated sweep
  (the first one included) skips all and the verification sweep after it
  repeats one plain sweep (2K sweeps in both modes);
- the logits the sweep kernel computed and the decisions it took agree with
  the float64 MLP on the recorded features;
- a predictor trained on traces of other networks (the n=500 d=20 and batch
  generators) saves (slab, state) evaluations on the n=1000 d=24 network with
  32 assignment states while returning the oracle's D_ac.
"""
import numpy as np
import pytest

import oracle
import paper_2407_11388_b300 as rac
from oracle import gating, mlp
from paper_2407_11388_b300 import learned

from cases import full_word, tuned_tightness
from gpu_helpers import from_dev, oracle_enforce, to_dev, torch

pytestmark = pytest.mark.gpu


def _random_net(seed, n, d, density, tight):
    """A random network drawn with numpy (independent of racgen)."""
    rng = np.random.default_rng(seed)
    pairs = [(x, y) for x in range(n) for y in range(x + 1, n) if rng.random() < density]
    scope = np.array([(x, y) if rng.random() < 0.5 else (y, x) for x, y in pairs],
                     np.int32).reshape(-1, 2)
    bits = rng.random((len(pairs), d, d)) >= tight
    rel = (bits * (1 << np.arange(d, dtype=np.uint64))).sum(2).astype(np.uint32)
    return scope, rel


def _states(seed, n, d, count):
    """Assignment-like states: 1-3 variables reduced to a single value, plus
    one state with every domain randomly restricted."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count - 1):
        dom = np.full(n, full_word(d), np.uint32)
        for x in rng.choice(n, size=1 + s % 3, replace=False):
            dom[x] = np.uint32(1 << int(rng.integers(d)))
        out.append(dom)
    keep = rng.random((n, d)) < 0.85
    dom = (keep * (1 << np.arange(d, dtype=np.uint64))).sum(1).astype(np.uint32)
    dom[dom == 0] = 1
    out.append(dom)
    return np.array(out, np.uint32)


def _run_learned(net, doms, pred=None, thr=0.0, cap=0, flags=0, max_sweeps=0):
    T = torch()
    B, n = doms.shape
    din = to_dev(doms.reshape(-1))
    dout = T.empty_like(din)
    sw = T.full((B,), -7, dtype=T.int32, device="cuda:0")
    st = T.full((B,), -7, dtype=T.int32, device="cuda:0")
    trace = rac.Trace(cap)
    rac.enforce_learned(net, din, dout, sw, st, predictor=pred, threshold=thr, trace=trace,
                        flags=flags, max_sweeps=max_sweeps)
    T.cuda.synchronize()
    return (from_dev(dout).reshape(B, n), sw.cpu().numpy(), st.cpu().numpy(), trace)


def _assert_exact(out, st, ref, what):
    ro, ri, rs = ref
    bad = np.flatnonzero(np.any(out != ro, axis=1) | (st != rs))
    assert bad.size == 0, "%s: states %s differ from the oracle" % (what, bad[:5].tolist())


# ---------------------------------------------------------------------------
# the predictor's kernels against the float64 reference
# ---------------------------------------------------------------------------

def _samples(seed, N):
    rng = np.random.default_rng(seed)
    X = rng.random((N, 8)).astype(np.float32)
    X[:, 0] = rng.integers(1, 17, N) / 16.0
    Y = (rng.random(N) < 0.35).astype(np.float32)
    return X, Y


@pytest.mark.parametrize("N", [1, 37, 2048])
def test_gradient_matches_float64(N):
    T = torch()
    X, Y = _samples(N, N)
    pred = rac.Predictor(seed=5)
    w = pred.get_weights(bf16=True).astype(np.float64)
    grad, loss = pred.gradient(T.from_numpy(X).cuda(), T.from_numpy(Y).cuda(), pos_weight=3.0)
    ref_loss, ref = mlp.loss_and_grad(w, X, Y, pos_weight=3.0, bf16=True)
    assert abs(loss - ref_loss) <= 1e-4 * max(1.0, abs(ref_loss))
    scale = np.abs(ref).max()
    err = np.abs(grad - ref)
    assert np.all(err <= 2e-3 * np.abs(ref) + 1e-4 * scale), (err.max(), scale)


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_logits_match_float64(tensor_cores):
    T = torch()
    X, _ = _samples(9, 1000)  # 1000: a partial last warp for the tensor-core routine
    pred = rac.Predictor(seed=3)
    w = pred.get_weights(bf16=True).astype(np.float64)
    z = T.empty(X.shape[0], dtype=T.float32, device="cuda:0")
    pred.predict(T.from_numpy(X).cuda(), z, tensor_cores=tensor_cores)
    ref, _ = mlp.forward(w, X, bf16=True)
    err = np.abs(z.cpu().numpy() - ref)
    assert np.all(err <= 2e-3 * (1.0 + np.abs(ref))), err.max()


def test_weights_round_trip_and_training_learns():
    T = torch()
    pred = rac.Predictor(seed=1)
    w0 = pred.get_weights()
    assert w0.shape == (rac.PREDICTOR_PARAMS,) and np.all(w0[-1:] == 0.0)
    pred.set_weights(w0 * 0.5)
    assert np.array_equal(pred.get_weights(), (w0 * 0.5).astype(np.float32))
    # a separable problem: y = [f1 + f2 > 1]
    rng = np.random.default_rng(2)
    X = rng.random((20000, 8)).astype(np.float32)
    Y = (X[:, 1] + X[:, 2] > 1.0).astype(np.float32)
    x, y = T.from_numpy(X).cuda(), T.from_numpy(Y).cuda()
    _, loss0 = pred.gradient(x, y)
    pred.train(x, y, steps=600, batch=2048, lr=3e-3, seed=4)
    _, loss1 = pred.gradient(x, y)
    z = learned.logits(pred, x).cpu().numpy()
    acc = np.mean((z > 0) == (Y > 0.5))
    assert loss1 < 0.5 * loss0 and acc > 0.95, (loss0, loss1, acc)


# ---------------------------------------------------------------------------
# trace records of the Proposition-2 recurrence against the oracle
# ---------------------------------------------------------------------------

TRACE_CASES = [(100, 12, 0.5, 0.2), (100, 20, 0.6, 0.1), (45, 5, 0.7, 0.15)]


@pytest.mark.parametrize("n,d,dens,c,B", [case + (6,) for case in TRACE_CASES] +
                         [TRACE_CASES[2] + (70,)])
def test_trace_matches_oracle(n, d, dens, c, B):
    """B = 70: three 32-state chunks per slab, each split over the group's
    warps its own way in late sweeps."""
    scope, rel = _random_net(n * 7 + d, n, d, dens, tuned_tightness(n, d, dens, c))
    doms = _states(d, n, d, B)
    with rac.Network(n, d, scope, rel) as net:
        rows = net.info()["rows_per_slab"]
        out, sw, st, trace = _run_learned(net, doms, cap=200000)
    ref = oracle_enforce(n, d, scope, rel, doms)
    _assert_exact(out, st, ref, "trace mode")
    assert np.array_equal(sw, ref[1]), "trace mode sweeps %s oracle %s" % (sw, ref[1])
    idx = gating.SlabIndex(n, d, scope, rel, rows)
    want = {}
    for s in range(doms.shape[0]):
        _, it, _, tr, _ = oracle.rac(n, d, scope, rel, doms[s], trace=True)
        seq = [doms[s]] + list(tr)
        for k in range(1, it + 1):
            # sweep 1: every pair is a candidate, and a variable counts as
            # changed when its input domain is not full
            changed = (seq[0] != full_word(d)) if k == 1 else (seq[k - 2] != seq[k - 1])
            for key in idx.keys:
                if k == 1 or gating.candidate(idx, key, changed):
                    want[(k, s) + key] = (gating.label(idx, key, seq[k - 1]),
                                          gating.features(idx, key, k, changed, seq[k - 1]))
    assert trace.count() == len(want) and len(want) > 0
    rec = trace.records()
    got = {}
    for f, lab, w in zip(rec["features"], rec["label"], rec["where"]):
        assert (w[0] >> 30) == 0  # no gated phase without a predictor
        key = (int(w[0]), int(w[1]), int(w[2]) & 0xFFFF, int(w[2]) >> 16, int(w[3]) & 0xFF)
        assert int(w[3]) >> 8 == rows
        got[key] = (lab, f)
    assert set(got) == set(want)
    for key, (lab, f) in got.items():
        wl, wf = want[key]
        assert lab == (1.0 if wl else 0.0), key
        assert np.allclose(f, wf, rtol=0, atol=2e-7), (key, f, wf)
    # every candidate was evaluated (sweep 1: every slab)
    assert trace.evaluated() == len(want)
    assert sum(1 for key in want if key[0] == 1) == len(idx.keys) * doms.shape[0]


# ---------------------------------------------------------------------------
# learned gating: exact results
# ---------------------------------------------------------------------------

LEARNED_CASES = [(100, 12, 0.5, 0.2), (130, 20, 0.6, 0.1), (64, 32, 0.8, 0.05)]


@pytest.mark.parametrize("n,d,dens,c", LEARNED_CASES)
def test_learned_exact_at_the_extremes(n, d, dens, c):
    scope, rel = _random_net(n * 3 + d, n, d, dens, tuned_tightness(n, d, dens, c))
    doms = _states(n + d, n, d, 8)
    ref = oracle_enforce(n, d, scope, rel, doms)
    K = ref[1]
    assert K.max() >= 3, "the case should cascade"
    pred = rac.Predictor(seed=7)
    with rac.Network(n, d, scope, rel) as net:
        _, _, _, tr_p2 = _run_learned(net, doms, None)
        out, sw, st, tr = _run_learned(net, doms, pred, thr=-np.inf)
        _assert_exact(out, st, ref, "threshold -inf")
        assert np.array_equal(sw, K), (sw, K)
        assert tr.evaluated() == tr_p2.evaluated()
        out, sw, st, _ = _run_learned(net, doms, pred, thr=-np.inf, flags=rac.VERIFY_FULL)
        _assert_exact(out, st, ref, "threshold -inf, full verification")
        assert np.array_equal(sw, K + 1), (sw, K)
        for flags in (0, rac.VERIFY_FULL):
            out, sw, st, _ = _run_learned(net, doms, pred, thr=np.inf, flags=flags)
            _assert_exact(out, st, ref, "threshold +inf, flags %d" % flags)
            assert np.array_equal(sw, 2 * K), (flags, sw, K)


@pytest.mark.parametrize("n,d,dens,c", LEARNED_CASES)
def test_learned_exact_and_kernel_logits(n, d, dens, c):
    T = torch()
    scope, rel = _random_net(n * 5 + d, n, d, dens, tuned_tightness(n, d, dens, c))
    doms = _states(2 * n + d, n, d, 8)
    ref = oracle_enforce(n, d, scope, rel, doms)
    for seed, flags in ((1, 0), (2, rac.VERIFY_FULL), (3, 0)):
        pred = rac.Predictor(seed=seed)
        w = pred.get_weights(bf16=True).astype(np.float64)
        with rac.Network(n, d, scope, rel) as net:
            # a threshold near the middle of this predictor's logits
            xs, _, _ = learned.collect_traces([(net, T.from_numpy(doms.view(np.int32)).cuda())])
            thr = float(np.median(learned.logits(pred, xs).cpu().numpy())) if xs.shape[0] else 0.0
            out, sw, st, trace = _run_learned(net, doms, pred, thr=thr, cap=300000, flags=flags)
        _assert_exact(out, st, ref, "predictor seed %d flags %d" % (seed, flags))
        assert np.all(sw >= ref[1])  # gated states stay supersets of the plain ones
        rec = trace.records()
        assert rec["label"].shape[0] == trace.count() > 0
        gated = (rec["where"][:, 0] >> 30) == 1
        z = rec["logit"]
        # decisions follow the kernel's own logits
        assert np.all((rec["label"][gated] == -1.0) == (z[gated] <= np.float32(thr)))
        assert np.all(rec["label"][~gated] >= 0.0)
        # and those logits are the MLP's (BF16 operands, FP32 accumulation)
        zref, _ = mlp.forward(w, rec["features"], bf16=True)
        err = np.abs(z - zref)
        assert np.all(err <= 2e-3 * (1.0 + np.abs(zref))), err.max()


@pytest.mark.parametrize("B", [48, 80])
def test_learned_many_states(B):
    """Learned gating with several 32-state chunks per slab: exact results and
    every trace label equal to whether the evaluation removed a value, with a
    random predictor and without one (the Proposition-2 recurrence)."""
    T = torch()
    n, d, dens, c = 100, 12, 0.5, 0.2
    scope, rel = _random_net(n * 11 + B, n, d, dens, tuned_tightness(n, d, dens, c))
    doms = _states(3 * n + B, n, d, B)
    ref = oracle_enforce(n, d, scope, rel, doms)
    with rac.Network(n, d, scope, rel) as net:
        for pred in (None, rac.Predictor(seed=B)):
            thr = 0.0
            if pred is not None:
                xs, _, _ = learned.collect_traces([(net, T.from_numpy(doms.view(np.int32)).cuda())])
                thr = float(np.median(learned.logits(pred, xs).cpu().numpy()))
            out, sw, st, trace = _run_learned(net, doms, pred, thr=thr, cap=300000)
            _assert_exact(out, st, ref, "B=%d predictor %s" % (B, pred is not None))
            rec = trace.records()
            assert rec["label"].shape[0] == trace.count() > 0
            assert np.all(np.isin(rec["label"], (-1.0, 0.0, 1.0)))


def test_learned_stop_on_wipeout():
    n, d, dens = 90, 10, 0.6
    scope, rel = _random_net(77, n, d, dens, tuned_tightness(n, d, dens, 0.3))
    doms = _states(78, n, d, 10)
    ref_stop = oracle_enforce(n, d, scope, rel, doms, flags=rac.STOP_ON_WIPEOUT)
    ref = oracle_enforce(n, d, scope, rel, doms)
    assert np.any(ref_stop[2] == rac.WIPEOUT)
    for flags in (rac.STOP_ON_WIPEOUT, rac.STOP_ON_WIPEOUT | rac.VERIFY_FULL):
        with rac.Network(n, d, scope, rel) as net:
            out, sw, st, _ = _run_learned(net, doms, rac.Predictor(seed=4), thr=0.0, flags=flags)
        assert np.array_equal(st, ref_stop[2])
        for s in range(doms.shape[0]):
            # a sound superset of D_ac; a wiped state holds an empty domain
            assert np.all((out[s] & ref[0][s]) == ref[0][s])
            assert np.all((out[s] & ~doms[s]) == 0)
            if st[s] == rac.WIPEOUT:
                assert np.any(out[s] == 0)
            else:
                assert np.array_equal(out[s], ref[0][s])


def test_learned_sweep_cap_and_empty_batch():
    T = torch()
    n, d, dens = 80, 8, 0.6
    scope, rel = _random_net(91, n, d, dens, tuned_tightness(n, d, dens, 0.2))
    doms = _states(92, n, d, 4)
    ref = oracle_enforce(n, d, scope, rel, doms)
    with rac.Network(n, d, scope, rel) as net:
        for flags in (0, rac.VERIFY_FULL):
            out, sw, st, _ = _run_learned(net, doms, rac.Predictor(seed=1), thr=np.inf,
                                          max_sweeps=2, flags=flags)
            # sweep 1 skips everything, sweep 2 is plain sweep 1
            for s in range(doms.shape[0]):
                assert sw[s] == 2
                assert st[s] == (ref[2][s] if ref[1][s] == 1 else rac.ETIMEOUT)
        empty = T.empty(0, dtype=T.int32, device="cuda:0")
        rac.enforce_learned(net, empty, empty, empty, empty, predictor=None, n_states=0)


# ---------------------------------------------------------------------------
# what the trained predictor gains
# ---------------------------------------------------------------------------

def _racgen_items(T, specs):
    import racgen
    items = []
    for seed, inst, n, d, p, t, B in specs:
        net = racgen.random_network(seed, inst, n, d, p, t)
        doms = np.array([racgen.assignment_state(seed, inst, s, n, d) for s in range(B)],
                        np.uint32)
        items.append((net, doms))
    return items


def test_trained_predictor_saves_evaluations():
    """Trained on traces of the n=500 d=20 dense generator and of the batch
    generator (other networks, other seeds), evaluated on the n=1000 d=24
    network with 32 assignment states: same D_ac and status as the oracle,
    fewer (slab, state) evaluations than plain RAC."""
    import racgen
    T = torch()
    train_specs = [(11, 0, 500, 20, 1.0, 0.35, 32)]
    train_specs += [(11, i) + tuple(racgen.batch_params(11, i)) + (16,) for i in range(6)]
    nets = []
    items = []
    for net_np, doms in _racgen_items(T, train_specs):
        net = rac.Network(net_np.n, net_np.d, net_np.scope, net_np.rel)
        nets.append(net)
        items.append((net, T.from_numpy(doms.view(np.int32)).cuda()))
    x, y, _ = learned.collect_traces(items)
    assert x.shape[0] > 10000 and 0.02 < float(y.mean()) < 0.98
    pred = learned.train(x, y, steps=3000, batch=4096, lr=2e-3, pos_weight=4.0, seed=1)
    thr = learned.choose_threshold(pred, x, y, recall=0.98)
    for net in nets:
        net.close()

    (ev_np, doms), = _racgen_items(T, [(0, 0, 1000, 24, 0.8, 0.3, 32)])
    n, d = ev_np.n, ev_np.d
    ref = oracle_enforce(n, d, ev_np.scope, ev_np.rel, doms)
    with rac.Network(n, d, ev_np.scope, ev_np.rel) as net:
        slabs = net.info()["n_slabs"]
        out, sw, st, tr = _run_learned(net, doms, pred, thr=thr)
        _assert_exact(out, st, ref, "trained predictor")
        learned_evals = tr.evaluated()
        out, sw_f, st, tr_f = _run_learned(net, doms, pred, thr=thr, flags=rac.VERIFY_FULL)
        _assert_exact(out, st, ref, "trained predictor, full verification")
        full_evals = tr_f.evaluated()
        _, sw_i, _, tr_i = _run_learned(net, doms, None)
        incr_evals = tr_i.evaluated()
    plain_evals = int(ref[1].sum()) * slabs
    print("evaluations: plain %d, Proposition 2 %d, learned %d (full verification %d); "
          "sweeps plain %d learned %d (%d)" % (plain_evals, incr_evals, learned_evals, full_evals,
                                             ref[1].max(), sw.max(), sw_f.max()))
    assert learned_evals < 0.9 * plain_evals, (learned_evals, plain_evals)
    assert learned_evals < incr_evals, (learned_evals, incr_evals)
