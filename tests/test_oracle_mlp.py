"""Pins of the float64 predictor reference and of the gating definitions
(oracle/mlp.py, oracle/gating.py) against facts that do not come from
themselves: the bfloat16 format, closed forms of hand-set weights, finite
differences of the loss, the C oracle's Eq. 1 sweep, and Proposition 2."""
import numpy as np
import pytest

import oracle
from oracle import gating, mlp


def test_bf16_rounding_fixed_by_the_format():
    # spacing of bfloat16 at 1 is 2^-7; halfway cases go to the even significand
    cases = {
        1.0: 1.0,
        1.0 + 2.0 ** -8: 1.0,                       # tie -> even (down)
        1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,       # tie -> even (up)
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,
        -(1.0 + 2.0 ** -8 + 2.0 ** -20): -(1.0 + 2.0 ** -7),
        0.1: 0.10009765625,                         # float32 0x3DCCCCCD -> 0x3DCD
        3.0: 3.0,
        0.0: 0.0,
        2.0 ** -130: 2.0 ** -130,                   # float32 subnormal, exact
    }
    for v, want in cases.items():
        assert mlp.bf16_round(np.array([v]))[0] == want, v


def _hand_params():
    W1 = np.zeros((64, 8)); b1 = np.zeros(64); W2 = np.zeros((64, 64)); b2 = np.zeros(64)
    w3 = np.zeros(64)
    W1[0, 0] = 1.0
    W1[1, 1] = -1.0
    b1[1] = 0.5
    W2[0, 0] = 2.0
    W2[3, 1] = 1.0
    w3[0] = 3.0
    w3[3] = -2.0
    return mlp.pack(W1, b1, W2, b2, w3, -1.0)


def test_forward_closed_form():
    # z = 3 * relu(2 relu(x0)) - 2 * relu(relu(0.5 - x1)) - 1
    p = _hand_params()
    X = np.zeros((4, 8))
    X[:, 0] = [0.5, -1.0, 0.25, 2.0]
    X[:, 1] = [0.0, 0.25, 1.0, 0.5]
    want = 6 * np.maximum(X[:, 0], 0) - 2 * np.maximum(0.5 - X[:, 1], 0) - 1
    for bf16 in (False, True):  # every value here is exact in bfloat16
        z, _ = mlp.forward(p, X, bf16=bf16)
        assert np.array_equal(z, want)


def test_loss_closed_form_at_zero_weights():
    # z = 0 everywhere: l = w(y) log 2, dL/db3 = mean w(y) (1/2 - y), rest 0
    rng = np.random.default_rng(0)
    X = rng.random((50, 8))
    Y = (rng.random(50) < 0.3).astype(float)
    pw = 3.0
    loss, g = mlp.loss_and_grad(np.zeros(mlp.N_PARAMS), X, Y, pos_weight=pw)
    w = np.where(Y > 0.5, pw, 1.0)
    assert np.isclose(loss, np.mean(w) * np.log(2.0), rtol=1e-14)
    assert np.isclose(g[-1], np.mean(w * (0.5 - Y)), rtol=1e-14)
    assert np.all(g[:-1] == 0.0)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.4, mlp.N_PARAMS)
    X = rng.random((40, 8))
    Y = (rng.random(40) < 0.4).astype(float)
    _, g = mlp.loss_and_grad(p, X, Y, pos_weight=2.5, bf16=False)
    eps = 1e-6
    for i in rng.choice(mlp.N_PARAMS, 60, replace=False).tolist() + [mlp.N_PARAMS - 1]:
        e = np.zeros_like(p)
        e[i] = eps
        lp, _ = mlp.loss_and_grad(p + e, X, Y, pos_weight=2.5, bf16=False)
        lm, _ = mlp.loss_and_grad(p - e, X, Y, pos_weight=2.5, bf16=False)
        num = (lp - lm) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def _random_net(seed, n, d, density, tight):
    rng = np.random.default_rng(seed)
    scope, rel = [], []
    full = (1 << d) - 1
    for x in range(n):
        for y in range(x + 1, n):
            if rng.random() < density:
                a = (x, y) if rng.random() < 0.5 else (y, x)
                scope.append(a)
                rel.append([sum(1 << b for b in range(d) if rng.random() >= tight) & full
                            for _ in range(d)])
    return np.array(scope, np.int32), np.array(rel, np.uint32)


def test_label_is_one_sweep_of_eq1_on_the_slab():
    """label(slab, D) == "the C oracle's single Eq. 1 sweep over only the
    slab's constraints removes something"."""
    n, d = 70, 5
    scope, rel = _random_net(3, n, d, 0.3, 0.3)
    idx = gating.SlabIndex(n, d, scope, rel, rows=8)
    rng = np.random.default_rng(4)
    seen = {True: 0, False: 0}
    for trial in range(6):
        keep = 0.6 + 0.08 * trial                   # values kept with this probability
        bits = rng.random((n, d)) < keep
        D = (bits * (1 << np.arange(d))).sum(1).astype(np.uint32)
        for key in idx.keys:
            cs = idx.members[key]
            out, it, st = oracle.rac(n, d, scope[cs], rel[cs], D, max_sweeps=1)
            want = not np.array_equal(out, D)
            got = gating.label(idx, key, D)
            assert got == want, (trial, key)
            seen[got] += 1
    assert seen[True] > 10 and seen[False] > 10


def test_non_candidates_never_remove():
    """Proposition 2 on the oracle's own trace: at sweep k >= 2 a slab none
    of whose variables changed in sweep k-1 removes nothing."""
    n, d = 200, 5  # sparse and tight: cascades stay local for a few sweeps
    scope, rel = _random_net(5, n, d, 0.04, 0.55)
    idx = gating.SlabIndex(n, d, scope, rel, rows=8)
    rng = np.random.default_rng(6)
    checked = 0
    for s in range(4):
        D0 = np.full(n, (1 << d) - 1, np.uint32)
        for v in rng.choice(n, 2, replace=False):
            D0[v] = 1 << int(rng.integers(d))
        _, it, _, tr, _ = oracle.rac(n, d, scope, rel, D0, trace=True)
        doms = [D0] + list(tr)
        for k in range(2, it + 1):
            changed = doms[k - 2] != doms[k - 1]
            for key in idx.keys:
                if not gating.candidate(idx, key, changed):
                    assert not gating.label(idx, key, doms[k - 1])
                    checked += 1
    assert checked > 100


def test_features_by_hand():
    # n = 40 (blocks 0 and 1), d = 4, rows = 8; constraint (0, 33) with 10 of
    # 16 pairs allowed, constraint (2, 1) (stored as (1, 2)) all allowed
    n, d = 40, 4
    r0 = [0b1111, 0b0011, 0b0101, 0b1000]           # 4 + 2 + 2 + 1 = 9 allowed
    r0[3] |= 0b0001                                 # 10 allowed
    scope = np.array([[0, 33], [2, 1]], np.int32)
    rel = np.array([r0, [0b1111] * 4], np.uint32)
    idx = gating.SlabIndex(n, d, scope, rel, rows=8)
    assert idx.keys == [(0, 0, 0), (0, 1, 0)]
    D = np.full(n, 0b1111, np.uint32)
    D[5] = 0b0001                                   # row variable, |D| = 1
    D[34] = 0b0011                                  # column variable, |D| = 2
    changed = np.zeros(n, bool)
    changed[[2, 7, 35]] = True
    f = gating.features(idx, (0, 1, 0), 3, changed, D)
    want = [3 / 16, 2 / 8, 1 / 32, 1 - 10 / 16, 1 / (8 * 32), 2 / 4,
            (7 * 4 + 2) / (8 * 4), 1 / 4]           # columns 32..39 exist (n = 40)
    assert np.allclose(f, want, rtol=0, atol=1e-15)
    assert gating.candidate(idx, (0, 1, 0), changed)
    changed[:] = False
    changed[20] = True                              # row 20 is outside rows 0..7
    assert not gating.candidate(idx, (0, 1, 0), changed)
