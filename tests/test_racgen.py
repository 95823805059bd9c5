"""The seeded input generator: its documented hashing rule, determinism and
the statistics of the random-CSP model (no GPU)."""
import hashlib

import numpy as np

import racgen

MASK = (1 << 64) - 1


def py_splitmix64(z):
    z = (z + 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def py_key(seed, tag, *fields):
    h = py_splitmix64(seed)
    h = py_splitmix64(h ^ tag)
    for f in fields:
        h = py_splitmix64(h ^ f)
    return h


def u01(h):
    return (h >> 11) * 2.0 ** -53


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0 first returns 0xE220A8397B1DCDAF (Steele, Lea
    # and Flood 2014; the reference stream used by xoshiro's seeding).
    assert racgen.splitmix64(0) == 0xE220A8397B1DCDAF
    for z in (1, 12345, MASK):
        assert racgen.splitmix64(z) == py_splitmix64(z)
    assert racgen.key(5, 2, 1, 2, 3) == py_key(5, 2, 1, 2, 3)


def test_network_follows_the_documented_rule():
    seed, inst, n, d, p, t = 17, 3, 30, 7, 0.4, 0.35
    net = racgen.random_network(seed, inst, n, d, p, t)
    pairs = [(x, y) for x in range(n) for y in range(x + 1, n)
             if u01(py_key(seed, 1, inst, x, y)) < p]
    assert [tuple(s) for s in net.scope.tolist()] == pairs
    for c, (x, y) in enumerate(pairs[:20]):
        P = py_key(seed, 2, inst, x, y)
        for a in range(d):
            want = sum(1 << b for b in range(d)
                       if not u01(py_splitmix64(P ^ ((a << 8) | b))) < t)
            assert int(net.rel[c, a]) == want


def test_deterministic_and_digest_stable():
    a = racgen.random_network(0, 0, 200, 20, 0.5, 0.3)
    b = racgen.random_network(0, 0, 200, 20, 0.5, 0.3)
    assert np.array_equal(a.scope, b.scope) and np.array_equal(a.rel, b.rel)
    c = racgen.random_network(1, 0, 200, 20, 0.5, 0.3)
    assert not (a.m == c.m and np.array_equal(a.rel[:100], c.rel[:100]))
    # bits above d are never set
    assert not np.any(a.rel >> np.uint32(20))


def test_model_statistics():
    net = racgen.random_network(2, 0, 400, 16, 0.6, 0.3)
    pairs = 400 * 399 // 2
    assert abs(net.m / pairs - 0.6) < 0.01
    bits = np.unpackbits(net.rel.view(np.uint8)).reshape(-1)  # 32 bits per row
    allowed = bits.sum() / (net.m * 16 * 16)
    assert abs(allowed - 0.7) < 0.005


def test_batch_params_ranges():
    seen_d = set()
    for inst in range(300):
        n, d, p, t = racgen.batch_params(0, inst)
        assert 50 <= n <= 800 and 8 <= d <= 32 and 0.3 <= p <= 1.0 and 0.2 <= t <= 0.4
        seen_d.add(d)
    assert len(seen_d) == 25


def test_assignment_states():
    for s in range(50):
        dom = racgen.assignment_state(4, 1, s, 60, 12)
        full = (1 << 12) - 1
        assigned = np.flatnonzero(dom != full)
        assert 1 <= len(assigned) <= 5
        for v in assigned:
            assert bin(int(dom[v])).count("1") == 1
    # d = 1: every domain is a singleton already, still k distinct picks
    assert np.all(racgen.assignment_state(4, 1, 0, 3, 1) == 1)


def test_digest_pin():
    """Byte digest of one small instance, so a change of the rule is seen."""
    net = racgen.random_network(0, 0, 50, 10, 0.5, 0.3)
    h = hashlib.sha256(net.scope.tobytes() + net.rel.tobytes()).hexdigest()
    assert net.m == 638
    assert h == DIGEST_50


# sha256 of scope + rel bytes of random_network(0, 0, 50, 10, 0.5, 0.3)
DIGEST_50 = "62fea4eed73582c9acc962a09182656e6e39817d010a3b24218e514e8f0f6c59"
