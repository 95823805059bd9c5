"""Randomised parity sweep (GPU): seeded draws of every knob the library
takes at once -- n, d, density, a tightness near the point where removals
cascade, the number and kind of states, the enforce flags, the sweep cap,
the tile rows, the grid cap and the entry point (rac_enforce,
rac_enforce_batch, rac_enforce_host, rac_enforce_noalloc, a multi-network
plan) -- each case compared bit for bit with the oracle on domains, sweep
counts and statuses."""
import numpy as np
import pytest

import racgen
import paper_2407_11388_b300 as rac
from paper_2407_11388_b300.autotune import admissible_rows
from cases import mixed_states, tuned_tightness
from gpu_helpers import assert_same, from_dev, oracle_enforce, to_dev, torch

pytestmark = pytest.mark.gpu

N_CASES = 48


def _draw(i):
    rng = np.random.default_rng(9000 + i)
    n = int(rng.choice([2, 5, 31, 33, 64, 97, 150, 333, 600, 900]))
    d = int(rng.integers(1, 33))
    dens = float(rng.choice([0.0, 0.1, 0.4, 0.8, 1.0]))
    tight = tuned_tightness(n, d, max(dens, 0.05), float(rng.choice([0.005, 0.05, 0.3, 1.0])))
    B = int(rng.choice([1, 1, 2, 3, 5, 17, 40]))
    flags = int(rng.choice([0, rac.INCREMENTAL, rac.STOP_ON_WIPEOUT,
                            rac.INCREMENTAL | rac.STOP_ON_WIPEOUT]))
    cap = int(rng.choice([0, 0, 0, 2, 5]))
    rows = rng.choice(admissible_rows(d) + [None, None])
    ctas = rng.choice([None, None, 1, 3, 64])
    entry = str(rng.choice(["enforce", "batch", "host", "noalloc", "plan"]))
    return rng, n, d, dens, tight, B, flags, cap, rows, ctas, entry


def _states(rng, seed, n, d, B):
    pool = list(mixed_states(rng, n, d))
    pool += [racgen.assignment_state(seed, 0, s, n, d) for s in range(B)]
    pick = rng.choice(len(pool), size=B, replace=True)
    return np.array([pool[j] for j in pick], np.uint32)


@pytest.mark.parametrize("i", range(N_CASES))
def test_random_configuration(i):
    rng, n, d, dens, tight, B, flags, cap, rows, ctas, entry = _draw(i)
    x = racgen.random_network(9000 + i, 0, n, d, dens, tight)
    doms = _states(rng, 9000 + i, n, d, B)
    want = oracle_enforce(n, d, x.scope, x.rel, doms, flags=flags, max_sweeps=cap)
    what = "case %d: n=%d d=%d density %.1f B=%d flags %d cap %d rows %s ctas %s %s" % (
        i, n, d, dens, B, flags, cap, rows, ctas, entry)
    T = torch()
    with rac.Network(n, d, x.scope, x.rel, rows=None if rows is None else int(rows),
                     max_ctas=None if ctas is None else int(ctas)) as net:
        if entry == "host":
            out, it, st = rac.enforce_host(net, doms, max_sweeps=cap, flags=flags)
            assert_same((out.reshape(B, n), it, st), want, what)
            return
        if entry == "noalloc" or (entry == "enforce" and B == 1):
            for s in range(B):
                din = to_dev(doms[s])
                dout = T.empty_like(din)
                it = T.empty(1, dtype=T.int32, device="cuda:0")
                st = T.empty(1, dtype=T.int32, device="cuda:0")
                fn = rac.enforce_noalloc if entry == "noalloc" else rac.enforce
                fn(net, din, dout, it, st, max_sweeps=cap, flags=flags)
                T.cuda.synchronize()
                got = (from_dev(dout)[None, :], it.cpu().numpy(), st.cpu().numpy())
                assert_same(got, tuple(a[s:s + 1] for a in want), what)
            return
        din = to_dev(doms.reshape(-1))
        dout = T.empty_like(din)
        it = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        st = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        items = np.zeros(B, np.int32)
        offs = np.arange(B, dtype=np.int64) * n
        if entry == "plan":
            # a second network of another shape in the same launch
            y = racgen.random_network(9500 + i, 0, 40, 7, 0.5, 0.45)
            with rac.Network(40, 7, y.scope, y.rel) as net2:
                ydom = racgen.assignment_state(9500 + i, 0, 0, 40, 7)
                flat = np.concatenate([doms.reshape(-1), ydom]).astype(np.uint32)
                din = to_dev(flat)
                dout = T.empty_like(din)
                it = T.full((B + 1,), -7, dtype=T.int32, device="cuda:0")
                st = T.full((B + 1,), -7, dtype=T.int32, device="cuda:0")
                items2 = np.concatenate([items, [1]]).astype(np.int32)
                offs2 = np.concatenate([offs, [B * n]]).astype(np.int64)
                with rac.Plan([net, net2], items2, offs2) as plan:
                    plan.enforce(din, dout, it, st, max_sweeps=cap, flags=flags)
                T.cuda.synchronize()
                out = from_dev(dout)
                got = (out[:B * n].reshape(B, n), it.cpu().numpy()[:B], st.cpu().numpy()[:B])
                assert_same(got, want, what)
                w2 = oracle_enforce(40, 7, y.scope, y.rel, ydom, flags=flags, max_sweeps=cap)
                assert_same((out[B * n:][None, :], it.cpu().numpy()[B:], st.cpu().numpy()[B:]),
                            w2, what + " (second network)")
            return
        rac.enforce_batch([net], items, offs, din, dout, it, st, max_sweeps=cap, flags=flags)
        T.cuda.synchronize()
        got = (from_dev(dout).reshape(B, n), it.cpu().numpy(), st.cpu().numpy())
        assert_same(got, want, what)


@pytest.mark.parametrize("i", range(24))
def test_random_configuration_tensor(i):
    """The same draws through the tensor-core kernel (RAC_KERNEL_TENSOR) with
    its operand store built from whole-word or packed rows of any tile
    height, through rac_enforce, rac_enforce_batch and rac_enforce_host."""
    rng, n, d, dens, tight, B, flags, cap, rows, ctas, _ = _draw(i)
    packed = bool(rng.integers(0, 2))
    entry = str(rng.choice(["enforce", "batch", "host"]))
    x = racgen.random_network(9000 + i, 0, n, d, dens, tight)
    doms = _states(rng, 9000 + i, n, d, B)
    want = oracle_enforce(n, d, x.scope, x.rel, doms, flags=flags, max_sweeps=cap)
    what = "tensor case %d: n=%d d=%d density %.1f B=%d flags %d cap %d rows %s packed %s %s" % (
        i, n, d, dens, B, flags, cap, rows, packed, entry)
    fl = flags | rac.KERNEL_TENSOR
    T = torch()
    with rac.Network(n, d, x.scope, x.rel, rows=None if rows is None else int(rows),
                     packed=packed) as net:
        if entry == "host":
            out, it, st = rac.enforce_host(net, doms, max_sweeps=cap, flags=fl)
            assert_same((out.reshape(B, n), it, st), want, what)
            return
        if entry == "enforce":
            for s in range(B):
                din = to_dev(doms[s])
                dout = T.empty_like(din)
                it = T.empty(1, dtype=T.int32, device="cuda:0")
                st = T.empty(1, dtype=T.int32, device="cuda:0")
                rac.enforce(net, din, dout, it, st, max_sweeps=cap, flags=fl)
                T.cuda.synchronize()
                got = (from_dev(dout)[None, :], it.cpu().numpy(), st.cpu().numpy())
                assert_same(got, tuple(a[s:s + 1] for a in want), what)
            return
        din = to_dev(doms.reshape(-1))
        dout = T.empty_like(din)
        it = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        st = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        rac.enforce_batch([net], np.zeros(B, np.int32), np.arange(B, dtype=np.int64) * n, din,
                          dout, it, st, max_sweeps=cap, flags=fl)
        T.cuda.synchronize()
        got = (from_dev(dout).reshape(B, n), it.cpu().numpy(), st.cpu().numpy())
        assert_same(got, want, what)
