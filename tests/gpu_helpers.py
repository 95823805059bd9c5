"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the CPU oracle on the same inputs."""
import numpy as np

import oracle
import paper_2407_11388_b300 as rac


def torch():
    import torch as _t
    return _t


def to_dev(a):
    t = torch()
    return t.from_numpy(np.ascontiguousarray(a).view(np.int32)).to("cuda:0")


def from_dev(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_enforce(n, d, scope, rel, doms, flags=0, max_sweeps=0, net=None, shuffle_seed=None):
    """Enforce each row of doms (B, n) on the GPU.  B == 1 goes through
    rac_enforce, B > 1 through rac_enforce_batch (with shuffled offsets when
    shuffle_seed is given).  Returns (dom_out (B, n), iterations, status)."""
    T = torch()
    doms = np.ascontiguousarray(doms, dtype=np.uint32).reshape(-1, n)
    B = doms.shape[0]
    own = net is None
    if own:
        net = rac.Network(n, d, scope, rel)
    try:
        if B == 1:
            din = to_dev(doms[0])
            dout = T.empty_like(din)
            it = T.empty(1, dtype=T.int32, device="cuda:0")
            st = T.empty(1, dtype=T.int32, device="cuda:0")
            rac.enforce(net, din, dout, it, st, max_sweeps=max_sweeps, flags=flags)
            T.cuda.synchronize()
            return from_dev(dout)[None, :], it.cpu().numpy(), st.cpu().numpy()
        slots = np.arange(B)
        if shuffle_seed is not None:
            slots = np.random.default_rng(shuffle_seed).permutation(B)
        packed = np.zeros((B, n), np.uint32)
        packed[slots] = doms
        din = to_dev(packed.reshape(-1))
        dout = T.empty_like(din)
        it = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        st = T.full((B,), -7, dtype=T.int32, device="cuda:0")
        rac.enforce_batch([net], np.zeros(B, np.int32), slots.astype(np.int64) * n, din, dout,
                          it, st, max_sweeps=max_sweeps, flags=flags)
        T.cuda.synchronize()
        out = from_dev(dout).reshape(B, n)[slots]
        return out, it.cpu().numpy(), st.cpu().numpy()
    finally:
        if own:
            net.close()


def oracle_enforce(n, d, scope, rel, doms, flags=0, max_sweeps=0, threads=8):
    doms = np.ascontiguousarray(doms, dtype=np.uint32).reshape(-1, n)
    outs, its, sts = [], [], []
    for s in range(doms.shape[0]):
        o, it, st = oracle.rac(n, d, scope, rel, doms[s],
                               stop_on_wipeout=bool(flags & rac.STOP_ON_WIPEOUT),
                               max_sweeps=max_sweeps, threads=threads)
        outs.append(o)
        its.append(it)
        sts.append(st)
    return np.array(outs, np.uint32), np.array(its, np.int32), np.array(sts, np.int32)


def assert_same(gpu, ref, what=""):
    go, gi, gs = gpu
    ro, ri, rs = ref
    bad = np.flatnonzero(np.any(go != ro, axis=1) | (gi != ri) | (gs != rs))
    if bad.size:
        s = int(bad[0])
        diff = np.flatnonzero(go[s] != ro[s])
        raise AssertionError(
            "%s: %d of %d states differ; state %d: iterations gpu %d oracle %d, status gpu %d "
            "oracle %d, %d domain words differ (first x=%s gpu=%s oracle=%s)" % (
                what, bad.size, go.shape[0], s, gi[s], ri[s], gs[s], rs[s], diff.size,
                diff[:1].tolist(), go[s][diff[:1]].tolist(), ro[s][diff[:1]].tolist()))
