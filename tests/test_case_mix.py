"""The random parity cases exercise the regimes that matter (no GPU)."""
import numpy as np

import oracle
from cases import width_cases


def test_width_cases_cover_the_regimes():
    """The per-width cases include long cascades, wipe-outs, and fixpoints
    without an empty domain after several sweeps (checked on the oracle)."""
    its, sts = [], []
    for d in range(1, 33):
        for n, scope, rel, doms in width_cases(d):
            for s in range(doms.shape[0]):
                _, it, st = oracle.rac(n, d, scope, rel, doms[s])
                its.append(it)
                sts.append(st)
    its, sts = np.array(its), np.array(sts)
    assert its.max() >= 15
    assert (sts == oracle.WIPEOUT).sum() >= 20
    assert ((sts == oracle.OK) & (its >= 5)).sum() >= 10
