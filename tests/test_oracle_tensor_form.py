"""The dense tensor form of a sweep (pins.tensor_form) on its own: the
regimes the tensor-form pin covers, and where the default mode must differ
from Eq. 1 over the real constraints (no GPU)."""
import numpy as np
import pytest

import oracle
import pins


def test_tensor_form_cases_cover_both_endings_and_cascades():
    seen = {oracle.OK: 0, oracle.WIPEOUT: 0}
    multi_stop = multi_default = 0
    for n, d, scope, rel, dom in pins.tensor_form_cases(21, 400):
        _, it, st = oracle.rac(n, d, scope, rel, dom, stop_on_wipeout=True)
        seen[st] += 1
        multi_stop += it >= 3
        _, it, st = oracle.rac(n, d, scope, rel, dom)
        multi_default += st == oracle.OK and it >= 3
    assert seen[oracle.OK] >= 100 and seen[oracle.WIPEOUT] >= 100, seen
    assert multi_stop >= 40 and multi_default >= 30, (multi_stop, multi_default)


@pytest.mark.parametrize("n,d", [(5, 3), (7, 4)])
def test_dense_form_wipes_everything_after_an_empty_domain(n, d):
    """Why the default mode differs after a wipe-out (reading c5): one empty
    domain makes every all-ones block give a zero count, so the dense form
    empties every domain, while Eq. 1 over the real constraints does not."""
    scope = np.array([[0, 1]], np.int32)
    rel = np.zeros((1, d), np.uint32)  # nothing allowed on (0, 1)
    dom = np.full(n, (1 << d) - 1, np.uint32)
    out_t, _, st_t = pins.tensor_form(n, d, scope, rel, dom, stop_on_wipeout=False)
    out_o, _, st_o = oracle.rac(n, d, scope, rel, dom)
    assert st_t == st_o == oracle.WIPEOUT
    assert (out_t == 0).all()
    assert out_o[0] == 0 and out_o[1] == 0 and (out_o[2:] == (1 << d) - 1).all()
