"""Invariants of the push-relabel state at the quiescent points of a solve
(after the preflow, after a global relabel, after a number of push-relabel
iterations, and after a full solve), read from exported snapshots:

* every residual pair keeps its total: cf(u,v) + cf(v,u) = c(u,v) + c(v,u)
  (BCSR), or cf + flow = c per arc (RCSR), and no residual is negative;
* no excess is negative, and the excess of every vertex is what the flows
  into and out of it leave (Alg. 1: pushes move excess along arcs and the
  preflow creates it at s's neighbours without charging s);
* after phase 2 only s and t hold excess, and t's is the flow value.

The same state is compared with the oracle elsewhere at the end of a solve;
these checks hold at every step in between, whatever the schedule."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import LAYOUTS, layout_code, wb

pytestmark = pytest.mark.gpu


def _check_state(m, G, n, s, layout, preflow_total):
    off = m.wbpr_export(G, "offsets")
    rows = np.repeat(np.arange(n), np.diff(off))
    col = m.wbpr_export(G, "col").astype(np.int64)
    cf = m.wbpr_export(G, "cf").astype(np.int64)
    cap0 = m.wbpr_export(G, "cap").astype(np.int64)
    e = m.wbpr_export(G, "excess")
    assert (e >= 0).all()
    if layout == "bcsr":
        rev = m.wbpr_export(G, "rev").astype(np.int64)
        pair = cap0 + cap0[rev]
        assert np.array_equal(cf + cf[rev], pair)
        assert (cf >= 0).all() and (cf <= pair).all()
        # net flow out of the row's vertex along slot a is cap0[a] - cf[a]
        bal = np.zeros(n, np.int64)
        np.add.at(bal, rows, cf - cap0)
    else:
        bf = m.wbpr_export(G, "bf").astype(np.int64)
        assert np.array_equal(cf + bf, cap0)
        assert (bf >= 0).all() and (cf >= 0).all()
        bal = np.zeros(n, np.int64)
        np.add.at(bal, col, bf)
        np.subtract.at(bal, rows, bf)
    bal[s] += preflow_total
    assert np.array_equal(e, bal)
    assert int(e.sum()) == preflow_total
    return e


@pytest.mark.parametrize("multi_push", [1, 0])
@pytest.mark.parametrize("layout", LAYOUTS)
def test_state_invariants_at_every_stage(layout, multi_push):
    m = wb()
    g = W.rmat(11, 8, 9)
    src, dst, cap = g.numpy()
    n, s, t = g.n, g.s, g.t
    o = m.wbpr_default_options()
    o.multi_push = multi_push
    G = m.wbpr_build(n, src.size, src, dst, cap, s, t, layout_code(layout), o)
    preflow_total = int(cap[(src == s) & (dst != s)].astype(np.int64).sum())
    m.wbpr_run_stage(G, 1)                      # preflow
    assert int(m.wbpr_export(G, "excess_total")[0]) == preflow_total
    _check_state(m, G, n, s, layout, preflow_total)
    for rounds in (3, 25, 200):
        m.wbpr_run_stage(G, 2)                  # one global relabel
        _check_state(m, G, n, s, layout, preflow_total)
        m.wbpr_run_stage(G, 3, rounds)          # push-relabel iterations
        _check_state(m, G, n, s, layout, preflow_total)
    flow = np.zeros(src.size, np.int32)
    value = m.wbpr_maxflow(G, None, flow)       # phases 1 and 2 from a fresh preflow
    e = _check_state(m, G, n, s, layout, preflow_total)
    others = np.ones(n, bool)
    others[[s, t]] = False
    assert (e[others] == 0).all()
    assert int(e[t]) == value and int(e[s]) == preflow_total - value
    G.close()
