"""Host-side checks that need no GPU: the C ABI library loads, exports every
function that include/wbpr.h declares, and rejects bad arguments before any
CUDA call; the layout restatements match hand-built examples."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wb():
    import paper_2404_00270_gb300 as wb
    from paper_2404_00270_gb300 import _build
    _build.build()
    wb.load()
    return wb


def _declared():
    text = open(os.path.join(ROOT, "include", "wbpr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wbpr_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree(wb):
    assert _declared() == sorted(wb.EXPORTED_SYMBOLS)


def test_every_declared_symbol_is_exported(wb):
    lib = wb.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_argument_errors_without_gpu(wb):
    with pytest.raises(wb.WbprError) as e:
        wb.wbpr_build(3, 1, [0], [1], [1], 0, 0)          # s == t
    assert e.value.status == -1
    with pytest.raises(wb.WbprError) as e:
        wb.wbpr_build(1, 0, [], [], [], 0, 0)             # n < 2
    assert e.value.status == -1
    with pytest.raises(wb.WbprError) as e:
        wb.wbpr_build(1 << 30, 0, [], [], [], 0, 1)       # n too large
    assert e.value.status == -5
    with pytest.raises(wb.WbprError) as e:
        wb.wbpr_build(4, 1, [0], [1], [1], 0, 1, layout=7)
    assert e.value.status == -1
    o = wb.wbpr_default_options()
    assert o.use_rev == 1 and o.gap == 1 and o.small_tile == 8
    assert o.avq_incremental == 2 and o.lean_build == 0 and o.bottom_up_edges == -1
    o.small_tile = 5
    with pytest.raises(wb.WbprError):
        wb.wbpr_build(4, 1, [0], [1], [1], 0, 1, opts=o)
    # the option ranges are checked before anything touches a device
    for field, bad in [("avq_incremental", 3), ("avq_incremental", -1), ("lean_build", 2),
                       ("bottom_up_edges", 3), ("bottom_up_edges", -2)]:
        o = wb.wbpr_default_options()
        setattr(o, field, bad)
        with pytest.raises(wb.WbprError) as e:
            wb.wbpr_build(4, 1, [0], [1], [1], 0, 1, opts=o)
        assert e.value.status == -1, field
    so = wb.wbpr_server_default_options()
    assert so.build_room == 1
    assert wb.wbpr_error_string(-4).startswith("iteration cap")


def test_layout_restatement_by_hand(oracle_mod):
    from oracle import layouts
    # diamond: 0->1 (3), 0->2 (2), 1->2 (1), 1->3 (2), 2->3 (3)
    src, dst, cap = [0, 0, 1, 1, 2], [1, 2, 2, 3, 3], [3, 2, 1, 2, 3]
    b = layouts.bcsr(4, src, dst, cap)
    # rows: 0:[1,2]  1:[0,2,3]  2:[0,1,3]  3:[1,2]
    assert list(b["offsets"]) == [0, 2, 5, 8, 10]
    assert list(b["col"]) == [1, 2, 0, 2, 3, 0, 1, 3, 1, 2]
    assert list(b["cap"]) == [3, 2, 0, 1, 2, 0, 0, 3, 0, 0]
    assert list(b["rev"]) == [2, 5, 0, 6, 8, 1, 3, 9, 4, 7]
    assert list(b["arc2slot"]) == [0, 1, 3, 4, 7]
    # merged antiparallel pair and duplicates: 0->1 (4), 1->0 (7), 0->1 (2), loop 1->1
    b = layouts.bcsr(2, [0, 1, 0, 1], [1, 0, 1, 1], [4, 7, 2, 9])
    assert list(b["col"]) == [1, 0] and list(b["cap"]) == [6, 7]
    assert list(b["arc2slot"]) == [0, 1, 0, 0xFFFFFFFF]
    r = layouts.rcsr(4, src, dst, cap)
    assert list(r["offsets"]) == [0, 2, 4, 5, 5]
    assert list(r["col"]) == [1, 2, 2, 3, 3]
    assert list(r["in_offsets"]) == [0, 0, 1, 3, 5]
    assert list(r["in_col"]) == [0, 0, 1, 1, 2]
    assert list(r["flow_idx"]) == [0, 1, 2, 3, 4]


def test_layout_restatement_invariants(oracle_mod):
    """The layouts of §3.2 checked from their definition with plain Python
    loops and dictionaries (no sorting or searching shared with the numpy
    restatement), on random graphs with self-loops, duplicates and
    antiparallel pairs: BCSR rows hold every neighbour joined in either
    direction, in increasing id, with the summed capacity of the arcs u -> v,
    rev pairs (u, v) with (v, u) both ways, arc2slot finds each arc's slot;
    RCSR out rows keep the arcs by (head, input position), in rows by (tail,
    out slot), and flow_idx points back at the same arc."""
    import random
    from oracle import layouts
    NONE = 0xFFFFFFFF
    rnd = random.Random(3)
    for trial in range(200):
        n = rnd.randint(2, 30)
        m = rnd.randint(0, 120)
        src = [rnd.randrange(n) for _ in range(m)]
        dst = [rnd.randrange(n) for _ in range(m)]
        cap = [rnd.randint(0, 50) for _ in range(m)]
        b = layouts.bcsr(n, src, dst, cap)
        off, col, bc, rev, a2s = (list(map(int, b[k])) for k in ("offsets", "col", "cap", "rev", "arc2slot"))
        total = {}
        nbrs = [set() for _ in range(n)]
        for u, v, c in zip(src, dst, cap):
            if u != v:
                total[(u, v)] = total.get((u, v), 0) + c
                nbrs[u].add(v)
                nbrs[v].add(u)
        assert off[0] == 0 and off[n] == len(col) == len(bc) == len(rev)
        row_of = {}
        for u in range(n):
            assert off[u] <= off[u + 1]
            row = col[off[u]:off[u + 1]]
            assert row == sorted(nbrs[u]) and len(set(row)) == len(row)
            for k in range(off[u], off[u + 1]):
                row_of[k] = u
                assert bc[k] == total.get((u, col[k]), 0)
        for k in range(len(col)):
            assert row_of[rev[k]] == col[k] and col[rev[k]] == row_of[k] and rev[rev[k]] == k
        for i, (u, v) in enumerate(zip(src, dst)):
            if u == v:
                assert a2s[i] == NONE
            else:
                assert row_of[a2s[i]] == u and col[a2s[i]] == v

        r = layouts.rcsr(n, src, dst, cap)
        off, col, rc, a2s = (list(map(int, r[k])) for k in ("offsets", "col", "cap", "arc2slot"))
        ioff, icol, fidx = (list(map(int, r[k])) for k in ("in_offsets", "in_col", "flow_idx"))
        slot = 0
        out_slot = {}
        for u in range(n):
            arcs = sorted((dst[i], i) for i in range(m) if src[i] == u and dst[i] != u)
            assert off[u] == slot and off[u + 1] == slot + len(arcs)
            for v, i in arcs:
                assert col[slot] == v and rc[slot] == cap[i] and a2s[i] == slot
                out_slot[i] = slot
                slot += 1
        assert off[n] == len(col) == slot
        assert all(a2s[i] == NONE for i in range(m) if src[i] == dst[i])
        pos = 0
        for v in range(n):
            ins = sorted((src[i], out_slot[i]) for i in range(m) if dst[i] == v and src[i] != v)
            assert ioff[v] == pos and ioff[v + 1] == pos + len(ins)
            for u, k in ins:
                assert icol[pos] == u and fidx[pos] == k and col[k] == v
                pos += 1
        assert ioff[n] == pos == len(icol)


def test_no_fallback_without_the_cuda_library():
    """The package has no CPU path: without libwbpr.so every call raises,
    and importing it (and its serving and tuning modules) loads nothing from
    the oracle."""
    import subprocess
    import sys
    code = (
        "import sys\n"
        "import paper_2404_00270_gb300 as wb, paper_2404_00270_gb300.autotune, paper_2404_00270_gb300.serve\n"
        "from paper_2404_00270_gb300 import _build\n"
        "assert not any(k == 'oracle' or k.startswith('oracle.') for k in sys.modules), 'oracle imported'\n"
        "_build.LIB = '/nonexistent/libwbpr.so'\n"
        "try:\n"
        "    wb.wbpr_build(4, 1, [0], [1], [1], 0, 1)\n"
        "except RuntimeError as e:\n"
        "    assert 'not built' in str(e), e\n"
        "    print('raised')\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0 and out.stdout.strip() == "raised", out.stderr[-2000:]
