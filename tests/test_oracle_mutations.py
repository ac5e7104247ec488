"""The oracle's pins have teeth: each plausible mistake planted in a copy of
the oracle's C source (a dropped term, a transposed operand, an off-by-one,
a wrong sign) makes at least one pin of ``oracle_pins`` fail.

A mistake in the gap heuristic alone is not in the list: the oracle only
stops after a fresh global relabel finds no active vertex, and that BFS
recomputes every height the gap step touched, so such a mistake can cost time
but cannot change a result.

Mutants are compiled into a temporary directory and run in a child process
with a 20 s limit (the unmutated pins take about 2 s), so a mutant that
loops forever also counts as caught.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "maxflow_oracle.c")

# (name, text to find, replacement, which occurrence (0 = first))
MUTANTS = [
    ("push_drops_reverse_residual", "g->res[a ^ 1] += d;\n            P->e[u] -= d;",
     "g->res[a ^ 1] += 0;\n            P->e[u] -= d;", 0),
    ("preflow_halves_excess", "P.e[g.head[a]] += d;", "P.e[g.head[a]] += d / 2;", 0),
    ("global_relabel_uses_forward_arc", "if (g->res[a ^ 1] > 0) {        /* residual arc v -> w exists */",
     "if (g->res[a] > 0) {", 0),
    ("sink_counted_as_active", "return v != P->s && v != P->t && P->e[v] > 0",
     "return v != P->s && P->e[v] > 0", 0),
    ("relabel_overshoots", "int64_t nh = (minh == INT32_MAX) ? P->cap_height : minh + 1;",
     "int64_t nh = (minh == INT32_MAX) ? P->cap_height : minh + 3;", 0),
    ("flow_output_is_residual", "flow[i] = (k < 0) ? 0 : (int32_t)(cap[i] - g.res[2 * k]);",
     "flow[i] = (k < 0) ? 0 : (int32_t)(g.res[2 * k]);", 0),
    ("cut_bfs_follows_reverse_arc", "if (g.res[a] > 0 && !source_side[v]) {",
     "if (g.res[a ^ 1] > 0 && !source_side[v]) {", 0),
    ("dinic_loses_a_unit", "total += b;", "total += b - (b > 1);", 0),
    ("verifier_value_sign", "if (-bal[s] != value || bal[t] != value)",
     "if (bal[s] != value || bal[t] != value)", 0),
    ("bruteforce_counts_internal_arcs", "if ((S >> src[i] & 1) && !(S >> dst[i] & 1)) c += cap[i];",
     "if ((S >> src[i] & 1) && (S >> dst[i] & 1)) c += cap[i];", 0),
    ("hopcroft_karp_miscounts", "++matched;", "matched += (matched < 3);", 0),
    ("residual_dist_step_two", "dist[v] = dist[w] + 1;", "dist[v] = dist[w] + 2;", 0),
]

CHILD = r"""
import sys
sys.path.insert(0, %r)
from tests import oracle_pins as P
for pin in P.ALL_PINS:
    pin()
print("ALL PINS PASSED")
"""


def _replace_nth(text, old, new, nth):
    idx = -1
    for _ in range(nth + 1):
        idx = text.find(old, idx + 1)
        if idx < 0:
            return None
    return text[:idx] + new + text[idx + len(old):]


@pytest.mark.parametrize("name,old,new,nth", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new, nth):
    text = open(SRC).read()
    mutated = _replace_nth(text, old, new, nth)
    assert mutated is not None, f"mutation site for {name} not found"
    csrc = tmp_path / "mut.c"
    csrc.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(csrc)])
    env = dict(os.environ, ORACLE_SO=str(so))
    try:
        r = subprocess.run([sys.executable, "-c", CHILD % ROOT], env=env, capture_output=True,
                           text=True, timeout=20)
        caught = r.returncode != 0
    except subprocess.TimeoutExpired:
        caught = True
    assert caught, f"mutant {name} passed every pin"


def test_unmutated_oracle_passes_child_harness(tmp_path):
    r = subprocess.run([sys.executable, "-c", CHILD % ROOT], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "ALL PINS PASSED" in r.stdout, r.stderr[-2000:]
