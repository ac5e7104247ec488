"""Vision-style minimum cuts (the image-segmentation use of §1): 4-connected
grids with a source and a sink arc on every pixel.  At 1024 x 1024 (1 M
pixels, 6.3 M arcs) the flow value, cut capacity and canonical cut side are
bit-exact against the oracle and the edge flows are certified, in both
layouts; at 4096 x 4096 (16.8 M pixels, 100 M arcs) the optimality
certificate holds and the GPU's cut side is the one the certificate
computes."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests.gpu_helpers import check_against_oracle, layout_code, wb

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", ["bcsr", "rcsr"])
def test_vision_1024_matches_oracle(layout):
    g = W.vision_grid(1024, 1024, 3)
    src, dst, cap = g.numpy()
    check_against_oracle(g.n, src, dst, cap, g.s, g.t, layout)


@pytest.mark.slow
def test_vision_4096_certificate():
    m = wb()
    g = W.vision_grid(4096, 4096, 7, device="cuda:0")
    G = m.wbpr_build(g.n, g.m, g.src, g.dst, g.cap, g.s, g.t, layout_code("bcsr"))
    flow = torch.empty(g.m, dtype=torch.int32, device="cuda:0")
    side = torch.empty(g.n, dtype=torch.uint8, device="cuda:0")
    value = m.wbpr_maxflow(G, None, flow)
    cut = m.wbpr_mincut(G, None, side)
    st = m.wbpr_get_stats(G)
    print(f"vision 4096x4096: value {value}, phase 1 + 2 {st['solve_ms']:.1f} ms")
    G.close()
    assert value == cut
    src, dst, cap = g.numpy()
    code, c2, S = oracle.verify_flow(g.n, src, dst, cap, g.s, g.t, flow.cpu().numpy(), value)
    assert code == 0 and c2 == value
    assert np.array_equal(S, side.cpu().numpy())
