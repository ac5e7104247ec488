"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare it with the oracle."""
import numpy as np
import pytest
import torch

import oracle

LAYOUTS = ("bcsr", "rcsr")


def wb():
    import paper_2404_00270_gb300 as wb
    wb.load(build_if_missing=True)
    return wb


def layout_code(name):
    m = wb()
    return m.WBPR_BCSR if name == "bcsr" else m.WBPR_RCSR


def gpu_solve(n, src, dst, cap, s, t, layout="bcsr", opts=None, device="cuda:0",
              want_cut=True):
    """Build + maxflow (with edge flows) + mincut through the C ABI."""
    m = wb()
    src_t = torch.as_tensor(np.asarray(src, np.int32), device=device)
    dst_t = torch.as_tensor(np.asarray(dst, np.int32), device=device)
    cap_t = torch.as_tensor(np.asarray(cap, np.int32), device=device)
    G = m.wbpr_build(n, src_t.numel(), src_t, dst_t, cap_t, s, t, layout_code(layout), opts)
    try:
        flow = torch.empty(max(1, src_t.numel()), dtype=torch.int32, device=device)
        value = m.wbpr_maxflow(G, None, flow[: src_t.numel()] if src_t.numel() else flow)
        out = {"value": value, "flow": flow[: src_t.numel()].cpu().numpy(), "stats": m.wbpr_get_stats(G)}
        if want_cut:
            side = torch.empty(n, dtype=torch.uint8, device=device)
            out["cut"] = m.wbpr_mincut(G, None, side)
            out["side"] = side.cpu().numpy()
        return out
    finally:
        G.close()


def check_against_oracle(n, src, dst, cap, s, t, layout="bcsr", opts=None, ref=None):
    """Value and canonical cut side bit-exact; edge flow certified."""
    src = np.asarray(src, np.int32)
    dst = np.asarray(dst, np.int32)
    cap = np.asarray(cap, np.int32)
    if ref is None:
        ref = oracle.maxflow_pr(n, src, dst, cap, s, t)
    got = gpu_solve(n, src, dst, cap, s, t, layout, opts)
    assert got["value"] == ref["value"], (layout, got["value"], ref["value"])
    assert got["cut"] == ref["value"], (layout, got["cut"], ref["value"])
    assert np.array_equal(got["side"], ref["source_side"]), layout
    code, cut, side = oracle.verify_flow(n, src, dst, cap, s, t, got["flow"], got["value"])
    assert code == 0, (layout, "certificate failed", code)
    assert cut == ref["value"] and np.array_equal(side, ref["source_side"])
    return got


needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")
