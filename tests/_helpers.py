"""Shared test plumbing: device/host array moves and oracle calls on a workload."""
from __future__ import annotations

import numpy as np

PRF = bytes(range(48))


def to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def from_dev(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def group_tables(wl, n_groups=None):
    """table id of every AND-group of a workload's predicate list"""
    ng = n_groups if n_groups is not None else wl["n_groups"]
    out = [None] * ng
    for p in wl["preds"]:
        out[p["group"]] = p["table"]
    return out


def alloc_outs(wl, preds=None, n_groups=None, offset=0):
    """three uint32 CUDA outputs per AND-group; offset > 0 shifts the start to break 16-byte alignment"""
    import torch
    preds = preds if preds is not None else wl["preds"]
    ng = n_groups if n_groups is not None else max(p["group"] for p in preds) + 1
    tabs = [None] * ng
    for p in preds:
        tabs[p["group"]] = p["table"]
    outs = []
    for g in range(ng):
        n = wl["tables"][tabs[g]]["values"].shape[1]
        grp = []
        for _ in range(3):
            base = torch.full((n + offset,), -1, dtype=torch.int32, device="cuda")
            grp.append(base[offset:])
        outs.append(grp)
    return outs


def load_tables(ctx, wl):
    for tid, t in enumerate(wl["tables"]):
        ctx.load_shares(tid, [to_dev(s) for s in t["shares"]], t["bits"])


def oracle_group(oracle, wl, tokens, query_id, group, elems, threads=8):
    tabs = [(t["shares"], t["bits"]) for t in wl["tables"]]
    return oracle.filter_group(tokens, query_id, PRF, tabs, group, elems, threads=threads)
