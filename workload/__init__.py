"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no FSS, AES, re-share or AND arithmetic: it draws graphs,
attribute values, their three additive shares (the data owner's encryption
step, Alg. 1, done here over Z_{2^n} instead of one-hot bits) and predicates.
Both the CUDA path and the oracle consume what it produces; neither is
imported here.

Recipe (the paper's dataset, 107,614 vertices / 13.7 M edges of a social
attributed graph, is not available; these stand in for it):

* graphs: Chung-Lu power law, weight w_i = (i+1)^(-1/(gamma-1)), gamma = 2.1,
  endpoints drawn independently with probability proportional to w, self-loops
  and repeated undirected edges rejected until M distinct edges exist;
* attributes: uniform on [0, 2^bits) or bounded Zipf(s) ranks k in [1, 2^bits]
  mapped to k - 1;
* shares: <x>_1, <x>_2 uniform in Z_{2^n}, <x>_3 = x - <x>_1 - <x>_2 mod 2^n;
* predicates: equality values and range bounds taken from attribute values of
  seeded "target" elements, so every AND-group has at least one match.
"""
from __future__ import annotations

import numpy as np

PRED_EQ, PRED_RANGE = 1, 2
COMBINE_AND, COMBINE_XOR, COMBINE_OR = 0, 1, 2


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def chung_lu(n_vertices: int, n_edges: int, gamma: float, seed: int) -> np.ndarray:
    """Undirected Chung-Lu graph as an (M, 2) uint32 array, endpoints (lo, hi), edge id = row."""
    g = rng(seed)
    w = (np.arange(n_vertices, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    max_edges = n_vertices * (n_vertices - 1) // 2
    if n_edges > max_edges:
        raise ValueError("more edges than vertex pairs")
    keys = np.empty(0, dtype=np.int64)
    order = np.empty(0, dtype=np.int64)
    drawn = 0
    while len(keys) < n_edges:
        need = n_edges - len(keys)
        batch = int(need * 1.3) + 1024
        a = np.minimum(np.searchsorted(cdf, g.random(batch)), n_vertices - 1).astype(np.int64)
        b = np.minimum(np.searchsorted(cdf, g.random(batch)), n_vertices - 1).astype(np.int64)
        keep = a != b
        lo, hi = np.minimum(a, b)[keep], np.maximum(a, b)[keep]
        new_keys = lo * n_vertices + hi
        new_order = np.arange(drawn, drawn + len(new_keys), dtype=np.int64)
        drawn += len(new_keys)
        allk = np.concatenate([keys, new_keys])
        allo = np.concatenate([order, new_order])
        uk, first = np.unique(allk, return_index=True)
        sel = np.sort(first)                       # keep arrival order of first occurrences
        keys, order = allk[sel], allo[sel]
    keys = keys[:n_edges]
    return np.stack([keys // n_vertices, keys % n_vertices], axis=1).astype(np.uint32)


def uniform_attrs(g: np.random.Generator, n_attrs: int, n_elems: int, bits: int) -> np.ndarray:
    return g.integers(0, 1 << bits, size=(n_attrs, n_elems), dtype=np.uint64).astype(np.uint32)


def zipf_attrs(g: np.random.Generator, n_attrs: int, n_elems: int, s: float, bits: int) -> np.ndarray:
    """Bounded Zipf(s) on ranks [1, 2^bits] by rejection, returned as rank - 1."""
    top = 1 << bits
    out = np.empty(n_attrs * n_elems, dtype=np.uint64)
    filled = 0
    while filled < len(out):
        k = g.zipf(s, size=max(1024, int((len(out) - filled) * 1.6)))
        k = k[(k >= 1) & (k <= top)]
        take = min(len(k), len(out) - filled)
        out[filled:filled + take] = k[:take] - 1
        filled += take
    return out.reshape(n_attrs, n_elems).astype(np.uint32)


def share3(g: np.random.Generator, values: np.ndarray, bits: int):
    """Three additive shares over Z_{2^bits} of a uint32 array (any shape)."""
    mask = np.uint64((1 << bits) - 1)
    v = values.astype(np.uint64)
    s1 = g.integers(0, 1 << bits, size=v.shape, dtype=np.uint64)
    s2 = g.integers(0, 1 << bits, size=v.shape, dtype=np.uint64)
    s3 = (v - s1 - s2) & mask
    return s1.astype(np.uint32), s2.astype(np.uint32), s3.astype(np.uint32)


def eq_pred(table: int, attr: int, group: int, value: int, combine: int = COMBINE_AND):
    return {"kind": PRED_EQ, "table": table, "attr": attr, "group": group, "lo": int(value), "hi": int(value),
            "combine": combine}


def range_pred(table: int, attr: int, group: int, lo: int, hi: int, combine: int = COMBINE_AND):
    return {"kind": PRED_RANGE, "table": table, "attr": attr, "group": group, "lo": int(lo), "hi": int(hi),
            "combine": combine}


def range_around(g: np.random.Generator, value: int, bits: int, width_frac: float):
    """An inclusive range of about width_frac * 2^bits values that contains value."""
    top = (1 << bits) - 1
    width = max(1, int(width_frac * (top + 1)))
    lo = max(0, int(value) - int(g.integers(0, width)))
    hi = min(top, lo + width - 1)
    if hi < value:
        hi = int(value)
    return lo, hi


def onehot_words(bits: int) -> int:
    """32-bit words of one packed one-hot vector of length 2^bits (at least one word)."""
    return max(1, (1 << bits) // 32)


def onehot_shares(g: np.random.Generator, values: np.ndarray, bits: int):
    """Binary RSS of one-hot encodings (the data owner's encryption of Sec. V-B): value v
    becomes e_v in {0,1}^(2^bits), bit l in bit l % 32 of word l // 32, and
    e_v = <e>_1 xor <e>_2 xor <e>_3 with <e>_1, <e>_2 uniform on the 2^bits valid bits.
    values: [n_attrs, n_elems]; returns three uint32 arrays [n_attrs, n_elems, W]."""
    wds = onehot_words(bits)
    valid = np.uint32(0xFFFFFFFF) if bits >= 5 else np.uint32((1 << (1 << bits)) - 1)
    na, ne = values.shape
    e = np.zeros((na, ne, wds), dtype=np.uint32)
    v = values.astype(np.int64)
    ai, ei = np.meshgrid(np.arange(na), np.arange(ne), indexing="ij")
    e[ai, ei, v // 32] = (np.uint32(1) << (v % 32).astype(np.uint32))
    s1 = g.integers(0, 1 << 32, size=e.shape, dtype=np.uint64).astype(np.uint32) & valid
    s2 = g.integers(0, 1 << 32, size=e.shape, dtype=np.uint64).astype(np.uint32) & valid
    return s1, s2, e ^ s1 ^ s2


def onehot_table(values: np.ndarray, bits: int, g: np.random.Generator):
    """A one-hot element table: plaintext rows and the three binary one-hot share sets."""
    return {"values": values, "bits": bits, "shares": onehot_shares(g, values, bits), "onehot": True}


def table(values: np.ndarray, bits: int, g: np.random.Generator):
    """A resident element table: its plaintext rows and their three share sets."""
    return {"values": values, "bits": bits, "shares": share3(g, values, bits)}


# ---------------------------------------------------------------- the five workloads

def tiny_path(seed: int = 1):
    """1,000 vertices / 4,000 Chung-Lu edges; 2 uint16 vertex attributes (uniform), 1 uint16
    edge attribute (Zipf 1.1); query = 3-vertex path v0-v1-v2 with an equality predicate on
    v0.a0 and a range predicate on the edge (v1, v2); n = 16."""
    g = rng(seed)
    edges = chung_lu(1000, 4000, 2.1, seed + 1)
    vt = table(uniform_attrs(g, 2, 1000, 16), 16, g)
    et = table(zipf_attrs(g, 1, 4000, 1.1, 16), 16, g)
    # a target embedding: edge te = (v1, v2) and a neighbour v0 of v1 other than v2
    while True:
        te = int(g.integers(0, 4000))
        v1, v2 = (int(v) for v in edges[te])
        nbrs = [int(b) if int(a) == v1 else int(a) for a, b in edges if v1 in (int(a), int(b))]
        nbrs = [v for v in nbrs if v != v2]
        if nbrs:
            tv = nbrs[int(g.integers(0, len(nbrs)))]
            break
    lo, hi = range_around(g, int(et["values"][0, te]), 16, 0.05)
    preds = [eq_pred(0, 0, 0, vt["values"][0, tv]), range_pred(1, 0, 1, lo, hi)]
    return {"name": "tiny_path_1k_4k_n16", "n_bits": 16, "tables": [vt, et], "edges": edges,
            "n_vertices": 1000, "preds": preds, "n_groups": 2,
            "query_vertices": 3, "query_edges": [(0, 1), (1, 2)],
            "vertex_group": {0: 0}, "edge_group": {1: 1}}


def bulk_vertex_filter(n_vertices: int = 1 << 20, seed: int = 2):
    """n_vertices vertices with 4 uint32 attributes uniform on [0, 2^32); 8 predicates (equality
    on a0..a3, range on a0..a3) ANDed together; n = 32.  The predicates are drawn around a few
    target vertices so the AND has matches."""
    g = rng(seed)
    vt = table(uniform_attrs(g, 4, n_vertices, 32), 32, g)
    target = int(g.integers(0, n_vertices))
    preds = []
    for a in range(4):
        preds.append(eq_pred(0, a, 0, vt["values"][a, target]))
    for a in range(4):
        lo, hi = range_around(g, int(vt["values"][a, target]), 32, float(g.uniform(0.05, 0.6)))
        preds.append(range_pred(0, a, 0, lo, hi))
    return {"name": f"bulk_vertex_filter_{n_vertices}v_4attr_8pred_n32", "n_bits": 32, "tables": [vt],
            "preds": preds, "n_groups": 1, "target": target}


def random_query(g: np.random.Generator, tables, n_bits: int, n_preds: int, n_query_vertices: int,
                 vertex_table: int = 0, edge_table: int = 1, eq_frac: float = 0.5):
    """A query of n_query_vertices vertices with n_preds predicates spread over its vertices and
    edges (a path plus chords), one AND-group per predicated query element."""
    qv = n_query_vertices
    qedges = [(i, i + 1) for i in range(qv - 1)]
    if qv >= 3:
        qedges.append((0, qv - 1))
    slots = [("v", i) for i in range(qv)] + [("e", i) for i in range(len(qedges))]
    g.shuffle(slots)
    preds, group_of = [], {}
    for k in range(n_preds):
        kind, idx = slots[k % len(slots)]
        t = vertex_table if kind == "v" else edge_table
        tab = tables[t]
        attr = int(g.integers(0, tab["values"].shape[0]))
        key = (kind, idx)
        if key not in group_of:
            group_of[key] = len(group_of)
        target = int(g.integers(0, tab["values"].shape[1]))
        v = int(tab["values"][attr, target])
        if g.random() < eq_frac:
            preds.append(eq_pred(t, attr, group_of[key], v))
        else:
            lo, hi = range_around(g, v, n_bits, float(g.uniform(0.01, 0.5)))
            preds.append(range_pred(t, attr, group_of[key], lo, hi))
    preds.sort(key=lambda p: p["group"])
    return {"preds": preds, "n_groups": len(group_of), "query_vertices": qv, "query_edges": qedges}


def edge_graph(n_vertices: int, n_edges: int, n_vattrs: int, n_eattrs: int, seed: int,
               vertex_zipf: float | None = None, edge_zipf: float = 1.2, with_edges: bool = False):
    """A Chung-Lu graph's vertex and edge tables (uint32 attributes, n = 32)."""
    g = rng(seed)
    if vertex_zipf is None:
        vals = uniform_attrs(g, n_vattrs, n_vertices, 32)
    else:
        vals = zipf_attrs(g, n_vattrs, n_vertices, vertex_zipf, 32)
    vt = table(vals, 32, g)
    et = table(zipf_attrs(g, n_eattrs, n_edges, edge_zipf, 32), 32, g)
    out = {"tables": [vt, et], "n_bits": 32, "n_vertices": n_vertices, "n_edges": n_edges}
    if with_edges:
        out["edges"] = chung_lu(n_vertices, n_edges, 2.1, seed + 1)
    return out


def triangle_pendant(graph, seed: int = 3):
    """Triangle v0-v1-v2 plus pendant edge v0-v3: 6 predicates, alternating equality/range,
    on v0, v1, v2 and on the edges (v0,v1), (v1,v2), (v0,v3); one AND-group per element."""
    g = rng(seed)
    vt, et = graph["tables"]
    preds = []
    slots = [(0, 0), (1, 0), (0, 1), (1, 1), (0, 2), (1, 2)]   # (table, element slot)
    for k, (t, slot) in enumerate(slots):
        tab = vt if t == 0 else et
        attr = int(g.integers(0, tab["values"].shape[0]))
        target = int(g.integers(0, tab["values"].shape[1]))
        v = int(tab["values"][attr, target])
        if k % 2 == 0:
            preds.append(eq_pred(t, attr, k, v))
        else:
            lo, hi = range_around(g, v, 32, 0.3)
            preds.append(range_pred(t, attr, k, lo, hi))
    return {"preds": preds, "n_groups": 6, "query_vertices": 4,
            "query_edges": [(0, 1), (1, 2), (2, 0), (0, 3)]}


def query_mix(graph, n_queries: int, seed: int, max_preds: int = 6):
    """n_queries queries with 2-8 vertices and 1-max_preds predicates each (uniform, seeded)."""
    g = rng(seed)
    out = []
    for _ in range(n_queries):
        qv = int(g.integers(2, 9))
        npred = int(g.integers(1, max_preds + 1))
        out.append(random_query(g, graph["tables"], graph["n_bits"], npred, qv))
    return out
