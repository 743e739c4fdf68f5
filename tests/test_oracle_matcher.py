"""Pins for the plaintext subgraph matcher (Def. 2) and the oblivious filter feeding it.

The worked example of Sec. III (Fig. 1 and the two results g1, g2 printed
after it): a university located in Harbin, two persons aged 30..40 who
graduated from it, one working at a software company and one at an Internet
company.  The figure's graph is not in the text, so the toy graph below is
built to agree with everything the text states; the expected matches are the
paper's g1 = U1 -> {P1 -> C1, P3 -> C2} and g2 = U1 -> {P2 -> C1, P3 -> C2}.
"""
import numpy as np

import oracle
import workload as W

PRF = bytes(range(48))

# vertex ids
U1, U2, P1, P2, P3, P4, C1, C2, C3 = range(9)
TYPE_U, TYPE_P, TYPE_C = 1, 2, 3
HARBIN, BEIJING = 10, 11
SOFTWARE, INTERNET, FINANCE = 20, 21, 22


def _fig1_graph():
    types = [TYPE_U, TYPE_U, TYPE_P, TYPE_P, TYPE_P, TYPE_P, TYPE_C, TYPE_C, TYPE_C]
    value = [HARBIN, BEIJING, 35, 32, 38, 50, SOFTWARE, INTERNET, FINANCE]
    edges = [(U1, P1), (U1, P2), (U1, P3), (U1, P4), (U2, P2), (P1, C1), (P2, C1), (P3, C2),
             (P4, C2), (P2, C3), (P1, P3)]
    attrs = np.array([types, value], dtype=np.uint32)
    return attrs, np.array(edges, dtype=np.uint32)


# query vertices: 0 = U (Harbin), 1 = P (age in [30,40]) -> 3 = C (software),
#                 2 = P (age in [30,40]) -> 4 = C (Internet)
Q_EDGES = [(0, 1), (0, 2), (1, 3), (2, 4)]
Q_PREDS = [
    W.eq_pred(0, 0, 0, TYPE_U), W.eq_pred(0, 1, 0, HARBIN),
    W.eq_pred(0, 0, 1, TYPE_P), W.range_pred(0, 1, 1, 30, 40),
    W.eq_pred(0, 0, 2, TYPE_P), W.range_pred(0, 1, 2, 30, 40),
    W.eq_pred(0, 0, 3, TYPE_C), W.eq_pred(0, 1, 3, SOFTWARE),
    W.eq_pred(0, 0, 4, TYPE_C), W.eq_pred(0, 1, 4, INTERNET),
]
PAPER_RESULTS = [(U1, P1, P3, C1, C2), (U1, P2, P3, C1, C2)]


def test_fig1_plaintext_matcher():
    attrs, edges = _fig1_graph()
    ok = [oracle.plain_group(Q_PREDS, q, attrs).astype(bool) for q in range(5)]
    got = oracle.match(9, edges, 5, Q_EDGES, ok, [None] * 4)
    assert got == PAPER_RESULTS


def test_fig1_oblivious_filter_then_match():
    attrs, edges = _fig1_graph()
    bits = 8
    g = W.rng(11)
    t = W.table(attrs, bits, g)
    toks = oracle.keygen(Q_PREDS, bits, bytes(range(16)))
    ok = []
    for q in range(5):
        out = oracle.filter_group(toks, 4, PRF, [(t["shares"], bits)], q, np.arange(9))
        ok.append(oracle.reconstruct(out).astype(bool))
    assert oracle.match(9, edges, 5, Q_EDGES, ok, [None] * 4) == PAPER_RESULTS


def test_matcher_injective_and_edges():
    # triangle query on K4 has 4*3*2 = 24 ordered embeddings
    edges = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], dtype=np.uint32)
    got = oracle.match(4, edges, 3, [(0, 1), (1, 2), (2, 0)], [None] * 3, [None] * 3)
    assert len(got) == 24 and all(len(set(e)) == 3 for e in got)
    # on a 4-cycle there is no triangle
    cyc = np.array([(0, 1), (1, 2), (2, 3), (3, 0)], dtype=np.uint32)
    assert oracle.match(4, cyc, 3, [(0, 1), (1, 2), (2, 0)], [None] * 3, [None] * 3) == []


def test_tiny_path_workload_oblivious_equals_plaintext():
    wl = W.tiny_path(seed=1)
    tabs = [(t["shares"], t["bits"]) for t in wl["tables"]]
    toks = oracle.keygen(wl["preds"], wl["n_bits"], bytes(range(16)))
    vt, et = wl["tables"]
    bits_v = oracle.reconstruct(oracle.filter_group(toks, 1, PRF, tabs, 0, np.arange(1000), threads=8))
    bits_e = oracle.reconstruct(oracle.filter_group(toks, 1, PRF, tabs, 1, np.arange(4000), threads=8))
    assert np.array_equal(bits_v, oracle.plain_group(wl["preds"], 0, vt["values"]))
    assert np.array_equal(bits_e, oracle.plain_group(wl["preds"], 1, et["values"]))
    vok = [bits_v.astype(bool), None, None]
    eok = [None, bits_e.astype(bool)]
    got = oracle.match(1000, wl["edges"], 3, wl["query_edges"], vok, eok)
    want = oracle.match(1000, wl["edges"], 3, wl["query_edges"],
                        [oracle.plain_group(wl["preds"], 0, vt["values"]).astype(bool), None, None],
                        [None, oracle.plain_group(wl["preds"], 1, et["values"]).astype(bool)])
    assert got == want and len(got) > 0


def test_distinct_matches_closed_forms():
    """Ordered embeddings against distinct subgraphs: |Aut(query)| embeddings per subgraph."""
    k4 = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], dtype=np.uint32)
    k5 = np.array([(a, b) for a in range(5) for b in range(a + 1, 5)], dtype=np.uint32)
    tri = [(0, 1), (1, 2), (2, 0)]
    sq = [(0, 1), (1, 2), (2, 3), (3, 0)]
    path = [(0, 1), (1, 2)]
    none3, none4 = [None] * 3, [None] * 4
    # triangles: C(4, 3) = 4 in K4, C(5, 3) = 10 in K5, each 6 times (|Aut(C3)| = 6)
    e = oracle.match(4, k4, 3, tri, none3, none3)
    assert (len(e), oracle.distinct_matches(e, tri)) == (24, 4)
    e = oracle.match(5, k5, 3, tri, none3, none3)
    assert (len(e), oracle.distinct_matches(e, tri)) == (60, 10)
    # 4-cycles in K4: 3, each 8 times (|Aut(C4)| = 8)
    e = oracle.match(4, k4, 4, sq, none4, none4)
    assert (len(e), oracle.distinct_matches(e, sq)) == (24, 3)
    # 2-edge paths in K4: 4 centres x C(3, 2) leaf pairs = 12, each twice
    e = oracle.match(4, k4, 3, path, none3, [None] * 2)
    assert (len(e), oracle.distinct_matches(e, path)) == (24, 12)
    # a predicate on one end breaks the path's symmetry: no two embeddings share an image
    ok0 = np.array([True, False, False, False])
    e = oracle.match(4, k4, 3, path, [ok0, None, None], [None] * 2)
    assert len(e) == oracle.distinct_matches(e, path) == 6


def test_fig1_results_are_distinct_subgraphs():
    attrs, edges = _fig1_graph()
    ok = [oracle.plain_group(Q_PREDS, q, attrs).astype(bool) for q in range(5)]
    got = oracle.match(9, edges, 5, Q_EDGES, ok, [None] * 4)
    assert oracle.distinct_matches(got, Q_EDGES) == len(PAPER_RESULTS)
