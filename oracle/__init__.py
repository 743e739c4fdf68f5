"""Plain CPU oracle for OblivGM's masked secure predicate evaluation.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  The
product package never imports it and it never imports the product package.

The arithmetic lives in ``oracle.c`` (plain byte-oriented FIPS-197 AES, the
DPF/DCF constructions the paper cites, the token of Sec. V-C, secEval of
Alg. 3 with the re-share of Sec. III-B and the AND fold of Sec. V-D).  This
module compiles it with gcc, loads it with ctypes and adds the plaintext
definitions the results reconstruct to:

* ``plain_pred``  -- Def. 2: ``Att == value`` (equality) or ``Att in range``;
* ``match``       -- Def. 2 subgraph matching by brute-force backtracking.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboblivgm_oracle.so")

KIND_DPF, KIND_DCF = 1, 2
PRED_EQ, PRED_RANGE = 1, 2
COMBINE_AND, COMBINE_XOR, COMBINE_OR = 0, 1, 2
BETA_PRIME = 0xAAAAAAAB        # 3^{-1} mod 2^32
MASK32 = 0xFFFFFFFF

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain gcc, portable C99)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _Table(ctypes.Structure):
    _fields_ = [("n_elems", ctypes.c_uint64), ("n_attrs", ctypes.c_uint32), ("n_bits", ctypes.c_uint32),
                ("share", ctypes.c_void_p * 3)]


class _Pred(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in ("kind", "table", "attr", "group", "lo", "hi", "combine")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            u8p, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
            l.orc_init.restype = None
            l.orc_aes128.argtypes = [u8p, u8p, u8p]
            l.orc_prg.argtypes = [ctypes.c_int, u8p, u8p]
            l.orc_key_len.argtypes = [ctypes.c_int, ctypes.c_int]
            l.orc_key_len.restype = ctypes.c_size_t
            for g in (l.orc_dpf_gen, l.orc_dcf_gen):
                g.argtypes = [ctypes.c_int, u32, u32, u8p, u8p, u8p, u8p]
                g.restype = None
            for e in (l.orc_dpf_eval, l.orc_dcf_eval):
                e.argtypes = [u8p, u32]
                e.restype = u32
            l.orc_token_len.argtypes = [ctypes.POINTER(_Pred), u32, ctypes.c_int]
            l.orc_token_len.restype = ctypes.c_size_t
            l.orc_keygen.argtypes = [ctypes.POINTER(_Pred), u32, ctypes.c_int, u8p, u8p, u8p, u8p, ctypes.c_size_t]
            l.orc_filter.argtypes = [u8p, u8p, u8p, ctypes.POINTER(ctypes.c_size_t), u32, u8p,
                                     ctypes.POINTER(_Table), u32, u32, u8p, u64, u8p]
            l.orc_pred_z.argtypes = [u8p, u8p, u8p, ctypes.POINTER(ctypes.c_size_t), u32, u32, u8p, u8p]
            for g in (l.orc_dpf_gen_g, l.orc_dcf_gen_g):
                g.argtypes = [ctypes.c_int, u32, u32, u8p, u8p, u8p, u8p, ctypes.c_int]
                g.restype = None
            l.orc_keygen_onehot.argtypes = l.orc_keygen.argtypes
            l.orc_token_len_onehot.argtypes = l.orc_token_len.argtypes
            l.orc_token_len_onehot.restype = ctypes.c_size_t
            l.orc_key_len_et.argtypes = [ctypes.c_int, ctypes.c_int]
            l.orc_key_len_et.restype = ctypes.c_size_t
            for g in (l.orc_dpf_gen_et, l.orc_dcf_gen_et):
                g.argtypes = [ctypes.c_int, u32, u8p, u8p, u8p, u8p]
                g.restype = None
            l.orc_prf_bit.argtypes = [u8p, u64, u32, u32, u32]
            l.orc_prf_bit.restype = u32
            l.orc_eval_et.argtypes = [u8p, u32]
            l.orc_eval_et.restype = u32
            l.orc_filter_onehot.argtypes = [u8p, u8p, u8p, ctypes.POINTER(ctypes.c_size_t), u32, u8p,
                                            ctypes.POINTER(_Table), u32, u32, u8p, u64, u8p]
            l.orc_reshare.argtypes = [u8p, u8p, u8p, u64, u32, u32, u32]
            l.orc_fresh_token_len.argtypes = [ctypes.POINTER(_Pred), u32, ctypes.c_int, u8p, u32]
            l.orc_fresh_token_len.restype = u64
            l.orc_keygen_fresh.argtypes = [ctypes.POINTER(_Pred), u32, ctypes.c_int, u8p, u32, u8p, u8p, u8p, u8p,
                                           u64]
            l.orc_filter_fresh.argtypes = [u8p, u8p, u8p, u32, u8p, ctypes.POINTER(_Table), u32, u32, u8p, u64, u8p]
            l.orc_prp.argtypes = [u8p, u64, u64]
            l.orc_prp.restype = u64
            l.orc_shuffle.argtypes = [ctypes.c_int, u64, u32, u8p, u8p, u8p, u8p, u8p, u8p, u8p, u8p, u8p]
            l.orc_fetch_multi.argtypes = [u64, u8p, u8p, u8p, ctypes.POINTER(_Table), u32, u8p, u8p, u8p, u8p, u8p,
                                          u64, u8p, u8p]
            l.orc_fetch_multi.restype = ctypes.c_int64
            l.orc_fresh_direct.argtypes = [ctypes.POINTER(_Pred), u32, ctypes.c_int, u8p, u32, u8p, u32, u8p,
                                           ctypes.POINTER(_Table), u32, u8p, u64, u8p]
            l.orc_aes_blocks.restype = u64
            l.orc_test_plant.argtypes = [ctypes.c_int]
            l.orc_test_plant.restype = None
            l.orc_sbox.argtypes = [u32]
            l.orc_sbox.restype = u32
            l.orc_init()
            _lib = l
    return _lib


def _buf(b: bytes):
    return ctypes.create_string_buffer(bytes(b), len(b))


def _addr(buf):
    return ctypes.cast(buf, ctypes.c_void_p)


# ---------------------------------------------------------------- primitives

def aes128(key: bytes, block: bytes) -> bytes:
    """AES-128 encryption of one block (FIPS-197)."""
    out = ctypes.create_string_buffer(16)
    lib().orc_aes128(_addr(_buf(key)), _addr(_buf(block)), _addr(out))
    return out.raw


def aes_blocks_reset() -> None:
    """Zero the calling thread's count of AES-128 blocks the oracle has encrypted."""
    lib().orc_aes_blocks_reset()


def aes_blocks() -> int:
    """AES-128 blocks the oracle has encrypted on the calling thread since the last reset
    (test instrumentation: the benchmark's algorithmic block counts are checked against it)."""
    return int(lib().orc_aes_blocks())


def sbox(x: int) -> int:
    """The oracle's AES S-box entry for byte x (built from the GF(2^8) inverse and the affine map)."""
    return int(lib().orc_sbox(x))


PLANT_NONE, PLANT_CONST, PLANT_CLEARED_BIT, PLANT_MASK_OVERLAP = 0, 1, 2, 3


def test_plant(mode: int) -> None:
    """Plant a deliberate mistake in the calling thread's oracle (test instrumentation, so a test
    can show that its pin fails on it): 1 constant Converts and mask words, 2 Converts reading the
    cleared control bit, 3 <r>_1 read from r's bytes; 0 removes it."""
    lib().orc_test_plant(mode)


def prg(which: int, seed: bytes) -> bytes:
    """H_K(s) = AES_K(s) xor s with fixed key K_which (0 L, 1 R, 2 vL, 3 vR)."""
    out = ctypes.create_string_buffer(16)
    lib().orc_prg(which, _addr(_buf(seed)), _addr(out))
    return out.raw


def key_len(kind: int, n: int) -> int:
    return lib().orc_key_len(kind, n)


def _gen(fn, kind, n, alpha, beta, s0, s1):
    L = key_len(kind, n)
    k0, k1 = ctypes.create_string_buffer(L), ctypes.create_string_buffer(L)
    fn(n, alpha & MASK32, beta & MASK32, _addr(_buf(s0)), _addr(_buf(s1)), _addr(k0), _addr(k1))
    return k0.raw, k1.raw


def dpf_gen(n: int, alpha: int, beta: int, s0: bytes, s1: bytes):
    """DPF Gen for f^=_{alpha,beta} over Z_{2^32} (domain {0,1}^n)."""
    return _gen(lib().orc_dpf_gen, KIND_DPF, n, alpha, beta, s0, s1)


def dcf_gen(n: int, alpha: int, beta: int, s0: bytes, s1: bytes):
    """DCF Gen for g^<_{alpha,beta} over Z_{2^32} (domain {0,1}^n)."""
    return _gen(lib().orc_dcf_gen, KIND_DCF, n, alpha, beta, s0, s1)


def dpf_gen_z2(n: int, alpha: int, s0: bytes, s1: bytes):
    """DPF Gen for f^=_{alpha,1} over Z_2 (the one-hot mode's output group)."""
    L = key_len(KIND_DPF, n)
    k0, k1 = ctypes.create_string_buffer(L), ctypes.create_string_buffer(L)
    lib().orc_dpf_gen_g(n, alpha & MASK32, 1, _addr(_buf(s0)), _addr(_buf(s1)), _addr(k0), _addr(k1), 1)
    return k0.raw, k1.raw


def dcf_gen_z2(n: int, alpha: int, s0: bytes, s1: bytes):
    """DCF Gen for g^<_{alpha,1} over Z_2."""
    L = key_len(KIND_DCF, n)
    k0, k1 = ctypes.create_string_buffer(L), ctypes.create_string_buffer(L)
    lib().orc_dcf_gen_g(n, alpha & MASK32, 1, _addr(_buf(s0)), _addr(_buf(s1)), _addr(k0), _addr(k1), 1)
    return k0.raw, k1.raw


def key_len_et(kind: int, n: int) -> int:
    """Length of an early-terminated Z_2 key (the one-hot mode's keys)."""
    return lib().orc_key_len_et(kind, n)


def _gen_et(fn, kind, n, alpha, s0, s1):
    L = key_len_et(kind, n)
    k0, k1 = ctypes.create_string_buffer(L), ctypes.create_string_buffer(L)
    fn(n, alpha & MASK32, _addr(_buf(s0)), _addr(_buf(s1)), _addr(k0), _addr(k1))
    return k0.raw, k1.raw


def dpf_gen_et(n: int, alpha: int, s0: bytes, s1: bytes):
    """DPF Gen for [x == alpha] over Z_2 with early termination (2^min(n,7) outputs per leaf seed)."""
    return _gen_et(lib().orc_dpf_gen_et, KIND_DPF, n, alpha, s0, s1)


def dcf_gen_et(n: int, alpha: int, s0: bytes, s1: bytes):
    """DCF Gen for [x < alpha] over Z_2 with early termination."""
    return _gen_et(lib().orc_dcf_gen_et, KIND_DCF, n, alpha, s0, s1)


def eval_et(key: bytes, x: int) -> int:
    """Eval of an early-terminated Z_2 key (DPF or DCF, from its header) at x: 0 or 1."""
    return lib().orc_eval_et(_addr(_buf(key)), x & MASK32)


def prf_bit(key: bytes, elem: int, step: int, table: int, query: int) -> int:
    """The one-hot mode's re-share PRF into Z_2 (bit elem mod 128 of one AES block)."""
    return lib().orc_prf_bit(_addr(_buf(key)), elem, step, table, query)


def dpf_eval(key: bytes, x: int) -> int:
    return lib().orc_dpf_eval(_addr(_buf(key)), x & MASK32)


def dcf_eval(key: bytes, x: int) -> int:
    return lib().orc_dcf_eval(_addr(_buf(key)), x & MASK32)


def eval_many(key: bytes, xs, kind: int) -> np.ndarray:
    """Eval one key at many points (plain loop over the C Eval)."""
    k = _buf(key)
    fn = lib().orc_dpf_eval if kind == KIND_DPF else lib().orc_dcf_eval
    return np.array([fn(_addr(k), int(x) & MASK32) for x in xs], dtype=np.uint32)


# ---------------------------------------------------------------- token + secEval

def _preds(preds):
    arr = (_Pred * len(preds))()
    for i, p in enumerate(preds):
        arr[i].kind, arr[i].table, arr[i].attr = p["kind"], p["table"], p["attr"]
        arr[i].group, arr[i].lo, arr[i].hi = p.get("group", 0), p["lo"], p.get("hi", p["lo"])
        arr[i].combine = p.get("combine", COMBINE_AND)
    return arr


def token_len(preds, n: int) -> int:
    return lib().orc_token_len(_preds(preds), len(preds), n)


def keygen(preds, n: int, seed: bytes):
    """The three server tokens tok^(1..3) for a list of predicates (Sec. V-C).

    Each predicate is a dict with kind (PRED_EQ / PRED_RANGE), table, attr,
    group (AND-group index) and lo (= alpha for EQ), hi (inclusive, RANGE).
    """
    arr = _preds(preds)
    L = token_len(preds, n)
    bufs = [ctypes.create_string_buffer(L) for _ in range(3)]
    rc = lib().orc_keygen(arr, len(preds), n, _addr(_buf(seed)), *[_addr(b) for b in bufs], L)
    if rc != 0:
        raise ValueError(f"oracle keygen rejected the predicates (code {rc})")
    return tuple(b.raw for b in bufs)


def keygen_onehot(preds, n: int, seed: bytes):
    """Tokens of the one-hot mode (Sec. V-C as written): no mask, early-terminated Z_2 keys
    with beta = 1."""
    arr = _preds(preds)
    L = lib().orc_token_len_onehot(arr, len(preds), n)
    bufs = [ctypes.create_string_buffer(L) for _ in range(3)]
    rc = lib().orc_keygen_onehot(arr, len(preds), n, _addr(_buf(seed)), *[_addr(b) for b in bufs], L)
    if rc != 0:
        raise ValueError(f"oracle one-hot keygen rejected the predicates (code {rc})")
    return tuple(b.raw for b in bufs)


def filter_onehot(tokens, query_id: int, prf_keys: bytes, tables, group: int, elems) -> np.ndarray:
    """One-hot secEval (Eq. predEval) + binary re-share + binary AND of one AND-group.

    tables: list of (three uint32 arrays [n_attrs, n_elems, W], n_bits) of one-hot shares.
    Returns the three binary RSS share sets as 0/1 values, shape (3, len(elems)).
    """
    elems = np.ascontiguousarray(elems, dtype=np.uint64)
    arr = (_Table * len(tables))()
    keep = []
    for i, (shares, n_bits) in enumerate(tables):
        shares = [np.ascontiguousarray(x, dtype=np.uint32) for x in shares]
        keep.extend(shares)
        arr[i].n_attrs, arr[i].n_elems = shares[0].shape[0], shares[0].shape[1]
        arr[i].n_bits = n_bits
        for j in range(3):
            arr[i].share[j] = shares[j].ctypes.data
    toks = [_buf(t) for t in tokens]
    lens = (ctypes.c_size_t * 3)(*[len(t) for t in tokens])
    out = np.zeros((3, len(elems)), dtype=np.uint32)
    if len(elems):
        rc = lib().orc_filter_onehot(*[_addr(t) for t in toks], lens, query_id, _addr(_buf(prf_keys)), arr,
                                     len(tables), group, elems.ctypes.data, len(elems), out.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle one-hot filter failed (code {rc})")
    del keep
    return out


def reconstruct_bits(shares) -> np.ndarray:
    """XOR of the three binary share sets."""
    s = np.asarray(shares, dtype=np.uint32)
    return (s[0] ^ s[1] ^ s[2]) & 1


def _tables(tables):
    """tables: list of 3-tuples of uint32 arrays shaped [n_attrs, n_elems] plus n_bits."""
    arr = (_Table * len(tables))()
    keep = []
    for i, (shares, n_bits) in enumerate(tables):
        shares = [np.ascontiguousarray(s, dtype=np.uint32) for s in shares]
        keep.extend(shares)
        arr[i].n_attrs, arr[i].n_elems = shares[0].shape
        arr[i].n_bits = n_bits
        for j in range(3):
            arr[i].share[j] = shares[j].ctypes.data
    return arr, keep


def filter_group(tokens, query_id: int, prf_keys: bytes, tables, group: int, elems,
                 threads: int = 1) -> np.ndarray:
    """secEval + re-share + AND fold of one AND-group on the listed elements.

    Returns the three RSS share sets, shape (3, len(elems)), uint32.
    ``threads`` > 1 splits the element list across threads (the C code holds
    no shared mutable state after initialisation).
    """
    elems = np.ascontiguousarray(elems, dtype=np.uint64)
    tarr, keep = _tables(tables)
    toks = [_buf(t) for t in tokens]
    lens = (ctypes.c_size_t * 3)(*[len(t) for t in tokens])
    pk = _buf(prf_keys)
    out = np.zeros((3, len(elems)), dtype=np.uint32)

    def run(lo, hi):
        part = np.ascontiguousarray(elems[lo:hi])
        o = np.zeros((3, hi - lo), dtype=np.uint32)
        rc = lib().orc_filter(*[_addr(t) for t in toks], lens, query_id, _addr(pk), tarr, len(tables),
                              group, part.ctypes.data, hi - lo, o.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle filter failed (code {rc})")
        out[:, lo:hi] = o

    n = len(elems)
    if threads <= 1 or n < 2 * threads:
        if n:
            run(0, n)
    else:
        cuts = np.linspace(0, n, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda i: run(cuts[i], cuts[i + 1]), range(threads)))
    del keep
    return out


def pred_z(tokens, pred: int, xhat: int):
    """z_1..z_3 and the six key-half outputs y of one predicate at masked input xhat."""
    toks = [_buf(t) for t in tokens]
    lens = (ctypes.c_size_t * 3)(*[len(t) for t in tokens])
    z = (ctypes.c_uint32 * 3)()
    y = (ctypes.c_uint32 * 6)()
    rc = lib().orc_pred_z(*[_addr(t) for t in toks], lens, pred, xhat & MASK32,
                          ctypes.cast(z, ctypes.c_void_p), ctypes.cast(y, ctypes.c_void_p))
    if rc != 0:
        raise ValueError("bad token")
    return list(z), list(y)


def reshare(prf_keys: bytes, z, elem: int, step: int, table: int, query: int):
    zi = (ctypes.c_uint32 * 3)(*[int(v) & MASK32 for v in z])
    out = (ctypes.c_uint32 * 3)()
    lib().orc_reshare(_addr(_buf(prf_keys)), ctypes.cast(zi, ctypes.c_void_p), ctypes.cast(out, ctypes.c_void_p),
                      elem, step, table, query)
    return list(out)


def reconstruct(shares) -> np.ndarray:
    """Sum of the three share sets mod 2^32."""
    s = np.asarray(shares, dtype=np.uint64)
    return ((s[0] + s[1] + s[2]) & MASK32).astype(np.uint32)


# ---------------------------------------------------------------- plaintext definitions

def plain_pred(pred, values) -> np.ndarray:
    """Def. 2 on plaintext values: equality or inclusive range membership, as 0/1."""
    v = np.asarray(values, dtype=np.uint64)
    if pred["kind"] == PRED_EQ:
        return (v == pred["lo"]).astype(np.uint32)
    return ((v >= pred["lo"]) & (v <= pred["hi"])).astype(np.uint32)


def plain_group(preds, group: int, attrs) -> np.ndarray:
    """The group's predicates on plaintext attribute rows attrs[attr][elem], folded left to
    right as Boolean values (Sec. V-D): all hold (AND), the paper's "one of" written with
    XOR, or at least one (OR), per predicate's "combine"."""
    res = None
    for p in preds:
        if p.get("group", 0) != group:
            continue
        b = plain_pred(p, attrs[p["attr"]]).astype(bool)
        op = p.get("combine", COMBINE_AND)
        if res is None:
            res = b
        elif op == COMBINE_AND:
            res = res & b
        elif op == COMBINE_XOR:
            res = res != b
        else:
            res = res | b
    return None if res is None else res.astype(np.uint32)


def match(n_vertices: int, edges, query_vertices: int, query_edges, vertex_ok, edge_ok):
    """Def. 2 attributed subgraph matching, brute-force backtracking (tiny graphs only).

    edges: array (M, 2) of undirected graph edges, edge id = row index.
    query_edges: list of (qa, qb) pairs over query vertices 0..query_vertices-1.
    vertex_ok[qv]: bool array over graph vertices (None = no predicate).
    edge_ok[qe]:   bool array over graph edge ids (None = no predicate).
    Returns the sorted list of embeddings (tuples mapping query vertex -> graph vertex),
    injective, each query edge mapped onto a graph edge whose predicate holds.
    """
    adj = [dict() for _ in range(n_vertices)]
    for eid, (a, b) in enumerate(np.asarray(edges)):
        a, b = int(a), int(b)
        adj[a][b] = eid
        adj[b][a] = eid
    qadj = [[] for _ in range(query_vertices)]
    for qe, (qa, qb) in enumerate(query_edges):
        qadj[qa].append((qb, qe))
        qadj[qb].append((qa, qe))
    out = []
    assign = [-1] * query_vertices

    def ok_vertex(qv, v):
        return vertex_ok[qv] is None or bool(vertex_ok[qv][v])

    def extend(qv):
        if qv == query_vertices:
            out.append(tuple(assign))
            return
        # candidates: neighbours of an already-mapped query neighbour, else all vertices
        anchor = next(((qn, qe) for qn, qe in qadj[qv] if assign[qn] >= 0), None)
        cands = adj[assign[anchor[0]]].keys() if anchor else range(n_vertices)
        used = set(a for a in assign if a >= 0)
        for v in cands:
            if v in used or not ok_vertex(qv, v):
                continue
            good = True
            for qn, qe in qadj[qv]:
                if assign[qn] < 0:
                    continue
                eid = adj[v].get(assign[qn])
                if eid is None or (edge_ok[qe] is not None and not edge_ok[qe][eid]):
                    good = False
                    break
            if good:
                assign[qv] = v
                extend(qv + 1)
                assign[qv] = -1

    extend(0)
    return sorted(out)


def distinct_matches(embeddings, query_edges) -> int:
    """Number of distinct matched subgraphs among ordered embeddings (Def. 2).

    Two embeddings that differ by an automorphism of the query graph map it onto the same
    subgraph, and two embeddings with the same vertex set and the same image of the query's
    edges differ by such an automorphism; so the orbits are counted by their images."""
    seen = set()
    for emb in embeddings:
        image = frozenset(frozenset((emb[a], emb[b])) for a, b in query_edges)
        seen.add((frozenset(emb), image))
    return len(seen)


# ---------------------------------------------------------------- secFetch, case I

FETCH_STEP = 256


def fetch_unique(x_shares, tables, table: int, attrs, query_id: int, group: int, prf_keys: bytes):
    """secFetch case I (Alg. 4, Sec. V-D) over Z_{2^32}: with x_c the RSS result of a filter
    (one matching candidate), the matched element's index and attribute values.

    index:  sum_c c * [[x_c]]                      -- linear in the shares, RSS as it stands;
    attr a: sum_c [[v_c]] (x) [[x_c]], per server w_i = sum_c v_i x_i + v_i x_{i+1} + v_{i+1} x_i,
            then one re-share with counter (element = a, step = 256 + group, table, query).
    Returns a (3, 1 + len(attrs)) uint32 array: share set i of [index, attr values...].
    """
    x = [np.asarray(s, dtype=np.uint64) for s in x_shares]
    n = len(x[0])
    shares, _bits = tables[table]
    c = np.arange(n, dtype=np.uint64)
    out = np.zeros((3, 1 + len(attrs)), dtype=np.uint64)
    for i in range(3):
        out[i, 0] = int(np.sum((c * x[i]) & MASK32)) & MASK32
    for col, a in enumerate(attrs):
        v = [np.asarray(shares[j][a], dtype=np.uint64) for j in range(3)]
        w = []
        for i in range(3):
            i1 = (i + 1) % 3
            prod = (v[i] * x[i] + v[i] * x[i1] + v[i1] * x[i]) & MASK32
            w.append(int(np.sum(prod)) & MASK32)
        r = reshare(prf_keys, w, a, FETCH_STEP + group, table, query_id)
        for i in range(3):
            out[i, 1 + col] = r[i]
    return out.astype(np.uint32)


# ---------------------------------------------------------------- fresh keys per element

def _elems_arr(table_elems):
    return np.ascontiguousarray(table_elems, dtype=np.uint64)


def fresh_token_len(preds, n: int, table_elems) -> int:
    te = _elems_arr(table_elems)
    L = lib().orc_fresh_token_len(_preds(preds), len(preds), n, te.ctypes.data, len(te))
    if L == 0:
        raise ValueError("oracle rejected the fresh-key predicates")
    return int(L)


def keygen_fresh(preds, n: int, table_elems, seed: bytes):
    """Fresh-key tokens (one mask and one key triple per element and predicate), three bytes objects."""
    te = _elems_arr(table_elems)
    L = fresh_token_len(preds, n, te)
    bufs = [np.zeros(L, dtype=np.uint8) for _ in range(3)]
    rc = lib().orc_keygen_fresh(_preds(preds), len(preds), n, te.ctypes.data, len(te), _addr(_buf(seed)),
                                *[b.ctypes.data for b in bufs], L)
    if rc != 0:
        raise ValueError(f"oracle fresh keygen failed (code {rc})")
    return tuple(b.tobytes() for b in bufs)


def _run_split(fn, n_out_cols, elems, threads):
    out = np.zeros((3, len(elems)), dtype=np.uint32)

    def run(lo, hi):
        part = np.ascontiguousarray(elems[lo:hi])
        o = np.zeros((3, hi - lo), dtype=np.uint32)
        rc = fn(part, o)
        if rc != 0:
            raise ValueError(f"oracle fresh filter failed (code {rc})")
        out[:, lo:hi] = o

    n = len(elems)
    if threads <= 1 or n < 2 * threads:
        if n:
            run(0, n)
    else:
        cuts = np.linspace(0, n, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda i: run(cuts[i], cuts[i + 1]), range(threads)))
    return out


def filter_fresh(tokens, query_id: int, prf_keys: bytes, tables, group: int, elems, threads: int = 1):
    """Servers' secEval on fresh-key tokens: (3, len(elems)) RSS shares of the group's AND."""
    elems = np.ascontiguousarray(elems, dtype=np.uint64)
    tarr, keep = _tables(tables)
    toks = [np.frombuffer(t, dtype=np.uint8) for t in tokens]
    pk = _buf(prf_keys)

    def fn(part, o):
        return lib().orc_filter_fresh(*[t.ctypes.data for t in toks], query_id, _addr(pk), tarr, len(tables),
                                      group, part.ctypes.data, len(part), o.ctypes.data)

    out = _run_split(fn, 3, elems, threads)
    del keep
    return out


def fresh_direct(preds, n: int, seed: bytes, query_id: int, prf_keys: bytes, tables, group: int, elems,
                 threads: int = 1):
    """The fresh-key result of one group computed from the client seed, keys made where used."""
    elems = np.ascontiguousarray(elems, dtype=np.uint64)
    tarr, keep = _tables(tables)
    te = _elems_arr([t[0][0].shape[1] for t in tables])
    pa, sd, pk = _preds(preds), _buf(seed), _buf(prf_keys)

    def fn(part, o):
        return lib().orc_fresh_direct(pa, len(preds), n, te.ctypes.data, len(te), _addr(sd), query_id, _addr(pk),
                                      tarr, group, part.ctypes.data, len(part), o.ctypes.data)

    out = _run_split(fn, 3, elems, threads)
    del keep
    return out


def fresh_layout(kind: int, n: int, N: int):
    """Byte offsets inside one predicate's data block of a fresh token (the documented layout):
    dict with rA, rB, cb (RANGE), and per key block (half, sub) its seed/scw/tl/tr/vcw/cw offsets."""
    N4 = (N + 3) // 4 * 4
    eq = kind == PRED_EQ
    kdcf = not eq
    kb = 16 * N + 16 * n * N + 8 * N4 + 4 * N4 + (4 * n * N4 if kdcf else 0)
    lay = {"rA": 0, "rB": 4 * N4, "keys_at": (8 if eq else 12) * N4, "key_block": kb, "N4": N4}
    if not eq:
        lay["cb"] = 8 * N4
    return lay


# ---------------------------------------------------------------- secShuffle / secFetch case II

SHUF_ADD, SHUF_XOR = 0, 1


def prp(seed: bytes, n: int, x: int) -> int:
    """The pair's pseudo-random permutation of [0, n) at x (Feistel with cycle walking)."""
    return int(lib().orc_prp(_addr(_buf(seed)), n, x))


def shuffle(shares, seeds: bytes, group: int = SHUF_ADD):
    """secShuffle (Alg. 5) of a 3-out-of-3 shared table: shares = three uint32 arrays [n, W];
    seeds = s12 || s23 || s31 (48 bytes).  Returns the three output share arrays [n, W]."""
    D = [np.ascontiguousarray(s, dtype=np.uint32) for s in shares]
    n, W = D[0].shape
    out = [np.zeros((n, W), dtype=np.uint32) for _ in range(3)]
    scratch = np.zeros(max(1, 8 * n * W), dtype=np.uint32)
    perm = np.zeros(max(1, 3 * n), dtype=np.uint64)
    sd = _buf(seeds)
    rc = lib().orc_shuffle(group, n, W, *[d.ctypes.data for d in D], _addr(sd), *[o.ctypes.data for o in out],
                           scratch.ctypes.data, perm.ctypes.data)
    if rc != 0:
        raise ValueError("oracle shuffle failed")
    return out


def fetch_multi(x_shares, table, attrs, seeds: bytes, cap: int):
    """secFetch case II: (count, [3 arrays (min(count, cap), 1 + len(attrs))]) of the kept records."""
    x = [np.ascontiguousarray(v, dtype=np.uint32) for v in x_shares]
    n = len(x[0])
    tarr, keep = _tables([table])
    at = np.ascontiguousarray(attrs, dtype=np.uint32)
    W = 2 + len(at)
    out = [np.zeros((max(1, cap), W - 1), dtype=np.uint32) for _ in range(3)]
    scratch = np.zeros(max(1, 14 * n * W), dtype=np.uint32)
    perm = np.zeros(max(1, 3 * n), dtype=np.uint64)
    m = lib().orc_fetch_multi(n, *[v.ctypes.data for v in x], tarr, len(at), at.ctypes.data, _addr(_buf(seeds)),
                              *[o.ctypes.data for o in out], cap, scratch.ctypes.data, perm.ctypes.data)
    del keep
    if m < 0:
        raise ValueError("oracle fetch_multi rejected its arguments")
    return int(m), [o[:min(m, cap)] for o in out]
