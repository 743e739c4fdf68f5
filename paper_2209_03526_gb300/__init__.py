"""GB300 library for OblivGM's secure predicate evaluation (arXiv 2209.03526).

Thin Python binding over the C ABI in ``include/oblivgm.h``: argument
marshalling only.  Every step of the evaluation (mask-open, DPF/DCF walks,
per-server sums, re-share, AND fold) runs in the library's CUDA kernels; the
token generation runs in the library's host C++.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the shared library cannot
be loaded every call raises.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

from . import _native as N
from ._native import (AES_BITSLICED, AES_TTABLE, ALL_PAIRS, COMBINE_AND, COMBINE_OR, COMBINE_XOR, EAGAIN, EBUSY, ECUDA, EFAULT_DEVICE, EINVAL,
                      ENOENT, ENOMEM, ERANGE, ETIMEOUT, KEY_DCF, KEY_DPF, POLL_LIMIT_DEFAULT_MS,
                      OK, PRED_EQ, PRED_RANGE, OblivgmError)
from .build import build

__all__ = ["Context", "keygen", "keygen_onehot", "build", "OblivgmError", "PRED_EQ", "PRED_RANGE", "KEY_DPF", "KEY_DCF",
           "COMBINE_AND", "COMBINE_XOR", "COMBINE_OR",
           "ALL_PAIRS", "version", "token_len", "fresh_token_size"]


def _lib():
    return N.load()


def version() -> int:
    return _lib().oblivgm_version()


def _pred_array(preds):
    arr = (N.Pred * len(preds))()
    for i, p in enumerate(preds):
        arr[i].kind, arr[i].table, arr[i].attr = int(p["kind"]), int(p["table"]), int(p["attr"])
        arr[i].group, arr[i].lo, arr[i].hi = int(p.get("group", 0)), int(p["lo"]), int(p.get("hi", p["lo"]))
        arr[i].combine = int(p.get("combine", COMBINE_AND))
    return arr


def token_len(preds, n_bits: int) -> int:
    """Bytes of each server's token (oblivgm_keygen size query)."""
    arr = _pred_array(preds)
    lens = (N.c_size * 3)()
    seed = (ctypes.c_uint8 * 16)()
    N.check(_lib().oblivgm_keygen(arr, len(preds), n_bits, ctypes.addressof(seed), None, 0, lens), "oblivgm_keygen")
    return lens[0]


def keygen(preds, n_bits: int, seed: bytes):
    """oblivgm_keygen: the three servers' tokens (bytes) for a list of predicate dicts."""
    arr = _pred_array(preds)
    L = token_len(preds, n_bits)
    bufs = [ctypes.create_string_buffer(L) for _ in range(3)]
    ptrs = (N.c_vp * 3)(*[ctypes.addressof(b) for b in bufs])
    lens = (N.c_size * 3)()
    sb = ctypes.create_string_buffer(bytes(seed), 16)
    N.check(_lib().oblivgm_keygen(arr, len(preds), n_bits, ctypes.addressof(sb), ptrs, L, lens), "oblivgm_keygen")
    return tuple(b.raw[:lens[i]] for i, b in enumerate(bufs))


def fresh_token_size(preds, n_bits: int, table_elems) -> int:
    """oblivgm_fresh_token_size: bytes of each server's fresh-key token."""
    arr = _pred_array(preds)
    te = (ctypes.c_uint64 * len(table_elems))(*[int(v) for v in table_elems])
    out = ctypes.c_uint64()
    N.check(_lib().oblivgm_fresh_token_size(arr, len(preds), n_bits, ctypes.addressof(te), len(table_elems),
                                            ctypes.byref(out)), "oblivgm_fresh_token_size")
    return out.value


def keygen_onehot(preds, n_bits: int, seed: bytes):
    """oblivgm_keygen_onehot: tokens of the one-hot mode (no mask, Z_2 keys, beta = 1)."""
    arr = _pred_array(preds)
    lens = (N.c_size * 3)()
    sb = ctypes.create_string_buffer(bytes(seed), 16)
    N.check(_lib().oblivgm_keygen_onehot(arr, len(preds), n_bits, ctypes.addressof(sb), None, 0, lens),
            "oblivgm_keygen_onehot")
    L = lens[0]
    bufs = [ctypes.create_string_buffer(L) for _ in range(3)]
    ptrs = (N.c_vp * 3)(*[ctypes.addressof(b) for b in bufs])
    N.check(_lib().oblivgm_keygen_onehot(arr, len(preds), n_bits, ctypes.addressof(sb), ptrs, L, lens),
            "oblivgm_keygen_onehot")
    return tuple(b.raw[:lens[i]] for i, b in enumerate(bufs))


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _tok_arrays(tokens):
    bufs = [ctypes.create_string_buffer(bytes(t), len(t)) for t in tokens]
    ptrs = (N.c_vp * 3)(*[ctypes.addressof(b) for b in bufs])
    lens = (N.c_size * 3)(*[len(t) for t in tokens])
    return bufs, ptrs, lens


class Context:
    """An oblivgm context on one CUDA device (oblivgm_create / oblivgm_destroy)."""

    def __init__(self, device: int = 0, prf_keys: bytes = bytes(range(48)), serve_arena_bytes: int = 0,
                 serve_max_inflight: int = 0):
        lib = _lib()
        cfg = N.Config()
        for i in range(3):
            for j in range(16):
                cfg.prf_keys[i][j] = prf_keys[16 * i + j]
        cfg.serve_arena_bytes = serve_arena_bytes
        cfg.serve_max_inflight = serve_max_inflight
        h = N.c_vp()
        N.check(lib.oblivgm_create(ctypes.byref(h), device, ctypes.byref(cfg)), "oblivgm_create")
        self._h = h
        self._lib = lib
        self.device = device
        self.prf_keys = bytes(prf_keys)

    # -------------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.oblivgm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sync(self, stream=None):
        N.check(self._lib.oblivgm_sync(self._h, _stream_handle(stream)), "oblivgm_sync")

    def launch_count(self) -> int:
        return self._lib.oblivgm_launch_count(self._h)

    # ----------------------------------------------------------- share store
    def load_shares(self, table_id: int, shares: Sequence, n_bits: int, stream=None):
        """shares: three uint32 arrays [n_attrs, n_elems] (torch CUDA/CPU tensors or numpy)."""
        ptrs, keep, kind, shape = [], [], None, None
        for s in shares:
            if hasattr(s, "is_cuda"):
                import torch
                t = s.contiguous()
                if t.dtype not in (torch.int32, torch.uint32):
                    raise TypeError("shares must be 32-bit tensors")
                k = N.MEM_DEVICE if t.is_cuda else N.MEM_HOST
                ptrs.append(t.data_ptr())
                shape = tuple(t.shape)
            else:
                import numpy as np
                t = np.ascontiguousarray(s, dtype=np.uint32)
                k = N.MEM_HOST
                ptrs.append(t.ctypes.data)
                shape = t.shape
            if kind is not None and k != kind:
                raise TypeError("all three share sets must live in the same memory")
            kind = k
            keep.append(t)
        n_attrs, n_elems = shape
        arr = (N.c_vp * 3)(*ptrs)
        N.check(self._lib.oblivgm_load_shares(self._h, table_id, n_elems, n_attrs, n_bits, arr, kind,
                                              _stream_handle(stream) if kind == N.MEM_DEVICE else None),
                "oblivgm_load_shares")

    def fetch_unique(self, query_id: int, group: int, table_id: int, x, attrs, out, stream=None):
        """secFetch case I: x = the group's three result share tensors; out = int32 CUDA tensor of
        3 * (1 + len(attrs)) words ([share set][index, attributes...])."""
        xs = (N.c_vp * 3)(*[t.data_ptr() for t in x])
        at = (N.c_u32 * max(1, len(attrs)))(*attrs)
        N.check(self._lib.oblivgm_fetch_unique(self._h, query_id, group, table_id, xs, len(attrs), at,
                                               out.data_ptr(), _stream_handle(stream)), "oblivgm_fetch_unique")

    def load_onehot(self, table_id: int, shares: Sequence, n_bits: int, stream=None):
        """shares: three uint32 CUDA tensors [n_attrs, n_elems, W] of binary one-hot shares."""
        ts = [s.contiguous() for s in shares]
        n_attrs, n_elems = ts[0].shape[0], ts[0].shape[1]
        arr = (N.c_vp * 3)(*[t.data_ptr() for t in ts])
        kind = N.MEM_DEVICE if ts[0].is_cuda else N.MEM_HOST
        N.check(self._lib.oblivgm_load_onehot(self._h, table_id, n_elems, n_attrs, n_bits, arr, kind,
                                              _stream_handle(stream) if kind == N.MEM_DEVICE else None),
                "oblivgm_load_onehot")

    def filter_onehot(self, query_id: int, tokens, outs, stream=None):
        """outs: per AND-group three int32 CUDA tensors of ceil(n_elems / 32) packed words."""
        _, tp, tl = _tok_arrays(tokens)
        flat = [t.data_ptr() for g in outs for t in g]
        arr = (N.c_vp * len(flat))(*flat)
        N.check(self._lib.oblivgm_filter_onehot(self._h, query_id, tp, tl, len(outs), arr, _stream_handle(stream)),
                "oblivgm_filter_onehot")

    def unload_shares(self, table_id: int):
        N.check(self._lib.oblivgm_unload_shares(self._h, table_id), "oblivgm_unload_shares")

    # ------------------------------------------------------------ raw batches
    def _eval(self, fn, name, keys: bytes, n_keys: int, points, key_of_point, out, all_pairs: bool, stream):
        kb = ctypes.create_string_buffer(bytes(keys), len(keys))
        N.check(fn(self._h, ctypes.addressof(kb), n_keys, points.data_ptr(),
                   key_of_point.data_ptr() if key_of_point is not None else None, points.numel(),
                   ALL_PAIRS if all_pairs else 0, out.data_ptr(), out.numel(), _stream_handle(stream)), name)

    def keygen_device(self, kind: int, n_bits: int, alpha, beta, seed: bytes, out, stream=None):
        """oblivgm_keygen_device: len(alpha) key pairs into the uint8 CUDA tensor out."""
        sb = ctypes.create_string_buffer(bytes(seed), 16)
        N.check(self._lib.oblivgm_keygen_device(self._h, kind, n_bits, alpha.numel(), alpha.data_ptr(),
                                                beta.data_ptr(), ctypes.addressof(sb), out.data_ptr(), out.numel(),
                                                _stream_handle(stream)), "oblivgm_keygen_device")

    def eval_device_keys(self, kind: int, n_bits: int, keys, n_keys: int, points, out, key_of_point=None,
                         all_pairs=False, stream=None):
        """Raw Eval with device-resident wire keys (OBLIVGM_KEYS_DEVICE)."""
        fn = self._lib.oblivgm_eval_dpf_batch if kind == KEY_DPF else self._lib.oblivgm_eval_dcf_batch
        flags = N.KEYS_DEVICE | (n_bits << 8) | (ALL_PAIRS if all_pairs else 0)
        N.check(fn(self._h, keys.data_ptr(), n_keys, points.data_ptr(),
                   key_of_point.data_ptr() if key_of_point is not None else None, points.numel(), flags,
                   out.data_ptr(), out.numel(), _stream_handle(stream)), "oblivgm_eval_batch")

    def eval_dpf_batch(self, keys: bytes, n_keys: int, points, out, key_of_point=None, all_pairs=False, stream=None):
        self._eval(self._lib.oblivgm_eval_dpf_batch, "oblivgm_eval_dpf_batch", keys, n_keys, points, key_of_point,
                   out, all_pairs, stream)

    def eval_dcf_batch(self, keys: bytes, n_keys: int, points, out, key_of_point=None, all_pairs=False, stream=None):
        self._eval(self._lib.oblivgm_eval_dcf_batch, "oblivgm_eval_dcf_batch", keys, n_keys, points, key_of_point,
                   out, all_pairs, stream)

    # ---------------------------------------------------- filter and combine
    def filter_and_combine(self, query_id: int, tokens, outs, stream=None):
        """outs: list over AND-groups of three uint32 CUDA tensors (share sets 1..3)."""
        _, tp, tl = _tok_arrays(tokens)
        flat = [t.data_ptr() for g in outs for t in g]
        arr = (N.c_vp * len(flat))(*flat)
        N.check(self._lib.oblivgm_filter_and_combine(self._h, query_id, tp, tl, len(outs), arr,
                                                     _stream_handle(stream)), "oblivgm_filter_and_combine")

    def keygen_fresh(self, preds, n_bits: int, table_elems, seed: bytes, toks, stream=None):
        """oblivgm_keygen_fresh: the client's fresh-key tokens into three uint8 CUDA tensors."""
        arr = _pred_array(preds)
        te = (ctypes.c_uint64 * len(table_elems))(*[int(v) for v in table_elems])
        sb = ctypes.create_string_buffer(bytes(seed), 16)
        ptrs = (N.c_vp * 3)(*[t.data_ptr() for t in toks])
        cap = min(t.numel() for t in toks)
        N.check(self._lib.oblivgm_keygen_fresh(self._h, arr, len(preds), n_bits, ctypes.addressof(te),
                                               len(table_elems), ctypes.addressof(sb), ptrs, cap,
                                               _stream_handle(stream)), "oblivgm_keygen_fresh")

    def filter_fresh(self, query_id: int, toks, outs, stream=None):
        """oblivgm_filter_fresh on three device-resident fresh tokens (uint8 CUDA tensors)."""
        ptrs = (N.c_vp * 3)(*[t.data_ptr() for t in toks])
        flat = [t.data_ptr() for g in outs for t in g]
        arr = (N.c_vp * len(flat))(*flat)
        cap = min(t.numel() * t.element_size() for t in toks)
        N.check(self._lib.oblivgm_filter_fresh(self._h, query_id, ptrs, cap, len(outs), arr, _stream_handle(stream)),
                "oblivgm_filter_fresh")

    def shuffle(self, ins, seeds: bytes, outs, group: int = 0, stream=None):
        """oblivgm_shuffle: ins / outs three int32 CUDA tensors [n_rows, width]; seeds s12 || s23 || s31."""
        n, w = ins[0].shape
        ip = (N.c_vp * 3)(*[t.data_ptr() for t in ins])
        op = (N.c_vp * 3)(*[t.data_ptr() for t in outs])
        sb = ctypes.create_string_buffer(bytes(seeds), 48)
        N.check(self._lib.oblivgm_shuffle(self._h, group, n, w, ip, ctypes.addressof(sb), op, _stream_handle(stream)),
                "oblivgm_shuffle")

    def fetch_multi(self, table_id: int, x, attrs, seeds: bytes, outs, stream=None) -> int:
        """oblivgm_fetch_multi (secFetch case II): outs three int32 CUDA tensors [cap, 1 + len(attrs)];
        returns the number of matched records."""
        xp = (N.c_vp * 3)(*[t.data_ptr() for t in x])
        op = (N.c_vp * 3)(*[t.data_ptr() for t in outs])
        at = (ctypes.c_uint32 * max(1, len(attrs)))(*attrs)
        sb = ctypes.create_string_buffer(bytes(seeds), 48)
        cnt = ctypes.c_uint64()
        N.check(self._lib.oblivgm_fetch_multi(self._h, table_id, xp, len(attrs), ctypes.addressof(at),
                                              ctypes.addressof(sb), op, outs[0].shape[0], ctypes.byref(cnt),
                                              _stream_handle(stream)), "oblivgm_fetch_multi")
        return cnt.value

    def filter_plain(self, query_id: int, tokens, outs, stream=None):
        """The plain per-query path (one launch per key half, global-memory AES tables)."""
        _, tp, tl = _tok_arrays(tokens)
        flat = [t.data_ptr() for g in outs for t in g]
        arr = (N.c_vp * len(flat))(*flat)
        N.check(self._lib.oblivgm_filter_plain(self._h, query_id, tp, tl, len(outs), arr, _stream_handle(stream)),
                "oblivgm_filter_plain")

    def filter_and_combine_noalloc(self, query_id: int, tokens, outs, stream=None):
        """As filter_and_combine, with the workspace in the library's fixed device array
        (no device allocation during the call; calls must not overlap on the GPU)."""
        _, tp, tl = _tok_arrays(tokens)
        flat = [t.data_ptr() for g in outs for t in g]
        arr = (N.c_vp * len(flat))(*flat)
        N.check(self._lib.oblivgm_filter_and_combine_noalloc(self._h, query_id, tp, tl, len(outs), arr,
                                                             _stream_handle(stream)),
                "oblivgm_filter_and_combine_noalloc")

    def _batch_args(self, query_ids, tokens_list, outs_list):
        nq = len(query_ids)
        keep = []
        tok_ptrs = (N.c_vp * (3 * nq))()
        tok_lens = (N.c_size * (3 * nq))()
        for q, toks in enumerate(tokens_list):
            for i in range(3):
                b = ctypes.create_string_buffer(bytes(toks[i]), len(toks[i]))
                keep.append(b)
                tok_ptrs[3 * q + i] = ctypes.addressof(b)
                tok_lens[3 * q + i] = len(toks[i])
        ng = (N.c_u32 * nq)(*[len(o) for o in outs_list])
        out_arrays = (N.c_vp * nq)()
        for q, outs in enumerate(outs_list):
            flat = [t.data_ptr() for g in outs for t in g]
            a = (N.c_vp * len(flat))(*flat)
            keep.append(a)
            out_arrays[q] = ctypes.addressof(a)
        qids = (N.c_u32 * nq)(*query_ids)
        return keep, qids, tok_ptrs, tok_lens, ng, out_arrays

    def plan_create(self, query_ids, tokens_list, outs_list):
        """A prepared batch (oblivgm_plan_create); launch it with plan_launch, free with plan_destroy."""
        keep, qids, tp, tl, ng, oa = self._batch_args(query_ids, tokens_list, outs_list)
        h = N.c_vp()
        N.check(self._lib.oblivgm_plan_create(self._h, len(query_ids), qids, tp, tl, ng, oa, ctypes.byref(h)),
                "oblivgm_plan_create")
        return h

    def plan_launch(self, plan, stream=None):
        N.check(self._lib.oblivgm_plan_launch(plan, _stream_handle(stream)), "oblivgm_plan_launch")

    def plan_describe(self, plan) -> dict:
        """The launch a plan fixed (oblivgm_plan_describe)."""
        wp, th, tile, grid = (ctypes.c_uint32() for _ in range(4))
        items = ctypes.c_uint64()
        N.check(self._lib.oblivgm_plan_describe(plan, ctypes.byref(wp), ctypes.byref(th), ctypes.byref(tile),
                                                ctypes.byref(items), ctypes.byref(grid)), "oblivgm_plan_describe")
        return {"kernel": "k_filter_wp" if wp.value else "k_filter", "threads": th.value, "tile": tile.value,
                "items": items.value, "grid": grid.value}

    def plan_destroy(self, plan):
        N.check(self._lib.oblivgm_plan_destroy(plan), "oblivgm_plan_destroy")

    def filter_batch(self, query_ids, tokens_list, outs_list, stream=None):
        """Several queries in one persistent launch; outs_list[q] as in filter_and_combine."""
        nq = len(query_ids)
        keep = []
        tok_ptrs = (N.c_vp * (3 * nq))()
        tok_lens = (N.c_size * (3 * nq))()
        for q, toks in enumerate(tokens_list):
            for i in range(3):
                b = ctypes.create_string_buffer(bytes(toks[i]), len(toks[i]))
                keep.append(b)
                tok_ptrs[3 * q + i] = ctypes.addressof(b)
                tok_lens[3 * q + i] = len(toks[i])
        ng = (N.c_u32 * nq)(*[len(o) for o in outs_list])
        out_arrays = (N.c_vp * nq)()
        for q, outs in enumerate(outs_list):
            flat = [t.data_ptr() for g in outs for t in g]
            a = (N.c_vp * len(flat))(*flat)
            keep.append(a)
            out_arrays[q] = ctypes.addressof(a)
        qids = (N.c_u32 * nq)(*query_ids)
        N.check(self._lib.oblivgm_filter_batch(self._h, nq, qids, tok_ptrs, tok_lens, ng, out_arrays,
                                               _stream_handle(stream)), "oblivgm_filter_batch")

    # ---------------------------------------------------------------- serving
    def submit(self, tokens) -> int:
        """Returns a ticket, or raises OblivgmError with status EAGAIN when not admitted."""
        _, tp, tl = _tok_arrays(tokens)
        t = N.c_u64()
        N.check(self._lib.oblivgm_submit(self._h, tp, tl, ctypes.byref(t)), "oblivgm_submit")
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Returns None if not finished (timeout_ms == 0), else a dict describing the result."""
        r = N.Result()
        st = self._lib.oblivgm_poll(self._h, ticket, timeout_ms, ctypes.byref(r))
        if st == EAGAIN:
            return None
        N.check(st, "oblivgm_poll")
        groups = []
        for g in range(r.n_groups):
            groups.append({"table": r.table[g], "n_elems": r.n_elems[g], "shares": [r.shares[g][j] for j in range(3)]})
        return {"ticket": r.ticket, "latency_ms": r.latency_ms, "groups": groups}

    def set_poll_limit(self, max_ms: int) -> int:
        """Longest wait of any poll (a negative timeout waits this long); returns the old limit."""
        prev = ctypes.c_uint32(0)
        N.check(self._lib.oblivgm_set_poll_limit(self._h, max_ms, ctypes.byref(prev)), "oblivgm_set_poll_limit")
        return prev.value

    def release(self, ticket: int):
        N.check(self._lib.oblivgm_release(self._h, ticket), "oblivgm_release")

    def serve_stats(self):
        v = [N.c_u64() for _ in range(4)]
        N.check(self._lib.oblivgm_serve_stats(self._h, *[ctypes.byref(x) for x in v]), "oblivgm_serve_stats")
        return {"admitted": v[0].value, "completed": v[1].value, "rejected": v[2].value, "reserved_bytes": v[3].value}

    # ----------------------------------------------------------------- tuning
    def autotune(self):
        t, e = N.c_u32(), N.c_u32()
        N.check(self._lib.oblivgm_autotune(self._h, ctypes.byref(t), ctypes.byref(e)), "oblivgm_autotune")
        return t.value, e.value

    def prg_batch(self, layout: int, key: int, first: int, n_blocks: int, out, parity: bool = False, stream=None):
        """H_K(B_c) for the counter blocks c = first .. first + n_blocks - 1 (multiples of 32) in the
        given AES layout: out gets 4 words per block, or one parity word per 32 blocks."""
        N.check(self._lib.oblivgm_prg_batch(self._h, layout, key, first, n_blocks, N.PRG_PARITY if parity else 0,
                                            out.data_ptr(), out.numel(), _stream_handle(stream)),
                "oblivgm_prg_batch")

    def autotune_aes_layout(self):
        """Time both AES layouts of the PRG; returns (chosen layout, T-table blocks/s, bitsliced blocks/s)."""
        lay = ctypes.c_uint32()
        tt, bs = ctypes.c_double(), ctypes.c_double()
        N.check(self._lib.oblivgm_autotune_aes_layout(self._h, ctypes.byref(lay), ctypes.byref(tt), ctypes.byref(bs)),
                "oblivgm_autotune_aes_layout")
        return lay.value, tt.value, bs.value

    def test_fail_next_alloc(self):
        """Failure-path test hook: the next device workspace allocation reports ENOMEM."""
        N.check(self._lib.oblivgm_test_fail_next_alloc(self._h), "oblivgm_test_fail_next_alloc")

    def test_expire_next_wait(self, limit_us: int):
        """Failure-path test hook: the next fused launch's key-staging waits run out after limit_us."""
        N.check(self._lib.oblivgm_test_expire_next_wait(self._h, limit_us), "oblivgm_test_expire_next_wait")

    def set_schedule(self, threads: int = 0, elems_per_thread: int = 0):
        N.check(self._lib.oblivgm_set_schedule(self._h, threads, elems_per_thread), "oblivgm_set_schedule")

    def set_walk_parallel_tile(self, tile: int) -> int:
        """Fix the walk-parallel kernel's elements per tile (1..40; 0: chosen per launch).
        Returns the setting it replaces."""
        prev = ctypes.c_uint32(0)
        N.check(self._lib.oblivgm_set_walk_parallel_tile(self._h, tile, ctypes.byref(prev)),
                "oblivgm_set_walk_parallel_tile")
        return prev.value

    def set_walk_parallel(self, max_elems: int) -> int:
        """Batches of at most max_elems elements in all run the walk-parallel kernel (0: never,
        2**64 - 1: always).  Returns the setting it replaces."""
        prev = ctypes.c_uint64(0)
        N.check(self._lib.oblivgm_set_walk_parallel(self._h, max_elems, ctypes.byref(prev)),
                "oblivgm_set_walk_parallel")
        return prev.value


class _DeviceWords:
    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False), "version": 3}


def device_words(ptr: int, n: int, device: int = 0):
    """A zero-copy int32 CUDA tensor over n words at a library-owned device address (served results)."""
    import torch
    return torch.as_tensor(_DeviceWords(ptr, n), device=f"cuda:{device}")
