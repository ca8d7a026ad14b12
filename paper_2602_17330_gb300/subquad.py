"""Python binding of libsubquad (the C ABI declared in include/subquad.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory and the stream; tensors are passed to the C
entry points as raw device pointers.  There is no CPU path: if the shared
library is missing or fails to load, every call raises.

Two layers:
* ``lib()`` -- the ctypes handle, with ``subquad_*`` functions under their C
  names and signatures;
* ``Context`` -- owns a ``subquad_ctx`` bound to a device and a stream, with one
  method per entry point (``ctx.sign(...)`` calls ``subquad_sign``), allocating
  outputs as torch tensors.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsubquad.so")

SUBQUAD_OK = 0
SUBQUAD_ERR_ARG = -1
SUBQUAD_ERR_CAPACITY = -2
SUBQUAD_ERR_CUDA = -3
SUBQUAD_ERR_TIMEOUT = -4
SUBQUAD_ERR_NOMEM = -5
SUBQUAD_ERR_INPUT = -6
SUBQUAD_ERR_INTERNAL = -7

PROF_NAMES = ["sign", "band", "band_partition", "band_group", "band_emit", "band_pairsort", "align", "align_bin", "self",
              "fuse", "edit"]

TUNE_ALIGN_SHAPE = 0
TUNE_BAND_PART_LOG2 = 1
TUNE_FUSE_LANES = 2

_c = ctypes
_P = _c.c_void_p
_I64 = _c.c_int64

# name -> (restype, argtypes); every function declared in include/subquad.h
SIGNATURES = {
    "subquad_strerror": (_c.c_char_p, [_c.c_int]),
    "subquad_version": (_c.c_int, []),
    "subquad_create": (_c.c_int, [_c.POINTER(_P), _c.c_int, _P]),
    "subquad_destroy": (_c.c_int, [_P]),
    "subquad_set_stream": (_c.c_int, [_P, _P]),
    "subquad_check": (_c.c_int, [_P]),
    "subquad_scratch_bytes": (_I64, [_P]),
    "subquad_launch_count": (_I64, [_P]),
    "subquad_profile_enable": (_c.c_int, [_P, _c.c_int]),
    "subquad_profile_reset": (_c.c_int, [_P]),
    "subquad_profile_read": (_c.c_int, [_P, _c.c_int, _c.POINTER(_c.c_double), _c.POINTER(_I64)]),
    "subquad_set_tuning": (_c.c_int, [_P, _c.c_int, _c.c_int]),
    "subquad_get_tuning": (_c.c_int, [_P, _c.c_int, _c.POINTER(_c.c_int)]),
    "subquad_default_matrix": (_c.c_int, [_P]),
    "subquad_set_matrix": (_c.c_int, [_P, _P]),
    "subquad_pack_stride": (_c.c_int, [_c.c_int]),
    "subquad_pack": (_c.c_int, [_P, _P, _c.c_int, _P, _I64, _c.c_int, _P]),
    "subquad_sign": (_c.c_int, [_P, _P, _c.c_int, _I64, _c.c_int, _c.c_int, _c.c_int, _P, _P, _P]),
    "subquad_band_candidates": (_c.c_int, [_P, _P, _I64, _c.c_int, _c.c_int, _c.c_int32, _P, _I64,
                                           _c.POINTER(_I64)]),
    "subquad_band_candidates_async": (_c.c_int, [_P, _P, _I64, _c.c_int, _c.c_int, _c.c_int32, _P, _P, _I64, _P]),
    "subquad_band_stream_create": (_c.c_int, [_P, _P, _I64, _c.c_int, _c.c_int, _c.c_int32, _P, _c.POINTER(_P),
                                              _c.POINTER(_c.c_uint64)]),
    "subquad_band_stream_next": (_c.c_int, [_P, _P, _P, _I64, _c.POINTER(_I64), _c.POINTER(_c.c_int)]),
    "subquad_band_stream_reset": (_c.c_int, [_P]),
    "subquad_band_stream_destroy": (None, [_P]),
    "subquad_align_score_binned_async": (_c.c_int, [_P, _P, _c.c_int, _P, _P, _I64, _c.c_int, _c.c_int, _P]),
    "subquad_fuse_forward_async": (_c.c_int, [_P, _P, _P, _I64, _P, _P, _P, _c.c_int, _P, _c.c_int, _P, _c.c_int,
                                              _P, _P]),
    "subquad_align_score": (_c.c_int, [_P, _P, _c.c_int, _P, _I64, _c.c_int, _c.c_int, _P]),
    "subquad_self_scores": (_c.c_int, [_P, _P, _c.c_int, _I64, _c.c_int, _c.c_int, _P]),
    "subquad_align_score_binned": (_c.c_int, [_P, _P, _c.c_int, _P, _I64, _c.c_int, _c.c_int, _P]),
    "subquad_self_scores_binned": (_c.c_int, [_P, _P, _c.c_int, _I64, _c.c_int, _c.c_int, _P]),
    "subquad_fuse_forward": (_c.c_int, [_P, _P, _I64, _P, _P, _P, _c.c_int, _P, _c.c_int, _P, _c.c_int, _P, _P]),
    "subquad_topk_candidates": (_c.c_int, [_P, _P, _P, _I64, _I64, _P, _P, _P, _P, _P, _P, _I64, _c.c_int, _P,
                                           _P]),
    "subquad_topk_bruteforce": (_c.c_int, [_P, _P, _c.c_int, _I64, _P, _c.c_int, _c.c_int, _P, _I64, _c.c_int, _P,
                                           _P]),
    "subquad_pair_labels": (_c.c_int, [_P, _P, _I64, _P, _P, _P, _P]),
    "subquad_pair_weights": (_c.c_int, [_P, _P, _I64, _c.c_int, _P]),
    "subquad_bce_loss": (_c.c_int, [_P, _P, _P, _P, _I64, _P, _P]),
    "subquad_pair_index": (_c.c_int, [_P, _P, _I64, _I64, _P, _P, _P, _P]),
    "subquad_fuse_backward": (_c.c_int, [_P, _P, _I64, _P, _P, _P, _c.c_int, _P, _I64, _c.c_int, _P, _c.c_int, _P,
                                         _P, _P, _P, _P, _P, _P]),
    "subquad_fuse_backward_params_noalloc": (_c.c_int, [_P, _P, _I64, _P, _P, _P, _c.c_int, _P, _c.c_int, _P,
                                                        _c.c_int, _P, _P]),
    "subquad_fuse_forward_mc": (_c.c_int, [_P, _P, _I64, _P, _P, _P, _c.c_int, _P, _c.c_int, _P, _c.c_int, _P,
                                           _c.c_int, _c.c_int, _P, _P]),
    "subquad_fuse_backward_mc": (_c.c_int, [_P, _P, _I64, _P, _P, _P, _c.c_int, _P, _I64, _c.c_int, _P, _c.c_int, _P,
                                            _c.c_int, _c.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "subquad_sig_sequence_major": (_c.c_int, [_P, _P, _I64, _c.c_int, _c.c_int, _P]),
    "subquad_default_edit_costs": (_c.c_int, [_P]),
    "subquad_set_edit_costs": (_c.c_int, [_P, _c.c_int, _P]),
    "subquad_edit_distance": (_c.c_int, [_P, _P, _c.c_int, _P, _I64, _P]),
    "subquad_edit_distance_async": (_c.c_int, [_P, _P, _c.c_int, _P, _P, _I64, _P]),
    "subquad_graph_components": (_c.c_int, [_P, _P, _P, _I64, _I64, _c.c_double, _P, _P]),
    "subquad_rmt_threshold": (_c.c_int, [_P, _P, _P, _I64, _I64, _P, _c.c_int, _c.c_int, _c.c_double, _P, _P, _P, _P,
                                         _P]),
    "subquad_graph_prune": (_c.c_int, [_P, _P, _P, _I64, _c.c_double, _P, _P, _P]),
    "subquad_cluster_js": (_c.c_int, [_P, _P, _P, _I64, _c.c_int, _P]),
    "subquad_adam_step": (_c.c_int, [_P, _P, _P, _P, _P, _I64, _c.c_int, _c.c_float, _c.c_float, _c.c_float,
                                     _c.c_float]),
}

_lib = None


class SubquadError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        text = lib().subquad_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {text} (status {status})")


def lib():
    """Load libsubquad.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsubquad.so not found at {LIB_PATH}; build it with __graft_entry__.build()")
    handle = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(handle, name)
        fn.restype = res
        fn.argtypes = args
    _lib = handle
    return handle


def _check(status: int, where: str) -> None:
    if status != SUBQUAD_OK:
        raise SubquadError(status, where)


def default_matrix():
    """The library's built-in BLOSUM62 as a list of 400 ints (host-only)."""
    buf = (ctypes.c_int8 * 400)()
    _check(lib().subquad_default_matrix(ctypes.cast(buf, _P)), "subquad_default_matrix")
    return list(buf)


def default_edit_costs():
    """The library's default edit-distance substitution costs (400 ints, half
    units; host-only)."""
    buf = (ctypes.c_uint8 * 400)()
    _check(lib().subquad_default_edit_costs(ctypes.cast(buf, _P)), "subquad_default_edit_costs")
    return list(buf)


def pack_stride(max_len: int) -> int:
    return int(lib().subquad_pack_stride(max_len))


def _ptr(t):
    return None if t is None else _P(t.data_ptr())


class Context:
    """A subquad_ctx bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        handle = _P()
        _check(lib().subquad_create(ctypes.byref(handle), device, _P(stream.cuda_stream)), "subquad_create")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            lib().subquad_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- context ---------------------------------------------------------------
    def set_stream(self, stream):
        _check(lib().subquad_set_stream(self.handle, _P(stream.cuda_stream)), "subquad_set_stream")
        self.stream = stream

    def check(self):
        _check(lib().subquad_check(self.handle), "subquad_check")

    def scratch_bytes(self) -> int:
        return int(lib().subquad_scratch_bytes(self.handle))

    def launch_count(self) -> int:
        return int(lib().subquad_launch_count(self.handle))

    def profile(self, on: bool = True):
        _check(lib().subquad_profile_enable(self.handle, 1 if on else 0), "subquad_profile_enable")

    def profile_reset(self):
        _check(lib().subquad_profile_reset(self.handle), "subquad_profile_reset")

    def profile_read(self) -> dict:
        """{kernel tag: (total ms, launches)} since the last reset."""
        out = {}
        for k, name in enumerate(PROF_NAMES):
            t, c = ctypes.c_double(0.0), _I64(0)
            _check(lib().subquad_profile_read(self.handle, k, ctypes.byref(t), ctypes.byref(c)), "subquad_profile_read")
            out[name] = (float(t.value), int(c.value))
        return out

    def set_tuning(self, key: int, value: int):
        _check(lib().subquad_set_tuning(self.handle, key, value), "subquad_set_tuning")

    def get_tuning(self, key: int) -> int:
        v = ctypes.c_int(0)
        _check(lib().subquad_get_tuning(self.handle, key, ctypes.byref(v)), "subquad_get_tuning")
        return int(v.value)

    def set_matrix(self, matrix=None):
        if matrix is None:
            _check(lib().subquad_set_matrix(self.handle, None), "subquad_set_matrix")
            return
        buf = (ctypes.c_int8 * 400)(*[int(v) for v in list(matrix)])
        _check(lib().subquad_set_matrix(self.handle, ctypes.cast(buf, _P)), "subquad_set_matrix")

    def set_edit_costs(self, indel: int = 2, sub=None):
        buf = None
        if sub is not None:
            buf = (ctypes.c_uint8 * 400)(*[int(v) for v in list(sub)])
        _check(lib().subquad_set_edit_costs(self.handle, indel, None if buf is None else ctypes.cast(buf, _P)),
               "subquad_set_edit_costs")

    # -- helpers ---------------------------------------------------------------
    def _dev(self, t, dtype):
        t = t.to(self.device)
        if t.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {t.dtype}")
        return t.contiguous()

    def _empty(self, shape, dtype):
        return self.torch.empty(shape, dtype=dtype, device=self.device)

    # -- entry points ----------------------------------------------------------
    def pack(self, codes, lens, stride: int):
        """codes uint8 [n, code_stride], lens uint8 [n] -> packed uint8 [n, stride]."""
        torch = self.torch
        codes = self._dev(codes, torch.uint8)
        lens = self._dev(lens, torch.uint8)
        n = int(lens.shape[0])
        out = self._empty((n, stride), torch.uint8)
        _check(lib().subquad_pack(self.handle, _ptr(codes), int(codes.shape[1]) if n else 1, _ptr(lens), n, stride,
                                  _ptr(out)), "subquad_pack")
        return out

    def sign(self, packed, n: int, k: int, a, b, bands: int, rows: int):
        """-> int32 [bands, n, rows] (uint32 bit patterns)."""
        torch = self.torch
        a = self._dev(a, torch.int32)
        b = self._dev(b, torch.int32)
        out = self._empty((bands, n, rows), torch.int32)
        _check(lib().subquad_sign(self.handle, _ptr(packed), int(packed.shape[1]), n, k, bands, rows, _ptr(a),
                                  _ptr(b), _ptr(out)), "subquad_sign")
        return out

    def band_candidates(self, sig, n: int, bands: int, rows: int, bucket_cap: int = 0, capacity: int | None = None,
                        out=None):
        """-> int32 [|C|, 2] sorted candidate pairs.  Retries once with the
        required capacity when the first guess is too small."""
        torch = self.torch
        if out is None:
            capacity = capacity if capacity is not None else max(1 << 16, 8 * n)
            out = self._empty((capacity, 2), torch.int32)
        else:
            capacity = int(out.shape[0])
        count = _I64(0)
        st = lib().subquad_band_candidates(self.handle, _ptr(sig), n, bands, rows, bucket_cap, _ptr(out), capacity,
                                           ctypes.byref(count))
        if st == SUBQUAD_ERR_CAPACITY:
            out = self._empty((int(count.value), 2), torch.int32)
            st = lib().subquad_band_candidates(self.handle, _ptr(sig), n, bands, rows, bucket_cap, _ptr(out),
                                               int(count.value), ctypes.byref(count))
        _check(st, "subquad_band_candidates")
        return out[: int(count.value)]

    # -- batched, graph-capturable forms (counts stay on the device) ----------
    def band_candidates_async(self, sig, n: int, bands: int, rows: int, bucket_cap: int, pairs_out, d_num_pairs,
                              donor=None):
        """Writes |C| to the device tensor d_num_pairs (int64 [1]); no sync."""
        _check(lib().subquad_band_candidates_async(self.handle, _ptr(sig), n, bands, rows, bucket_cap, _ptr(donor),
                                                   _ptr(pairs_out), int(pairs_out.shape[0]), _ptr(d_num_pairs)),
               "subquad_band_candidates_async")

    def band_stream(self, sig, n: int, bands: int, rows: int, bucket_cap: int = 0, donor=None,
                    capacity: int = 1 << 22):
        """Streamed candidates: yields int32 [k, 2] device tensors (each sorted
        lexicographically; together exactly the pairs of
        band_candidates_async).  A buffer of ``capacity`` pairs is reused:
        consume (or copy) each batch before asking for the next."""
        torch = self.torch
        handle = _P()
        total = _c.c_uint64(0)
        _check(lib().subquad_band_stream_create(self.handle, _ptr(sig), n, bands, rows, bucket_cap, _ptr(donor),
                                                _c.byref(handle), _c.byref(total)), "subquad_band_stream_create")
        buf = self._empty((capacity, 2), torch.int32)
        try:
            done = _c.c_int(0)
            while not done.value:
                count = _I64(0)
                _check(lib().subquad_band_stream_next(self.handle, handle, _ptr(buf), capacity, _c.byref(count),
                                                      _c.byref(done)), "subquad_band_stream_next")
                if count.value:
                    yield buf[:count.value]
        finally:
            lib().subquad_band_stream_destroy(handle)

    def align_score_binned_async(self, packed, pairs, d_m, out, gap_open: int = 10, gap_extend: int = 1):
        _check(lib().subquad_align_score_binned_async(self.handle, _ptr(packed), int(packed.shape[1]), _ptr(pairs),
                                                      _ptr(d_m), int(pairs.shape[0]), gap_open, gap_extend,
                                                      _ptr(out)), "subquad_align_score_binned_async")

    def fuse_forward_async(self, pairs, d_m, sw, self_sc, packed, emb, params, hidden: int, out, alpha=None):
        _check(lib().subquad_fuse_forward_async(self.handle, _ptr(pairs), _ptr(d_m), int(pairs.shape[0]), _ptr(sw),
                                                _ptr(self_sc), _ptr(packed), int(packed.shape[1]), _ptr(emb),
                                                int(emb.shape[1]), _ptr(params), hidden, _ptr(out), _ptr(alpha)),
               "subquad_fuse_forward_async")

    def align_score(self, packed, pairs, gap_open: int = 10, gap_extend: int = 1, out=None, binned: bool = False):
        """binned=False: subquad_align_score (pairs in input order);
        binned=True: subquad_align_score_binned (length-binned work list)."""
        torch = self.torch
        m = int(pairs.shape[0])
        out = self._empty((m,), torch.int32) if out is None else out
        name = "subquad_align_score_binned" if binned else "subquad_align_score"
        _check(getattr(lib(), name)(self.handle, _ptr(packed), int(packed.shape[1]), _ptr(pairs), m, gap_open,
                                    gap_extend, _ptr(out)), name)
        return out

    def edit_distance(self, packed, pairs, out=None):
        """subquad_edit_distance: int32 [m] distances under the context's costs."""
        torch = self.torch
        m = int(pairs.shape[0])
        out = self._empty((m,), torch.int32) if out is None else out
        _check(lib().subquad_edit_distance(self.handle, _ptr(packed), int(packed.shape[1]), _ptr(pairs), m, _ptr(out)),
               "subquad_edit_distance")
        return out

    def edit_distance_async(self, packed, pairs, d_m, out):
        _check(lib().subquad_edit_distance_async(self.handle, _ptr(packed), int(packed.shape[1]), _ptr(pairs),
                                                 _ptr(d_m), int(pairs.shape[0]), _ptr(out)),
               "subquad_edit_distance_async")

    def self_scores(self, packed, gap_open: int = 10, gap_extend: int = 1, out=None, binned: bool = False):
        torch = self.torch
        n = int(packed.shape[0])
        out = self._empty((n,), torch.int32) if out is None else out
        name = "subquad_self_scores_binned" if binned else "subquad_self_scores"
        _check(getattr(lib(), name)(self.handle, _ptr(packed), int(packed.shape[1]), n, gap_open, gap_extend,
                                    _ptr(out)), name)
        return out

    def fuse_forward(self, pairs, sw, self_sc, packed, emb, params, hidden: int, want_alpha: bool = False,
                     out=None, alpha=None):
        torch = self.torch
        m = int(pairs.shape[0])
        emb = self._dev(emb, torch.float32)
        params = self._dev(params, torch.float32)
        out = self._empty((m,), torch.float32) if out is None else out
        if want_alpha and alpha is None:
            alpha = self._empty((m,), torch.float32)
        _check(lib().subquad_fuse_forward(self.handle, _ptr(pairs), m, _ptr(sw), _ptr(self_sc), _ptr(packed),
                                          int(packed.shape[1]), _ptr(emb), int(emb.shape[1]), _ptr(params), hidden,
                                          _ptr(out), _ptr(alpha) if want_alpha else None), "subquad_fuse_forward")
        return (out, alpha) if want_alpha else out


    # -- cross-donor retrieval -----------------------------------------------
    def topk_candidates(self, pairs, scores, n: int, donor, queries, k: int, index=None):
        """-> (top_id uint32-as-int32 [nq, k], top_score int32 [nq, k])."""
        torch = self.torch
        m = int(pairs.shape[0])
        donor = self._dev(donor, torch.int32)
        queries = self._dev(queries, torch.int32)
        nq = int(queries.shape[0])
        index = self.pair_index(pairs, n) if index is None else index
        ids = self._empty((nq, k), torch.int32)
        sc = self._empty((nq, k), torch.int32)
        _check(lib().subquad_topk_candidates(self.handle, _ptr(pairs), _ptr(scores), m, n, _ptr(donor),
                                             _ptr(index["perm_i"]), _ptr(index["off_i"]), _ptr(index["perm_j"]),
                                             _ptr(index["off_j"]), _ptr(queries), nq, k, _ptr(ids), _ptr(sc)),
               "subquad_topk_candidates")
        return ids, sc

    def topk_bruteforce(self, packed, donor, queries, k: int, gap_open: int = 10, gap_extend: int = 1):
        torch = self.torch
        n = int(packed.shape[0])
        donor = self._dev(donor, torch.int32)
        queries = self._dev(queries, torch.int32)
        nq = int(queries.shape[0])
        ids = self._empty((nq, k), torch.int32)
        sc = self._empty((nq, k), torch.int32)
        _check(lib().subquad_topk_bruteforce(self.handle, _ptr(packed), int(packed.shape[1]), n, _ptr(donor),
                                             gap_open, gap_extend, _ptr(queries), nq, k, _ptr(ids), _ptr(sc)),
               "subquad_topk_bruteforce")
        return ids, sc

    # -- gate training ---------------------------------------------------------
    def pair_labels(self, pairs, family, subgroup):
        torch = self.torch
        m = int(pairs.shape[0])
        family = self._dev(family, torch.int32)
        subgroup = self._dev(subgroup, torch.int32)
        label = self._empty((m,), torch.uint8)
        group = self._empty((m,), torch.int32)
        _check(lib().subquad_pair_labels(self.handle, _ptr(pairs), m, _ptr(family), _ptr(subgroup), _ptr(label),
                                         _ptr(group)), "subquad_pair_labels")
        return label, group

    def pair_weights(self, group, num_groups: int):
        torch = self.torch
        m = int(group.shape[0])
        w = self._empty((m,), torch.float32)
        _check(lib().subquad_pair_weights(self.handle, _ptr(group), m, num_groups, _ptr(w)), "subquad_pair_weights")
        return w

    def bce_loss(self, fused, label, weight, want_grad: bool = True, loss=None, grad=None):
        torch = self.torch
        m = int(fused.shape[0])
        loss = self._empty((1,), torch.float32) if loss is None else loss
        if want_grad and grad is None:
            grad = self._empty((m,), torch.float32)
        _check(lib().subquad_bce_loss(self.handle, _ptr(fused), _ptr(label), _ptr(weight), m, _ptr(loss),
                                      _ptr(grad) if want_grad else None), "subquad_bce_loss")
        return (loss, grad) if want_grad else loss

    def pair_index(self, pairs, n: int):
        torch = self.torch
        m = int(pairs.shape[0])
        idx = dict(perm_i=self._empty((max(m, 1),), torch.int32), off_i=self._empty((n + 1,), torch.int32),
                   perm_j=self._empty((max(m, 1),), torch.int32), off_j=self._empty((n + 1,), torch.int32))
        _check(lib().subquad_pair_index(self.handle, _ptr(pairs), m, n, _ptr(idx["perm_i"]), _ptr(idx["off_i"]),
                                        _ptr(idx["perm_j"]), _ptr(idx["off_j"])), "subquad_pair_index")
        return idx

    def fuse_backward(self, pairs, sw, self_sc, packed, emb, params, hidden: int, dL, index=None,
                      grad_params=None, grad_emb=None, want_emb: bool = True):
        torch = self.torch
        m = int(pairs.shape[0])
        n, d = int(emb.shape[0]), int(emb.shape[1])
        grad_params = self._empty((5 * hidden + 1,), torch.float32) if grad_params is None else grad_params
        if want_emb:
            if index is None:
                index = self.pair_index(pairs, n)
            grad_emb = self._empty((n, d), torch.float32) if grad_emb is None else grad_emb
        ix = index or {}
        _check(lib().subquad_fuse_backward(
            self.handle, _ptr(pairs), m, _ptr(sw), _ptr(self_sc), _ptr(packed), int(packed.shape[1]), _ptr(emb), n, d,
            _ptr(params), hidden, _ptr(dL), _ptr(ix.get("perm_i")), _ptr(ix.get("off_i")), _ptr(ix.get("perm_j")),
            _ptr(ix.get("off_j")), _ptr(grad_params), _ptr(grad_emb) if want_emb else None), "subquad_fuse_backward")
        return (grad_params, grad_emb) if want_emb else grad_params

    def fuse_backward_params_noalloc(self, pairs, sw, self_sc, packed, emb, params, hidden: int, dL, out=None):
        """Parameter gradient only, with no device allocation by the library
        (block partials in a static device array; see include/subquad.h)."""
        torch = self.torch
        m = int(pairs.shape[0])
        out = self._empty((5 * hidden + 1,), torch.float32) if out is None else out
        _check(lib().subquad_fuse_backward_params_noalloc(
            self.handle, _ptr(pairs), m, _ptr(sw), _ptr(self_sc), _ptr(packed), int(packed.shape[1]), _ptr(emb),
            int(emb.shape[1]), _ptr(params), hidden, _ptr(dL), _ptr(out)), "subquad_fuse_backward_params_noalloc")
        return out

    def sig_sequence_major(self, sig):
        """int32 [bands, n, rows] signatures of sign() -> int32 [n, bands*rows]."""
        bands, n, rows = (int(x) for x in sig.shape)
        out = self._empty((n, bands * rows), self.torch.int32)
        _check(lib().subquad_sig_sequence_major(self.handle, _ptr(sig), n, bands, rows, _ptr(out)),
               "subquad_sig_sequence_major")
        return out

    def fuse_forward_mc(self, pairs, sw, self_sc, packed, emb, sig_seq, params, hidden: int, channels: int,
                        want_weights: bool = False, out=None):
        """M-channel fusion (channels 2 or 3); sig_seq is the int32 [n, H]
        sequence-major signature (sig_sequence_major; unused for 2 channels)."""
        torch = self.torch
        m = int(pairs.shape[0])
        emb = self._dev(emb, torch.float32)
        params = self._dev(params, torch.float32)
        out = self._empty((m,), torch.float32) if out is None else out
        w = self._empty((m, channels), torch.float32) if want_weights else None
        H = int(sig_seq.shape[1]) if sig_seq is not None else 0
        _check(lib().subquad_fuse_forward_mc(self.handle, _ptr(pairs), m, _ptr(sw), _ptr(self_sc), _ptr(packed),
                                             int(packed.shape[1]), _ptr(emb), int(emb.shape[1]), _ptr(sig_seq), H,
                                             _ptr(params), hidden, channels, _ptr(out), _ptr(w)),
               "subquad_fuse_forward_mc")
        return (out, w) if want_weights else out

    def fuse_backward_mc(self, pairs, sw, self_sc, packed, emb, sig_seq, params, hidden: int, channels: int, dL,
                         index=None, grad_params=None, grad_emb=None, want_emb: bool = True):
        torch = self.torch
        m = int(pairs.shape[0])
        n, d = int(emb.shape[0]), int(emb.shape[1])
        grad_params = torch.empty_like(params) if grad_params is None else grad_params
        if want_emb:
            if index is None:
                index = self.pair_index(pairs, n)
            grad_emb = self._empty((n, d), torch.float32) if grad_emb is None else grad_emb
        ix = index or {}
        H = int(sig_seq.shape[1]) if sig_seq is not None else 0
        _check(lib().subquad_fuse_backward_mc(
            self.handle, _ptr(pairs), m, _ptr(sw), _ptr(self_sc), _ptr(packed), int(packed.shape[1]), _ptr(emb), n, d,
            _ptr(sig_seq), H, _ptr(params), hidden, channels, _ptr(dL), _ptr(ix.get("perm_i")),
            _ptr(ix.get("off_i")), _ptr(ix.get("perm_j")), _ptr(ix.get("off_j")), _ptr(grad_params),
            _ptr(grad_emb) if want_emb else None), "subquad_fuse_backward_mc")
        return (grad_params, grad_emb) if want_emb else grad_params

    # -- graph construction and RMT thresholding ---------------------------
    def graph_components(self, pairs, weights, n: int, tau: float, want_sizes: bool = False):
        torch = self.torch
        m = int(pairs.shape[0])
        labels = self._empty((n,), torch.int32)
        sizes = self._empty((n,), torch.int32) if want_sizes else None
        _check(lib().subquad_graph_components(self.handle, _ptr(pairs), _ptr(weights), m, n, float(tau), _ptr(labels),
                                              _ptr(sizes)), "subquad_graph_components")
        return (labels, sizes) if want_sizes else labels

    def rmt_threshold(self, pairs, weights, n: int, taus, s_max: int = 64, r_mid: float | None = None) -> dict:
        """The threshold scan; returns {tau_star, r_mean, num_ratios,
        num_levels, max_comp} (host lists, one entry per threshold)."""
        import math

        if r_mid is None:
            r_mid = 0.5 * ((2.0 * math.log(2.0) - 1.0) + (4.0 - 2.0 * math.sqrt(3.0)))
        T = len(taus)
        c_taus = (_c.c_double * T)(*[float(t) for t in taus])
        r_mean = (_c.c_double * T)()
        nr = (_I64 * T)()
        nl = (_I64 * T)()
        mc = (_c.c_int32 * T)()
        ts = _c.c_double(0.0)
        _check(lib().subquad_rmt_threshold(self.handle, _ptr(pairs), _ptr(weights), int(pairs.shape[0]), n,
                                           _c.cast(c_taus, _P), T, s_max, r_mid, _c.byref(ts), _c.cast(r_mean, _P),
                                           _c.cast(nr, _P), _c.cast(nl, _P), _c.cast(mc, _P)), "subquad_rmt_threshold")
        return {"tau_star": ts.value, "r_mean": list(r_mean), "num_ratios": list(nr), "num_levels": list(nl),
                "max_comp": list(mc)}

    def graph_prune(self, pairs, weights, tau: float):
        """-> (pairs int32 [k, 2], weights float [k]) with weights >= tau."""
        torch = self.torch
        m = int(pairs.shape[0])
        po = self._empty((max(m, 1), 2), torch.int32)
        wo = self._empty((max(m, 1),), torch.float32)
        cnt = self._empty((1,), torch.int64)
        _check(lib().subquad_graph_prune(self.handle, _ptr(pairs), _ptr(weights), m, float(tau), _ptr(po), _ptr(wo),
                                         _ptr(cnt)), "subquad_graph_prune")
        k = int(cnt.item())
        return po[:k], wo[:k]

    def cluster_js(self, labels, donor, num_donors: int):
        """-> float64 [num_donors, num_donors] sqrt-JS distances of the donors'
        cluster-mass vectors."""
        torch = self.torch
        donor = self._dev(donor, torch.int32)
        out = self._empty((num_donors, num_donors), torch.float64)
        _check(lib().subquad_cluster_js(self.handle, _ptr(labels), _ptr(donor), int(labels.shape[0]), num_donors,
                                        _ptr(out)), "subquad_cluster_js")
        return out

    def adam_step(self, param, grad, m1, m2, t: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8):
        _check(lib().subquad_adam_step(self.handle, _ptr(param), _ptr(grad), _ptr(m1), _ptr(m2), int(param.numel()),
                                       t, lr, beta1, beta2, eps), "subquad_adam_step")


# module-level names matching the C entry points, taking a Context first
def subquad_pack(ctx: Context, *a, **k):
    return ctx.pack(*a, **k)


def subquad_sign(ctx: Context, *a, **k):
    return ctx.sign(*a, **k)


def subquad_band_candidates(ctx: Context, *a, **k):
    return ctx.band_candidates(*a, **k)


def subquad_align_score(ctx: Context, *a, **k):
    return ctx.align_score(*a, **k)


def subquad_self_scores(ctx: Context, *a, **k):
    return ctx.self_scores(*a, **k)


def subquad_align_score_binned(ctx: Context, *a, **k):
    return ctx.align_score(*a, binned=True, **k)


def subquad_self_scores_binned(ctx: Context, *a, **k):
    return ctx.self_scores(*a, binned=True, **k)


def subquad_fuse_forward(ctx: Context, *a, **k):
    return ctx.fuse_forward(*a, **k)


def subquad_pair_labels(ctx: Context, *a, **k):
    return ctx.pair_labels(*a, **k)


def subquad_pair_weights(ctx: Context, *a, **k):
    return ctx.pair_weights(*a, **k)


def subquad_bce_loss(ctx: Context, *a, **k):
    return ctx.bce_loss(*a, **k)


def subquad_pair_index(ctx: Context, *a, **k):
    return ctx.pair_index(*a, **k)


def subquad_fuse_backward(ctx: Context, *a, **k):
    return ctx.fuse_backward(*a, **k)


def subquad_fuse_backward_params_noalloc(ctx: Context, *a, **k):
    return ctx.fuse_backward_params_noalloc(*a, **k)


def subquad_fuse_forward_mc(ctx: Context, *a, **k):
    return ctx.fuse_forward_mc(*a, **k)


def subquad_fuse_backward_mc(ctx: Context, *a, **k):
    return ctx.fuse_backward_mc(*a, **k)


def subquad_sig_sequence_major(ctx: Context, *a, **k):
    return ctx.sig_sequence_major(*a, **k)


def subquad_edit_distance(ctx: Context, *a, **k):
    return ctx.edit_distance(*a, **k)


def subquad_edit_distance_async(ctx: Context, *a, **k):
    return ctx.edit_distance_async(*a, **k)


def subquad_graph_components(ctx: Context, *a, **k):
    return ctx.graph_components(*a, **k)


def subquad_rmt_threshold(ctx: Context, *a, **k):
    return ctx.rmt_threshold(*a, **k)


def subquad_graph_prune(ctx: Context, *a, **k):
    return ctx.graph_prune(*a, **k)


def subquad_cluster_js(ctx: Context, *a, **k):
    return ctx.cluster_js(*a, **k)


def subquad_adam_step(ctx: Context, *a, **k):
    return ctx.adam_step(*a, **k)


def subquad_topk_candidates(ctx: Context, *a, **k):
    return ctx.topk_candidates(*a, **k)


def subquad_topk_bruteforce(ctx: Context, *a, **k):
    return ctx.topk_bruteforce(*a, **k)


def subquad_band_candidates_async(ctx: Context, *a, **k):
    return ctx.band_candidates_async(*a, **k)


def subquad_align_score_binned_async(ctx: Context, *a, **k):
    return ctx.align_score_binned_async(*a, **k)


def subquad_fuse_forward_async(ctx: Context, *a, **k):
    return ctx.fuse_forward_async(*a, **k)
