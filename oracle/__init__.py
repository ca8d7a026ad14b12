"""Oracle for the SubQuad affinity stage: numpy-facing wrappers around the plain
single-threaded C reference in ``subquad_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the library path must not.  It shares
no code with the CUDA sources (the seeded input generators are the only common
module, and they hold none of the method's arithmetic).

Every floating-point result is FP64.  Each function names the paper passage it
restates; the reading of each silent or ambiguous point is written beside it in
the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "subquad_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U32P = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
U8P = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
F32P = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with plain -O2 (no fast-math) into liboracle.so."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-Wall", "-fPIC", "-pthread",
                                   "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    c = ctypes
    lib.oracle_blosum62.argtypes = [I32P]
    lib.oracle_blosum62.restype = None
    lib.oracle_kmer_code.argtypes = [U8P, c.c_int]
    lib.oracle_kmer_code.restype = c.c_uint64
    lib.oracle_sign.argtypes = [U8P, c.c_int, U8P, c.c_int64, c.c_int, c.c_int, U32P, U32P, U32P]
    lib.oracle_sign.restype = None
    lib.oracle_candidates.argtypes = [U32P, c.c_int64, c.c_int, c.c_int, c.c_int, c.c_int, U32P, c.c_int64]
    lib.oracle_candidates.restype = c.c_int64
    lib.oracle_candidates_mt.argtypes = [U32P, c.c_int64, c.c_int, c.c_int, c.c_int, c.c_int, U32P, c.c_int64, c.c_int]
    lib.oracle_candidates_mt.restype = c.c_int64
    lib.oracle_sw.argtypes = [U8P, c.c_int, U8P, c.c_int, I32P, c.c_int, c.c_int]
    lib.oracle_sw.restype = c.c_int32
    lib.oracle_sw_pairs.argtypes = [U8P, c.c_int, U8P, U32P, c.c_int64, I32P, c.c_int, c.c_int, I32P]
    lib.oracle_sw_pairs.restype = None
    opt_f64 = c.c_void_p
    lib.oracle_fuse_forward.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, F32P, c.c_int,
                                        F64P, opt_f64, opt_f64, opt_f64]
    lib.oracle_fuse_forward.restype = c.c_int
    lib.oracle_fuse_backward.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, F32P, c.c_int,
                                         F64P, F64P, opt_f64]
    lib.oracle_fuse_backward.restype = c.c_int
    lib.oracle_fuse_backward_scale.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, F32P, c.c_int,
                                               F64P, F64P, opt_f64]
    lib.oracle_fuse_backward_scale.restype = c.c_int
    lib.oracle_fuse_forward_mc.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, opt_f64, c.c_int, F32P,
                                           c.c_int, c.c_int, F64P, opt_f64, opt_f64]
    lib.oracle_fuse_forward_mc.restype = c.c_int
    lib.oracle_fuse_backward_mc.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, opt_f64, c.c_int,
                                            F32P, c.c_int, c.c_int, F64P, F64P, opt_f64]
    lib.oracle_fuse_backward_mc.restype = c.c_int
    lib.oracle_fuse_backward_mc_scale.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, opt_f64, c.c_int,
                                                  F32P, c.c_int, c.c_int, F64P, F64P, opt_f64]
    lib.oracle_fuse_backward_mc_scale.restype = c.c_int
    lib.oracle_edit.argtypes = [U8P, c.c_int, U8P, c.c_int, c.c_int, U8P]
    lib.oracle_edit.restype = c.c_int32
    lib.oracle_edit_pairs.argtypes = [U8P, c.c_int, U8P, U32P, c.c_int64, c.c_int, U8P, I32P]
    lib.oracle_edit_pairs.restype = None
    lib.oracle_default_edit_costs.argtypes = [U8P]
    lib.oracle_default_edit_costs.restype = None
    lib.oracle_pair_labels.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, I32P]
    lib.oracle_pair_labels.restype = None
    lib.oracle_pair_weights.argtypes = [I32P, c.c_int64, c.c_int, F64P]
    lib.oracle_pair_weights.restype = c.c_int
    lib.oracle_bce_loss.argtypes = [F64P, U8P, F64P, c.c_int64, opt_f64]
    lib.oracle_bce_loss.restype = c.c_double
    lib.oracle_adam.argtypes = [F64P, F64P, F64P, F64P, c.c_int64, c.c_int, c.c_double, c.c_double,
                                c.c_double, c.c_double]
    lib.oracle_adam.restype = None
    lib.oracle_topk.argtypes = [U32P, I32P, c.c_int64, I32P, U32P, c.c_int64, c.c_int, U32P, I32P]
    lib.oracle_topk.restype = c.c_int
    lib.oracle_sign_mt.argtypes = [U8P, c.c_int, U8P, c.c_int64, c.c_int, c.c_int, U32P, U32P, U32P, c.c_int]
    lib.oracle_sign_mt.restype = c.c_int
    lib.oracle_sw_pairs_mt.argtypes = [U8P, c.c_int, U8P, U32P, c.c_int64, I32P, c.c_int, c.c_int, I32P, c.c_int]
    lib.oracle_sw_pairs_mt.restype = c.c_int
    lib.oracle_fuse_forward_mt.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, F32P, c.c_int, F64P,
                                           c.c_int]
    lib.oracle_fuse_forward_mt.restype = c.c_int
    lib.oracle_fuse_backward_params_mt.argtypes = [U32P, c.c_int64, I32P, I32P, U8P, F32P, c.c_int, F32P, c.c_int,
                                                   F64P, F64P, c.c_int]
    lib.oracle_fuse_backward_params_mt.restype = c.c_int
    _lib = lib
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _pairs(pairs):
    p = _c(pairs, np.uint32)
    if p.ndim != 2 or (p.size and p.shape[1] != 2):
        p = p.reshape(-1, 2)
    return p


# --------------------------------------------------------------------------
# BLOSUM62 and k-mers
# --------------------------------------------------------------------------

def blosum62() -> np.ndarray:
    """int32 [20, 20] in code order ACDEFGHIKLMNPQRSTVWY."""
    out = np.zeros(400, dtype=np.int32)
    _load().oracle_blosum62(out)
    return out.reshape(20, 20)


def kmer_code(codes_row, k: int) -> int:
    return int(_load().oracle_kmer_code(_c(codes_row[:k], np.uint8), k))


# --------------------------------------------------------------------------
# Algorithm 1, preprocessing: MinHash sketches and the candidate list
# --------------------------------------------------------------------------

def sign(codes, lens, k: int, a, b) -> np.ndarray:
    """MinHash signature, uint32 [n, H] (sequence-major)."""
    codes = _c(codes, np.uint8)
    lens = _c(lens, np.uint8)
    a = _c(a, np.uint32)
    b = _c(b, np.uint32)
    n, H = lens.shape[0], a.shape[0]
    if n and int(lens.min()) < k:
        raise ValueError("every sequence needs at least one k-mer")
    sig = np.zeros((n, H), dtype=np.uint32)
    _load().oracle_sign(codes, codes.shape[1], lens, n, k, H, a, b, sig)
    return sig


def candidates(sig, bands: int, rows: int, cap: int = 0) -> np.ndarray:
    """Candidate set C as a lexicographically sorted uint32 [|C|, 2] array."""
    sig = _c(sig, np.uint32)
    n, H = sig.shape
    lib = _load()
    capacity = max(1024, 4 * n)
    while True:
        out = np.zeros((capacity, 2), dtype=np.uint32)
        cnt = lib.oracle_candidates(sig, n, H, bands, rows, cap, out, capacity)
        if cnt < 0:
            raise MemoryError("oracle_candidates failed")
        if cnt <= capacity:
            return out[:cnt].copy()
        capacity = int(cnt)


def candidates_mt(sig, bands: int, rows: int, cap: int, threads: int) -> np.ndarray:
    """candidates() with the bands split over `threads` host threads (the
    same per-band routine and the same sort and deduplication: identical
    output)."""
    sig = _c(sig, np.uint32)
    n, H = sig.shape
    lib = _load()
    capacity = max(1024, 4 * n)
    while True:
        out = np.zeros((capacity, 2), dtype=np.uint32)
        cnt = lib.oracle_candidates_mt(sig, n, H, bands, rows, cap, out, capacity, int(threads))
        if cnt < 0:
            raise MemoryError("oracle_candidates_mt failed")
        if cnt <= capacity:
            return out[:cnt].copy()
        capacity = int(cnt)


# --------------------------------------------------------------------------
# Affinity computation: alignment channel
# --------------------------------------------------------------------------

def sw(a_codes, b_codes, gap_open: int = 10, gap_extend: int = 1, matrix=None) -> int:
    """Affine-gap local alignment score of two code sequences."""
    M = blosum62() if matrix is None else _c(matrix, np.int32)
    a = _c(a_codes, np.uint8)
    b = _c(b_codes, np.uint8)
    return int(_load().oracle_sw(a, a.shape[0], b, b.shape[0], _c(M.reshape(-1), np.int32), gap_open, gap_extend))


def sw_pairs(codes, lens, pairs, gap_open: int = 10, gap_extend: int = 1, matrix=None) -> np.ndarray:
    codes = _c(codes, np.uint8)
    lens = _c(lens, np.uint8)
    p = _pairs(pairs)
    M = blosum62() if matrix is None else _c(matrix, np.int32)
    out = np.zeros(p.shape[0], dtype=np.int32)
    _load().oracle_sw_pairs(codes, codes.shape[1], lens, p, p.shape[0], _c(M.reshape(-1), np.int32),
                            gap_open, gap_extend, out)
    return out


def self_scores(codes, lens, gap_open: int = 10, gap_extend: int = 1, matrix=None) -> np.ndarray:
    n = _c(lens, np.uint8).shape[0]
    idx = np.arange(n, dtype=np.uint32)
    return sw_pairs(codes, lens, np.stack([idx, idx], axis=1), gap_open, gap_extend, matrix)


# --------------------------------------------------------------------------
# Edit distance (the GPU appendix's edit-distance kernel)
# --------------------------------------------------------------------------

def default_edit_costs() -> np.ndarray:
    """uint8 [20, 20]: 0 on the diagonal, 1 where BLOSUM62 > 0, else 2."""
    out = np.zeros(400, dtype=np.uint8)
    _load().oracle_default_edit_costs(out)
    return out.reshape(20, 20)


def edit(a_codes, b_codes, indel: int = 2, sub=None) -> int:
    S = default_edit_costs() if sub is None else _c(sub, np.uint8)
    a = _c(a_codes, np.uint8)
    b = _c(b_codes, np.uint8)
    return int(_load().oracle_edit(a, a.shape[0], b, b.shape[0], indel, _c(S.reshape(-1), np.uint8)))


def edit_pairs(codes, lens, pairs, indel: int = 2, sub=None) -> np.ndarray:
    codes = _c(codes, np.uint8)
    lens = _c(lens, np.uint8)
    p = _pairs(pairs)
    S = default_edit_costs() if sub is None else _c(sub, np.uint8)
    out = np.zeros(p.shape[0], dtype=np.int32)
    _load().oracle_edit_pairs(codes, codes.shape[1], lens, p, p.shape[0], indel, _c(S.reshape(-1), np.uint8), out)
    return out


# --------------------------------------------------------------------------
# Affinity computation: per-pair gated fusion (Eq. alpha, Eq. wm, Eq. afused)
# --------------------------------------------------------------------------

def fuse_forward(pairs, sw_scores, self_sc, lens, emb, params, hidden: int):
    """Returns dict of FP64 arrays: fused, alpha, s (normalised SW), c (cosine)."""
    p = _pairs(pairs)
    m = p.shape[0]
    emb = _c(emb, np.float32)
    out = {k: np.zeros(m, dtype=np.float64) for k in ("fused", "alpha", "s", "c")}
    rc = _load().oracle_fuse_forward(p, m, _c(sw_scores, np.int32), _c(self_sc, np.int32), _c(lens, np.uint8),
                                     emb, emb.shape[1], _c(params, np.float32), hidden, out["fused"],
                                     _ptr(out["alpha"]), _ptr(out["s"]), _ptr(out["c"]))
    if rc != 0:
        raise MemoryError("oracle_fuse_forward failed")
    return out


def fuse_backward(pairs, sw_scores, self_sc, lens, emb, params, hidden: int, dL_dfused, with_emb: bool = True):
    """Returns (grad_params FP64 [P], grad_emb FP64 [n, d] or None)."""
    p = _pairs(pairs)
    emb = _c(emb, np.float32)
    gp = np.zeros(5 * hidden + 1, dtype=np.float64)
    ge = np.zeros(emb.shape, dtype=np.float64) if with_emb else None
    rc = _load().oracle_fuse_backward(p, p.shape[0], _c(sw_scores, np.int32), _c(self_sc, np.int32),
                                      _c(lens, np.uint8), emb, emb.shape[1], _c(params, np.float32), hidden,
                                      _c(dL_dfused, np.float64), gp, _ptr(ge))
    if rc != 0:
        raise MemoryError("oracle_fuse_backward failed")
    return gp, ge


def fuse_backward_scale(pairs, sw_scores, self_sc, lens, emb, params, hidden: int, dL_dfused,
                        with_emb: bool = True):
    """Rounding scale of the adjoint: (FP64 [P], FP64 [n, d] or None), the
    summed magnitude of every pair's contribution to each gradient entry, with
    cancelling factors taken as magnitude + 1.  A float32 gradient lies within
    a fixed multiple of unit roundoff times this scale of the exact one."""
    p = _pairs(pairs)
    emb = _c(emb, np.float32)
    sc = np.zeros(5 * hidden + 1, dtype=np.float64)
    se = np.zeros(emb.shape, dtype=np.float64) if with_emb else None
    rc = _load().oracle_fuse_backward_scale(p, p.shape[0], _c(sw_scores, np.int32), _c(self_sc, np.int32),
                                            _c(lens, np.uint8), emb, emb.shape[1], _c(params, np.float32), hidden,
                                            _c(dL_dfused, np.float64), sc, _ptr(se))
    if rc != 0:
        raise MemoryError("oracle_fuse_backward_scale failed")
    return sc, se


def mc_param_count(hidden: int, channels: int) -> int:
    """Parameters of the M-channel gate: W1 [h][M+1], b1 [h], W2 [M-1][h], b2 [M-1]."""
    return (channels + 1) * hidden + hidden + (channels - 1) * hidden + (channels - 1)


def fuse_forward_mc(pairs, sw_scores, self_sc, lens, emb, sig, params, hidden: int, channels: int):
    """M-channel fusion (M = 2 or 3).  sig: uint32 [n, H] sequence-major (used
    for M = 3).  Returns dict of FP64 arrays: fused [m], weights [m, M],
    jaccard [m] (0 for M = 2)."""
    p = _pairs(pairs)
    m = p.shape[0]
    emb = _c(emb, np.float32)
    sig_c = None if sig is None else _c(sig, np.uint32)
    H = 0 if sig_c is None else sig_c.shape[1]
    out = {"fused": np.zeros(m), "weights": np.zeros((m, channels)), "jaccard": np.zeros(m)}
    rc = _load().oracle_fuse_forward_mc(p, m, _c(sw_scores, np.int32), _c(self_sc, np.int32), _c(lens, np.uint8),
                                        emb, emb.shape[1], _ptr(sig_c), H, _c(params, np.float32), hidden, channels,
                                        out["fused"], _ptr(out["weights"]), _ptr(out["jaccard"]))
    if rc != 0:
        raise ValueError("oracle_fuse_forward_mc failed")
    return out


def fuse_backward_mc(pairs, sw_scores, self_sc, lens, emb, sig, params, hidden: int, channels: int, dL_dfused,
                     with_emb: bool = True):
    """Returns (grad_params FP64 [P], grad_emb FP64 [n, d] or None)."""
    p = _pairs(pairs)
    emb = _c(emb, np.float32)
    sig_c = None if sig is None else _c(sig, np.uint32)
    H = 0 if sig_c is None else sig_c.shape[1]
    gp = np.zeros(mc_param_count(hidden, channels), dtype=np.float64)
    ge = np.zeros(emb.shape, dtype=np.float64) if with_emb else None
    rc = _load().oracle_fuse_backward_mc(p, p.shape[0], _c(sw_scores, np.int32), _c(self_sc, np.int32),
                                         _c(lens, np.uint8), emb, emb.shape[1], _ptr(sig_c), H,
                                         _c(params, np.float32), hidden, channels, _c(dL_dfused, np.float64), gp,
                                         _ptr(ge))
    if rc != 0:
        raise ValueError("oracle_fuse_backward_mc failed")
    return gp, ge


def fuse_backward_mc_scale(pairs, sw_scores, self_sc, lens, emb, sig, params, hidden: int, channels: int,
                           dL_dfused, with_emb: bool = True):
    """Rounding scale of the M-channel adjoint: (FP64 [P], FP64 [n, d] or None)."""
    p = _pairs(pairs)
    emb = _c(emb, np.float32)
    sig_c = None if sig is None else _c(sig, np.uint32)
    H = 0 if sig_c is None else sig_c.shape[1]
    sc = np.zeros(mc_param_count(hidden, channels), dtype=np.float64)
    se = np.zeros(emb.shape, dtype=np.float64) if with_emb else None
    rc = _load().oracle_fuse_backward_mc_scale(p, p.shape[0], _c(sw_scores, np.int32), _c(self_sc, np.int32),
                                               _c(lens, np.uint8), emb, emb.shape[1], _ptr(sig_c), H,
                                               _c(params, np.float32), hidden, channels, _c(dL_dfused, np.float64),
                                               sc, _ptr(se))
    if rc != 0:
        raise ValueError("oracle_fuse_backward_mc_scale failed")
    return sc, se


# --------------------------------------------------------------------------
# Gate training objective and optimiser
# --------------------------------------------------------------------------

def pair_labels(pairs, family, subgroup):
    p = _pairs(pairs)
    m = p.shape[0]
    y = np.zeros(m, dtype=np.uint8)
    g = np.zeros(m, dtype=np.int32)
    _load().oracle_pair_labels(p, m, _c(family, np.int32), _c(subgroup, np.int32), y, g)
    return y, g


def pair_weights(group, num_groups: int) -> np.ndarray:
    g = _c(group, np.int32)
    w = np.zeros(g.shape[0], dtype=np.float64)
    if _load().oracle_pair_weights(g, g.shape[0], num_groups, w) != 0:
        raise ValueError("group id out of range")
    return w


def bce_loss(fused, label, weight):
    """Returns (loss, dL/dfused) in FP64."""
    f = _c(fused, np.float64)
    d = np.zeros(f.shape[0], dtype=np.float64)
    loss = _load().oracle_bce_loss(f, _c(label, np.uint8), _c(weight, np.float64), f.shape[0], _ptr(d))
    return float(loss), d


def adam_step(param, grad, m1, m2, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """In-place Adam step on FP64 arrays."""
    for a in (param, grad, m1, m2):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("adam_step works in place on contiguous float64 arrays")
    _load().oracle_adam(param, grad, m1, m2, param.shape[0], t, lr, beta1, beta2, eps)


# --------------------------------------------------------------------------
# Cross-donor retrieval
# --------------------------------------------------------------------------

def topk(pairs, scores, donor, queries, k: int):
    p = _pairs(pairs)
    q = _c(queries, np.uint32)
    ids = np.zeros((q.shape[0], k), dtype=np.uint32)
    sc = np.zeros((q.shape[0], k), dtype=np.int32)
    if _load().oracle_topk(p, _c(scores, np.int32), p.shape[0], _c(donor, np.int32), q, q.shape[0], k, ids, sc):
        raise MemoryError("oracle_topk failed")
    return ids, sc


# --------------------------------------------------------------------------
# All host cores: the same routines over contiguous index ranges in threads
# (identical results; the CPU baseline's N-core figure)
# --------------------------------------------------------------------------

def host_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def sign_mt(codes, lens, k: int, a, b, threads: int) -> np.ndarray:
    codes = _c(codes, np.uint8)
    lens = _c(lens, np.uint8)
    a = _c(a, np.uint32)
    b = _c(b, np.uint32)
    n, H = lens.shape[0], a.shape[0]
    if n and int(lens.min()) < k:
        raise ValueError("every sequence needs at least one k-mer")
    sig = np.zeros((n, H), dtype=np.uint32)
    if _load().oracle_sign_mt(codes, codes.shape[1], lens, n, k, H, a, b, sig, threads):
        raise MemoryError("oracle_sign_mt failed")
    return sig


def sw_pairs_mt(codes, lens, pairs, threads: int, gap_open: int = 10, gap_extend: int = 1, matrix=None):
    codes = _c(codes, np.uint8)
    lens = _c(lens, np.uint8)
    p = _pairs(pairs)
    M = blosum62() if matrix is None else _c(matrix, np.int32)
    out = np.zeros(p.shape[0], dtype=np.int32)
    if _load().oracle_sw_pairs_mt(codes, codes.shape[1], lens, p, p.shape[0], _c(M.reshape(-1), np.int32), gap_open,
                                  gap_extend, out, threads):
        raise MemoryError("oracle_sw_pairs_mt failed")
    return out


def fuse_forward_mt(pairs, sw_scores, self_sc, lens, emb, params, hidden: int, threads: int) -> np.ndarray:
    p = _pairs(pairs)
    emb = _c(emb, np.float32)
    out = np.zeros(p.shape[0], dtype=np.float64)
    if _load().oracle_fuse_forward_mt(p, p.shape[0], _c(sw_scores, np.int32), _c(self_sc, np.int32),
                                      _c(lens, np.uint8), emb, emb.shape[1], _c(params, np.float32), hidden, out,
                                      threads):
        raise MemoryError("oracle_fuse_forward_mt failed")
    return out


def fuse_backward_params_mt(pairs, sw_scores, self_sc, lens, emb, params, hidden: int, dL_dfused, threads: int):
    """Parameter gradient of the fusion adjoint (FP64 [5 h + 1]) over threads."""
    p = _pairs(pairs)
    emb = _c(emb, np.float32)
    gp = np.zeros(5 * hidden + 1, dtype=np.float64)
    if _load().oracle_fuse_backward_params_mt(p, p.shape[0], _c(sw_scores, np.int32), _c(self_sc, np.int32),
                                              _c(lens, np.uint8), emb, emb.shape[1], _c(params, np.float32), hidden,
                                              _c(dL_dfused, np.float64), gp, threads):
        raise MemoryError("oracle_fuse_backward_params_mt failed")
    return gp
