"""Gate training on the GPU: the fusion as a torch.autograd.Function over the
library's forward and adjoint kernels, and a full-batch trainer (weighted BCE
on family-match labels, inverse-subgroup weights, Adam) whose every step runs
in the library's kernels.
"""
from __future__ import annotations

import torch


class FuseFunction(torch.autograd.Function):
    """fused = F(emb, params) for a fixed pair list.  The forward stores only
    its inputs; the backward recomputes every pair's hidden activations in the
    adjoint kernel."""

    @staticmethod
    def forward(ctx_, emb, params, sub, pairs, sw, self_sc, packed, hidden, index):
        fused = sub.fuse_forward(pairs, sw, self_sc, packed, emb.detach(), params.detach(), hidden)
        ctx_.save_for_backward(emb, params)
        ctx_.sub, ctx_.pairs, ctx_.sw, ctx_.self_sc, ctx_.packed = sub, pairs, sw, self_sc, packed
        ctx_.hidden, ctx_.index = hidden, index
        return fused

    @staticmethod
    def backward(ctx_, grad_fused):
        emb, params = ctx_.saved_tensors
        want_emb = bool(ctx_.needs_input_grad[0])
        out = ctx_.sub.fuse_backward(ctx_.pairs, ctx_.sw, ctx_.self_sc, ctx_.packed, emb.detach(), params.detach(),
                                     ctx_.hidden, grad_fused.contiguous().float(), index=ctx_.index,
                                     want_emb=want_emb)
        gp, ge = out if want_emb else (out, None)
        return ge, gp, None, None, None, None, None, None, None


def fuse(sub, pairs, sw, self_sc, packed, emb, params, hidden: int, index=None):
    """Differentiable fused score (autograd over the library's kernels)."""
    if index is None and emb.requires_grad:
        index = sub.pair_index(pairs, int(emb.shape[0]))
    return FuseFunction.apply(emb, params, sub, pairs, sw, self_sc, packed, hidden, index)


class GateTrainer:
    """Full-batch training of the gate (and optionally the embeddings) on a
    fixed pair list; all state lives on the device."""

    def __init__(self, sub, pairs, sw, self_sc, packed, emb, params, hidden: int, labels, weights, lr: float = 1e-3,
                 train_emb: bool = True):
        self.sub, self.pairs, self.sw, self.self_sc, self.packed = sub, pairs, sw, self_sc, packed
        self.emb = emb.detach().clone().contiguous()
        self.params = params.detach().clone().contiguous()
        self.hidden, self.labels, self.weights, self.lr, self.train_emb = hidden, labels, weights, lr, train_emb
        self.index = sub.pair_index(pairs, int(emb.shape[0])) if train_emb else None
        z = torch.zeros_like
        self.m1p, self.m2p = z(self.params), z(self.params)
        self.m1e, self.m2e = (z(self.emb), z(self.emb)) if train_emb else (None, None)
        m = int(pairs.shape[0])
        dev = self.params.device
        self.fused = torch.empty((m,), dtype=torch.float32, device=dev)
        self.loss = torch.empty((1,), dtype=torch.float32, device=dev)
        self.dL = torch.empty((m,), dtype=torch.float32, device=dev)
        self.gp = torch.empty_like(self.params)
        self.ge = torch.empty_like(self.emb) if train_emb else None
        self.t = 0

    def step(self):
        s = self.sub
        s.fuse_forward(self.pairs, self.sw, self.self_sc, self.packed, self.emb, self.params, self.hidden,
                       out=self.fused)
        s.bce_loss(self.fused, self.labels, self.weights, loss=self.loss, grad=self.dL)
        s.fuse_backward(self.pairs, self.sw, self.self_sc, self.packed, self.emb, self.params, self.hidden, self.dL,
                        index=self.index, grad_params=self.gp, grad_emb=self.ge, want_emb=self.train_emb)
        self.t += 1
        s.adam_step(self.params, self.gp, self.m1p, self.m2p, self.t, self.lr)
        if self.train_emb:
            s.adam_step(self.emb, self.ge, self.m1e, self.m2e, self.t, self.lr)
        return self.loss

    def state(self) -> dict:
        st = {"t": self.t, "params": self.params, "m1p": self.m1p, "m2p": self.m2p}
        if self.train_emb:
            st.update(emb=self.emb, m1e=self.m1e, m2e=self.m2e)
        return st

    def checkpoint(self) -> dict:
        """Host copies of everything the next step reads (step count, gate
        parameters, embeddings, Adam moments)."""
        return {k: (v.detach().cpu().clone() if torch.is_tensor(v) else v) for k, v in self.state().items()}

    def restore(self, ckpt: dict) -> None:
        """Continue from a checkpoint: the steps after it reproduce those of
        the uninterrupted run bit for bit (every kernel is deterministic)."""
        st = self.state()
        if set(ckpt) != set(st):
            raise ValueError("checkpoint does not match this trainer (embedding training on/off)")
        for k, v in st.items():
            if torch.is_tensor(v):
                if tuple(ckpt[k].shape) != tuple(v.shape):
                    raise ValueError(f"checkpoint tensor {k} has shape {tuple(ckpt[k].shape)}, expected {tuple(v.shape)}")
                v.copy_(ckpt[k].to(v.device))
        self.t = int(ckpt["t"])

    def save(self, path: str) -> None:
        write_checkpoint(path, self.checkpoint())

    def load(self, path: str) -> None:
        self.restore(read_checkpoint(path))


# Checkpoint file: magic, format version, step count, tensor count; per tensor
# its name, dtype code and shape; the raw little-endian payloads; and a SHA-256
# of everything before it, checked on reading.
_MAGIC = b"SQGATE01"
_DTYPES = {torch.float32: 0, torch.int32: 1}
_CODES = {v: k for k, v in _DTYPES.items()}


def write_checkpoint(path: str, ckpt: dict) -> None:
    import hashlib
    import struct

    names = sorted(k for k, v in ckpt.items() if torch.is_tensor(v))
    head = bytearray(_MAGIC)
    head += struct.pack("<qq", int(ckpt["t"]), len(names))
    body = bytearray()
    for k in names:
        v = ckpt[k].detach().cpu().contiguous()
        if v.dtype not in _DTYPES:
            raise ValueError(f"checkpoint tensor {k}: unsupported dtype {v.dtype}")
        nb = k.encode()
        head += struct.pack("<H", len(nb)) + nb + struct.pack("<BB", _DTYPES[v.dtype], v.dim())
        head += struct.pack(f"<{v.dim()}q", *v.shape)
        body += v.numpy().tobytes()
    data = bytes(head + body)
    with open(path, "wb") as fh:
        fh.write(data + hashlib.sha256(data).digest())


def read_checkpoint(path: str) -> dict:
    import hashlib
    import struct

    import numpy as np

    with open(path, "rb") as fh:
        raw = fh.read()
    if len(raw) < len(_MAGIC) + 16 + 32 or raw[:len(_MAGIC)] != _MAGIC:
        raise ValueError("not a gate checkpoint")
    data, digest = raw[:-32], raw[-32:]
    if hashlib.sha256(data).digest() != digest:
        raise ValueError("gate checkpoint checksum mismatch")
    off = len(_MAGIC)
    t, count = struct.unpack_from("<qq", data, off)
    off += 16
    specs = []
    for _ in range(count):
        (ln,) = struct.unpack_from("<H", data, off)
        off += 2
        name = data[off:off + ln].decode()
        off += ln
        code, dim = struct.unpack_from("<BB", data, off)
        off += 2
        shape = struct.unpack_from(f"<{dim}q", data, off)
        off += 8 * dim
        specs.append((name, _CODES[code], shape))
    out = {"t": int(t)}
    for name, dt, shape in specs:
        npdt = np.float32 if dt == torch.float32 else np.int32
        nbytes = int(np.prod(shape, dtype=np.int64)) * 4
        out[name] = torch.from_numpy(np.frombuffer(data, dtype=npdt, count=nbytes // 4, offset=off).copy()).reshape(
            shape)
        off += nbytes
    if off != len(data):
        raise ValueError("gate checkpoint has trailing bytes")
    return out
