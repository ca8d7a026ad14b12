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
        torch.save(self.checkpoint(), path)

    def load(self, path: str) -> None:
        self.restore(torch.load(path, map_location="cpu"))
