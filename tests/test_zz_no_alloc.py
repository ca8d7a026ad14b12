"""The allocation-free parameter gradient (subquad_fuse_backward_params_noalloc).

It serves callers that cannot let the library call cudaMalloc -- for example a
training loop whose free device memory is held by a caching allocator, or one
that must avoid cudaMalloc's implicit device synchronisation.  Its block
partials live in a static device array instead of context scratch.  This test
calls it through the C ABI twice in a row and compares each result with the
allocating entry point (subquad_fuse_backward) under the gradient tolerance
of the other GPU tests.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

pytestmark = pytest.mark.gpu


def _close(got, want, scale, rel=1e-4, floor=1e-6):
    err = np.abs(got.astype(np.float64) - want.astype(np.float64))
    return bool((err <= rel * np.abs(want) + floor * scale).all())


@pytest.mark.parametrize("d,hidden", [(64, 16), (128, 32)])
def test_noalloc_matches_allocating_backward_twice(d, hidden):
    import torch

    from paper_2602_17330_gb300 import _build, subquad

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    with subquad.Context(0) as ctx:
        rep = synth.donor_repertoire(20_000, seed=21)
        a, b = synth.hash_coefficients(64, seed=21)
        packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
        sig = ctx.sign(packed, rep.n, 3, torch.from_numpy(a.view(np.int32)), torch.from_numpy(b.view(np.int32)), 16, 4)
        pairs = ctx.band_candidates(sig, rep.n, 16, 4, 2048)
        sw = ctx.align_score(packed, pairs)
        self_sc = ctx.self_scores(packed)
        emb = torch.from_numpy(synth.family_embeddings(rep.family, d, seed=21)).cuda()
        params = torch.from_numpy(synth.gate_parameters(hidden, seed=21)).cuda()
        m = int(pairs.shape[0])
        dL = torch.from_numpy((np.random.default_rng(21).standard_normal(m) / m).astype(np.float32)).cuda()
        want = ctx.fuse_backward(pairs, sw, self_sc, packed, emb, params, hidden, dL, want_emb=False)
        want_np = want.cpu().numpy()
        scale = float(dL.abs().sum()) * 20.0
        scratch_before = ctx.scratch_bytes()
        lib = subquad.lib()
        P = ctypes.c_void_p
        for call in range(2):
            out = torch.full((5 * hidden + 1,), float("nan"), dtype=torch.float32, device="cuda")
            st = lib.subquad_fuse_backward_params_noalloc(
                ctx.handle, P(pairs.data_ptr()), m, P(sw.data_ptr()), P(self_sc.data_ptr()), P(packed.data_ptr()),
                int(packed.shape[1]), P(emb.data_ptr()), d, P(params.data_ptr()), hidden, P(dL.data_ptr()),
                P(out.data_ptr()))
            assert st == 0, subquad.lib().subquad_strerror(st)
            ctx.check()
            got = out.cpu().numpy()
            assert np.isfinite(got).all(), f"call {call}: output not written"
            assert _close(got, want_np, scale), f"call {call}: differs from subquad_fuse_backward"
        assert ctx.scratch_bytes() == scratch_before, "the call grew the context scratch"
