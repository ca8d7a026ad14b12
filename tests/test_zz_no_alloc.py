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


@pytest.mark.parametrize("d,hidden", [(64, 16), (128, 32)])
def test_noalloc_matches_allocating_backward_twice(d, hidden):
    """Two calls in a row, the second on a shorter pair list and another
    upstream gradient, so a block partial left over from the first call would
    change the second result.  The entry point runs the same kernels with the
    same fixed grid and reduction order as subquad_fuse_backward, so each
    result must equal the allocating entry point's bit for bit."""
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
        m_all = int(pairs.shape[0])
        lib = subquad.lib()
        P = ctypes.c_void_p
        for call, (m, seed) in enumerate([(m_all, 21), (m_all - 12_345, 22)]):
            dL = torch.from_numpy((np.random.default_rng(seed).standard_normal(m) / m).astype(np.float32)).cuda()
            want = ctx.fuse_backward(pairs[:m], sw[:m], self_sc, packed, emb, params, hidden, dL, want_emb=False)
            want_np = want.cpu().numpy()
            scratch_before = ctx.scratch_bytes()
            out = torch.full((5 * hidden + 1,), float("nan"), dtype=torch.float32, device="cuda")
            st = lib.subquad_fuse_backward_params_noalloc(
                ctx.handle, P(pairs.data_ptr()), m, P(sw.data_ptr()), P(self_sc.data_ptr()), P(packed.data_ptr()),
                int(packed.shape[1]), P(emb.data_ptr()), d, P(params.data_ptr()), hidden, P(dL.data_ptr()),
                P(out.data_ptr()))
            assert st == 0, subquad.lib().subquad_strerror(st)
            ctx.check()
            got = out.cpu().numpy()
            assert np.array_equal(got, want_np), f"call {call}: differs from subquad_fuse_backward"
            assert ctx.scratch_bytes() == scratch_before, "the call grew the context scratch"
