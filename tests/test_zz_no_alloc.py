"""bm_seq_weights_static: sequence weights without device allocation.

Callers that cannot allocate device memory (another framework's caching
allocator holds it, or a serving loop must not enter the driver allocator)
use this entry point; its scratch is a fixed array inside the library.  The
test calls it through the C ABI and checks that its weights and M_eff equal
those of bm_seq_weights (the same exact tolerance the weight tests use),
on two calls in a row so that stale scratch from the first call would show.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu


def _call_static(lib, msa, w, seqid):
    meff = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.bm_seq_weights_static(ctypes.c_void_p(msa.data_ptr()), msa.shape[0], msa.shape[1],
                                   ctypes.c_double(seqid), ctypes.c_void_p(w.data_ptr()),
                                   ctypes.byref(meff), stream)
    return rc, meff.value


def test_static_scratch_weights_match_allocating_entry_point(bm):
    lib = bm.lib()
    for N, L, seed in [(3000, 96, 1), (777, 130, 2)]:  # second call: smaller N over stale scratch
        X = torch.from_numpy(synth.clustered_msa(N, L, 21, seed, n_ancestors=N // 8)).cuda()
        w_ref = torch.empty(N, dtype=torch.float32, device="cuda")
        meff_ref = bm.bm_seq_weights(X, w_ref, 0.8)
        w = torch.full((N,), -1.0, dtype=torch.float32, device="cuda")
        rc, meff = _call_static(lib, X, w, 0.8)
        assert rc == 0, lib.bm_last_error()
        torch.cuda.synchronize()
        assert torch.equal(w, w_ref)
        assert meff == meff_ref
        rc, meff2 = _call_static(lib, X, w, 0.8)  # repeat on the same inputs
        assert rc == 0 and meff2 == meff_ref
        assert torch.equal(w, w_ref)


def test_static_scratch_rejects_oversize(bm):
    lib = bm.lib()
    limit = 1048576
    X = torch.zeros((1, 8), dtype=torch.uint8, device="cuda")
    w = torch.empty(1, dtype=torch.float32, device="cuda")
    meff = ctypes.c_double()
    rc = lib.bm_seq_weights_static(ctypes.c_void_p(X.data_ptr()), limit + 1, 8, ctypes.c_double(0.8),
                                   ctypes.c_void_p(w.data_ptr()), ctypes.byref(meff), None)
    assert rc == bm.BM_EINVAL
    assert b"static scratch limit" in lib.bm_last_error()
