"""bm_seq_weights_static: sequence weights without device allocation.

Callers that cannot allocate device memory (another framework's caching
allocator holds it, or a serving loop must not enter the driver allocator)
use this entry point; its scratch is a fixed array inside the library.  The
tests call it through the C ABI and check
  * its weights and M_eff against the FP64 oracle's seq_weights (Eq. 7;
    bit-exact, as the weight parity tests require) and against the
    allocating entry point bm_seq_weights;
  * shapes that span several 256-symbol chunks of its identity kernel
    (L = 300) and sequence counts that are not multiples of 64;
  * two calls in a row, the second over the first call's stale scratch;
  * that a call allocates nothing: the device's free memory and torch's
    allocator figures are unchanged across calls after the first (which
    may load the library's module and with it the array).
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [(3000, 96, 1), (777, 130, 2), (1001, 300, 3), (65, 513, 4)]


def _call_static(lib, msa, w, seqid):
    meff = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.bm_seq_weights_static(ctypes.c_void_p(msa.data_ptr()), msa.shape[0], msa.shape[1],
                                   ctypes.c_double(seqid), ctypes.c_void_p(w.data_ptr()),
                                   ctypes.byref(meff), stream)
    return rc, meff.value


def test_static_scratch_weights_match_oracle_and_allocating_entry_point(bm, orc):
    lib = bm.lib()
    for N, L, seed in CASES:  # later calls: other N and L over stale scratch
        msa = synth.clustered_msa(N, L, 21, seed, n_ancestors=max(1, N // 8))
        X = torch.from_numpy(msa).cuda()
        w_o, meff_o = orc.seq_weights(msa, 0.8)
        w_ref = torch.empty(N, dtype=torch.float32, device="cuda")
        meff_ref = bm.bm_seq_weights(X, w_ref, 0.8)
        w = torch.full((N,), -1.0, dtype=torch.float32, device="cuda")
        rc, meff = _call_static(lib, X, w, 0.8)
        assert rc == 0, lib.bm_last_error()
        torch.cuda.synchronize()
        # weights are 1/N_m of an exact integer count: FP32 of the oracle's FP64
        assert np.array_equal(w.cpu().numpy(), w_o.astype(np.float32)), (N, L)
        assert abs(meff - meff_o) <= 1e-9 * meff_o, (N, L, meff, meff_o)
        assert torch.equal(w, w_ref)
        assert meff == meff_ref
        rc, meff2 = _call_static(lib, X, w, 0.8)  # repeat on the same inputs
        assert rc == 0 and meff2 == meff_ref
        assert torch.equal(w, w_ref)


def test_static_scratch_allocates_nothing(bm):
    lib = bm.lib()
    N, L = 2000, 120
    X = torch.from_numpy(synth.clustered_msa(N, L, 21, 9, n_ancestors=250)).cuda()
    w = torch.empty(N, dtype=torch.float32, device="cuda")
    rc, _ = _call_static(lib, X, w, 0.8)  # first call on the device: set-up
    assert rc == 0, lib.bm_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(3):
        rc, _ = _call_static(lib, X, w, 0.8)
        assert rc == 0, lib.bm_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0


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
