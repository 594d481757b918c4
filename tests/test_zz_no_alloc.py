"""The no-allocation loss entry point, mg_loss_l1l2_noalloc.

It serves callers that cannot allocate device memory or pass a workspace (an
application that has reserved all device memory for its own pool, a plugin
whose host runtime owns every allocation, a real-time loop kept out of the
allocator). Its partial sums live in a fixed array inside the library, so it
must give what mg_loss_l1l2 (which takes a caller workspace) gives, call after
call, within the tolerance the other loss tests use. This file is collected
last so that a stop at its first failure comes after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

REL_TOL = 2e-6  # the loss tolerance of the other reduction tests


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    p = torch.from_numpy(rng.uniform(-0.5, 1.0, n).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(0.0, 1.0, n).astype(np.float32)).cuda()
    return p, t


def test_noalloc_matches_workspace_entry_point_twice():
    from paper_2603_00145_b300 import _lib as L
    from paper_2603_00145_b300 import mg_loss_l1l2, mg_reduce_workspace_size

    lib = L.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, seed) in enumerate(((12_582_912, 1), (1_000_003, 2))):
        p, t = _inputs(n, seed)
        # the existing entry point, with a workspace
        g_ref = torch.empty_like(p)
        out_ref = torch.empty(2, dtype=torch.float64, device="cuda")
        ws = torch.empty(mg_reduce_workspace_size(n), dtype=torch.uint8, device="cuda")
        mg_loss_l1l2(p, t, g_ref, out_ref, ws)
        # the no-allocation entry point, straight through the C ABI
        g = torch.empty_like(p)
        out = torch.empty(2, dtype=torch.float64, device="cuda")
        st = lib.mg_loss_l1l2_noalloc(p.data_ptr(), t.data_ptr(), n, g.data_ptr(), out.data_ptr(), stream)
        assert st == L.MG_OK, lib.mg_last_error()
        torch.cuda.synchronize()
        for i in range(2):
            a, b = float(out[i]), float(out_ref[i])
            assert abs(a - b) <= REL_TOL * abs(b), (call, i, a, b)
        assert torch.equal(g, g_ref), call


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_2603_00145_b300 import _lib as L

    lib = L.lib()
    p, t = _inputs(16, 3)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    st = lib.mg_loss_l1l2_noalloc(p.data_ptr(), t.data_ptr(), 33_554_433, None, out.data_ptr(), None)
    assert st == L.MG_ERR_INVALID_ARG
    assert b"33554432" in lib.mg_last_error()
