"""mg_params_fwd / mg_params_bwd against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import params

pytestmark = pytest.mark.gpu


def test_params_fwd_bwd_match_oracle():
    from paper_2603_00145_b300 import ops

    rng = np.random.default_rng(2)
    n = 5003
    mc = (rng.normal(size=(n, 3)) * 0.3).astype(np.float32)
    qr = rng.normal(size=(n, 4)).astype(np.float32)
    ls = (rng.normal(size=(n, 3)) * 0.8).astype(np.float32)
    gm, gq, gs = (rng.normal(size=(n, w)).astype(np.float32) for w in (3, 4, 3))
    centre, half, lr, la = (0.3, 0.1, -0.2), 25.0, 1.5, 0.7
    d = lambda a: torch.from_numpy(a).cuda()
    mean, q, s = torch.empty(n, 3, device="cuda"), torch.empty(n, 4, device="cuda"), torch.empty(n, 3, device="cuda")
    an = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(ops.mg_params_workspace_size(n), dtype=torch.uint8, device="cuda")
    ops.mg_params_fwd(d(mc), d(qr), d(ls), centre, half, lr, mean, q, s, an, ws)
    ref = params.forward(mc, qr, ls, centre, half, lr)
    np.testing.assert_allclose(mean.cpu().numpy(), ref[0], rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(q.cpu().numpy(), ref[1], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(s.cpu().numpy(), ref[2], rtol=1e-6)
    assert abs(float(an.item()) - ref[3]) <= 1e-6 * max(1.0, ref[3])
    out = [torch.empty(n, w, device="cuda") for w in (3, 4, 3)]
    ops.mg_params_bwd(d(qr), d(ls), half, lr, la, d(gm), d(gq), d(gs), *out)
    want = params.backward(mc, qr, ls, centre, half, lr, la, gm, gq, gs)
    for got, w in zip(out, want):
        g = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - w) <= 1e-5 * np.linalg.norm(w)
