"""The fused reconstruction loss (smooth L1 + lambda_SSIM (1 - mean SSIM),
Sec. 3.5.2) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import mg_synth as ms
from oracle import ssim as orc_ssim

pytestmark = pytest.mark.gpu


def _stacks():
    # ragged sizes: partial tiles, a slice narrower than the window, several stacks
    return [ms.make_stack(ms.AXIAL, 3, 37, 50, 1.0, 1.0, 2.0, 2.0),
            ms.make_stack(ms.CORONAL, 2, 70, 33, 1.0, 1.0, 2.0, 2.0),
            ms.make_stack(ms.SAGITTAL, 2, 4, 9, 1.0, 1.0, 2.0, 2.0)]


def _slices(flat, stacks):
    out, o = [], 0
    for s in stacks:
        for _ in range(s.n_slices):
            out.append(flat[o:o + s.H * s.W].reshape(s.H, s.W))
            o += s.H * s.W
    return out


def _run(pred, target, stacks, lam=0.5, with_grad=True):
    from paper_2603_00145_b300 import ops

    D = ops.DeviceStacks(stacks)
    p = torch.from_numpy(pred.astype(np.float32)).cuda()
    t = torch.from_numpy(target.astype(np.float32)).cuda()
    g = torch.empty_like(p) if with_grad else None
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    ws = torch.empty(ops.mg_loss_recon_workspace_size(D), dtype=torch.uint8, device="cuda")
    ops.mg_loss_recon(p, t, D, lam, g, out, ws)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (g.cpu().numpy() if with_grad else None)


def _check(pred, target, stacks, lam=0.5):
    out, g = _run(pred, target, stacks, lam)
    p32 = pred.astype(np.float32).astype(np.float64)
    t32 = target.astype(np.float32).astype(np.float64)
    L, l1, ss, grads = orc_ssim.recon_loss(_slices(p32, stacks), _slices(t32, stacks), lam)
    gref = np.concatenate([x.ravel() for x in grads])
    assert abs(out[1] - l1) <= 1e-6 * max(abs(l1), 1e-3), (out[1], l1)
    assert abs(out[2] - ss) <= 2e-6, (out[2], ss)
    assert abs(out[0] - L) <= 2e-6 * max(abs(L), 1e-3), (out[0], L)
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert rel <= 1e-4, rel
    assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()
    return out, rel


def test_random_slices_ragged_stacks():
    st = _stacks()
    n = sum(s.n_slices * s.H * s.W for s in st)
    rng = np.random.default_rng(0)
    target = rng.uniform(0, 1, n)
    pred = np.clip(target + rng.normal(0, 0.1, n), -0.2, 1.2)
    pred[::97] += 1.7      # residuals on the linear branch of the smooth L1
    _check(pred, target, st)
    _check(pred, target, st, lam=0.0)


def test_rendered_slices_against_acquired():
    """Smooth images (a Gaussian render) against noisy simulated slices."""
    from gpu_util import render_gpu

    wl = ms.tiny_workload(0)
    G = ms.random_gaussians(300, 5, box=(-20, 20), sigma=(1.0, 3.0), aniso=2.0)
    _, out, _ = render_gpu(G, wl.stacks)
    vol = wl.phantom.volume_torch(device="cuda")
    tgt = torch.cat([ms.simulate_stack(vol, 1.0, s, seed=i, noise_sigma=0.01, device="cuda").reshape(-1)
                     for i, s in enumerate(wl.stacks)])
    _check(out.cpu().numpy().astype(np.float64), tgt.cpu().numpy().astype(np.float64), wl.stacks)


def test_deterministic_and_no_grad():
    st = _stacks()
    n = sum(s.n_slices * s.H * s.W for s in st)
    rng = np.random.default_rng(1)
    t = rng.uniform(0, 1, n)
    p = rng.uniform(0, 1, n)
    a, ga = _run(p, t, st)
    b, gb = _run(p, t, st)
    c, _ = _run(p, t, st, with_grad=False)
    assert np.array_equal(a, b) and np.array_equal(ga, gb) and np.array_equal(a, c)
    s1, _ = _run(t, t, st)
    assert abs(s1[2] - 1.0) < 1e-6 and s1[1] == 0.0


def test_invalid_arguments():
    from paper_2603_00145_b300 import ops, _lib as L

    st = _stacks()
    D = ops.DeviceStacks(st)
    x = torch.zeros(D.n_vox, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    ws = torch.empty(ops.mg_loss_recon_workspace_size(D), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.MgError):
        ops.mg_loss_recon(x, x, D, -1.0, None, out, ws)
    with pytest.raises(L.MgError):
        ops.mg_loss_recon(x, x, D, 0.5, None, out, ws[:8])
