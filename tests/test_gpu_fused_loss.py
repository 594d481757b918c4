"""mg_render_fwd_l1l2: the forward with the L1 + L2 slice loss fused into the
evaluation kernel gives the slices of mg_render_fwd and the gradient of
mg_loss_l1l2 bit for bit, and the loss of both within the error of their
FP32 partial sums (grouped differently: 16-voxel leaves there, 8x8 tiles
here) of the FP64 loss of the same slices (Sec. 3.5.2 with the plain fit's
loss)."""
import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _case(seed, n=300):
    rng = np.random.default_rng(seed)
    G = ms.random_gaussians(n, 300 + seed, box=(-22, 22), sigma=(0.6, 3.0), aniso=3.0, alpha=(0.1, 1.0),
                            negative_frac=0.1)
    stacks = [ms.make_stack(ms.AXIAL, 9, 37, 50, 1.0, 1.1, 3.0, 3.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 7, 48, 40, 0.9, 0.9, 2.0, 2.5, rng=rng,
                            max_rot_deg=5.0, max_trans_mm=1.0),
              ms.make_stack(ms.SAGITTAL, 5, 33, 17, 1.3, 1.2, 0.0, 4.0)]
    return G, stacks, rng


def _fused_vs_separate(G, stacks, rng, cells=None):
    from paper_2603_00145_b300 import SliceRenderer, mg_loss_l1l2, mg_reduce_workspace_size

    R = SliceRenderer(stacks, cells=cells)
    d = to_dev(G)
    nv = R.dev.n_vox
    target = torch.from_numpy(rng.uniform(0.0, 1.0, nv).astype(np.float32)).cuda()
    out1 = R.forward(*d)
    grad1 = torch.empty(nv, device="cuda")
    loss1 = torch.empty(2, dtype=torch.float64, device="cuda")
    mg_loss_l1l2(out1, target, grad1, loss1, torch.empty(mg_reduce_workspace_size(nv), dtype=torch.uint8,
                                                         device="cuda"))
    out2 = torch.empty(nv, device="cuda")
    grad2 = torch.empty(nv, device="cuda")
    loss2 = torch.empty(2, dtype=torch.float64, device="cuda")
    R.forward_l1l2(*d, target, out2, grad2, loss2)
    assert torch.equal(out1, out2)
    assert torch.equal(grad1, grad2)
    l1, l2 = loss1.cpu().numpy(), loss2.cpu().numpy()
    np.testing.assert_allclose(l2, l1, rtol=1e-6)
    # against the FP64 oracle's loss of the GPU's own slices (the leaf sums are FP32)
    r = out2.cpu().numpy().astype(np.float64) - target.cpu().numpy().astype(np.float64)
    want = np.abs(r).mean() + (r * r).mean()
    assert abs(l2[0] - want) <= 2e-6 * want
    assert abs(l2[1] - (r * r).sum()) <= 2e-6 * (r * r).sum()
    return R, d, grad2


def test_fused_loss_matches_separate_and_oracle():
    G, stacks, rng = _case(0)
    R, d, g = _fused_vs_separate(G, stacks, rng)
    # the backward runs on the fused forward's workspace
    gm, gq, gs, ga = R.backward(*d, g)
    ref = orc.grad(G, stacks, orc.records(G, stacks), g.cpu().numpy().astype(np.float64))
    rel = np.linalg.norm(ga.cpu().numpy() - ref["alpha"]) / np.linalg.norm(ref["alpha"])
    assert rel <= 1e-4, rel


def test_fused_loss_with_cell_grid_local_set():
    G, stacks, rng = _case(1)
    _fused_vs_separate(G, stacks, rng, cells=dict(grid_res=24, block_radius=3, centre=(0.0, 0.0, 0.0), half=24.0))


def test_fused_loss_without_gaussians():
    from paper_2603_00145_b300 import SliceRenderer

    stacks = [ms.make_stack(ms.AXIAL, 3, 20, 21, 1.0, 1.0, 3.0, 3.0)]
    R = SliceRenderer(stacks)
    nv = R.dev.n_vox
    target = torch.linspace(-1.0, 1.0, nv, device="cuda")
    e = torch.empty(0, 3, device="cuda")
    out = torch.empty(nv, device="cuda")
    grad = torch.empty(nv, device="cuda")
    loss = torch.empty(2, dtype=torch.float64, device="cuda")
    R.forward_l1l2(e, torch.empty(0, 4, device="cuda"), e.clone(), torch.empty(0, device="cuda"), target, out, grad,
                   loss)
    t = target.cpu().numpy().astype(np.float64)
    assert float(out.abs().max()) == 0.0
    np.testing.assert_allclose(loss.cpu().numpy()[0], np.abs(t).mean() + (t * t).mean(), rtol=2e-6)


def test_fused_loss_with_unaligned_target_and_grad():
    """Rows of 64 pixels are 16-byte aligned in `out`, while target and grad
    start one float past an aligned address: the empty tiles' vector path
    must check each pointer on its own (results as with aligned buffers)."""
    from paper_2603_00145_b300 import SliceRenderer

    rng = np.random.default_rng(7)
    G = ms.random_gaussians(60, 77, box=(-10, 10), sigma=(0.6, 1.5), aniso=2.0)
    stacks = [ms.make_stack(ms.AXIAL, 4, 64, 64, 1.0, 1.0, 2.0, 2.0)]
    R = SliceRenderer(stacks)
    d = to_dev(G)
    nv = R.dev.n_vox
    t_host = rng.uniform(0.0, 1.0, nv).astype(np.float32)
    tgt_a = torch.from_numpy(t_host).cuda()
    tgt_u = torch.empty(nv + 1, device="cuda")[1:]
    tgt_u.copy_(tgt_a)
    outs = []
    for tgt, off in ((tgt_a, 0), (tgt_u, 1)):
        out = torch.empty(nv, device="cuda")
        gbuf = torch.empty(nv + off, device="cuda")[off:]
        loss = torch.empty(2, dtype=torch.float64, device="cuda")
        R.forward_l1l2(*d, tgt, out, gbuf, loss)
        outs.append((out.clone(), gbuf.clone(), loss.cpu().numpy()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])
