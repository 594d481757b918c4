"""GPU parity of the paper's cell-grid local set (MG_LOCAL_CELLS, Eqs.
E4-E6) against the FP64 oracle: records bit-exact, slices, gradients, slice
poses and the volume sampler."""
import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from gpu_util import assert_grads_close, assert_render_close, gpu_bins, rel_l2, to_dev, TOL_GRAD_REL

pytestmark = pytest.mark.gpu


def _case(seed, n=300):
    rng = np.random.default_rng(seed)
    G = ms.random_gaussians(n, 700 + seed, box=(-20, 20), sigma=(0.6, 3.0), aniso=3.0, negative_frac=0.1)
    stacks = [ms.make_stack(ms.AXIAL, 6, 37, 45, 1.0, 1.1, 3.0, 3.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 5, 40, 36, 0.9, 0.9, 2.0, 2.5, rng=rng,
                            max_rot_deg=5.0, max_trans_mm=1.0, psf_u=1.0),
              ms.make_stack(ms.SAGITTAL, 4, 30, 18, 1.3, 1.2, 0.0, 4.0)]
    return G, stacks


@pytest.mark.parametrize("seed,res,radius", [(0, 20, 2), (1, 32, 5), (2, 12, 0)])
def test_cells_records_render_and_gradients(seed, res, radius):
    from paper_2603_00145_b300 import SliceRenderer

    G, stacks = _case(seed)
    cells = dict(grid_res=res, block_radius=radius, centre=(0.4, -0.3, 0.2), half=24.0)
    R = SliceRenderer(stacks, cells=cells)
    m, q, s, a = to_dev(G)
    out = R.forward(m, q, s, a)
    torch.cuda.synchronize()
    rec = orc.records(G, stacks, cells=cells)
    st, (gid, sl, rect, inset, toff, ent) = gpu_bins(R, G.n)
    assert st["status"] == 0 and st["records"] == rec.n
    assert np.array_equal(gid.numpy(), rec.gid) and np.array_equal(sl.numpy(), rec.slice)
    assert np.array_equal(rect.numpy(), rec.rect)
    assert np.array_equal(inset.numpy().view(np.uint64), rec.inset)
    want = orc.render(G, stacks, rec, cells=cells)
    assert_render_close(out.cpu().numpy(), want, "cells fwd")
    gout = np.random.default_rng(seed).normal(size=want.size).astype(np.float32)
    g = R.backward(m, q, s, a, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, stacks, rec, gout.astype(np.float64), cells)
    assert_grads_close(g, ref, G, "cells")
    # slice poses (unit quaternions for the oracle's rigid-motion chain)
    pg = R.pose_grad(m, q, s, a).cpu().numpy().astype(np.float64)
    qn = np.asarray(G.quat, np.float64)
    Gu = ms.Gaussians(G.mean, (qn / np.linalg.norm(qn, axis=1, keepdims=True)), G.scale, G.alpha)
    pw = orc.pose_grad(Gu, stacks, rec, gout.astype(np.float64), cells)
    assert rel_l2(pg[:, :3], pw[:, :3]) <= TOL_GRAD_REL and rel_l2(pg[:, 3:], pw[:, 3:]) <= 5 * TOL_GRAD_REL


def test_cells_sampler():
    from paper_2603_00145_b300.ops import VolumeSampler

    G, _ = _case(5, n=200)
    cells = dict(grid_res=24, block_radius=3, centre=(0.0, 0.0, 0.0), half=24.0)
    Gd, h = 40, 1.1
    S = VolumeSampler(Gd, h, (0.5, -0.25, 0.125), cells=cells)
    m, q, s, a = to_dev(G)
    got = S(m, q, s, a).cpu().numpy()
    want = orc.sample_volume(G, Gd, h, (0.5, -0.25, 0.125), cells=cells)
    assert_render_close(got, want, "cells sampler")


def test_cells_argument_checks():
    from paper_2603_00145_b300 import SliceRenderer, _lib as L

    G, stacks = _case(6, n=20)
    m, q, s, a = to_dev(G)
    R = SliceRenderer(stacks, cells=dict(grid_res=4096, block_radius=5, centre=(0, 0, 0), half=5.0))
    with pytest.raises(L.MgError):
        R.forward(m, q, s, a)   # a tile would span too many cells
    R = SliceRenderer(stacks, cells=dict(grid_res=16, block_radius=2, centre=(0, 0, 0), half=20.0))
    R.forward(m, q, s, a)
    with pytest.raises(L.MgError):
        R.pair_count(m, q, s, a)  # pair statistics are for the K-sigma local set
