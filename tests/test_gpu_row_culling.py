"""Per-row culling of the records' tile rectangles at its limits (the local
set of Sec. 3.3.1 restricted per tile): rectangles taller than eight tile
rows (the rows past the eighth are listed whole), wider than sixteen tiles
(insets capped at 15), needles above the 64:1 scale ratio (not culled; FP64
geometry), thin rotated ellipses, and ellipses clipped by the image border.
Records, rectangles, row insets and tile lists equal the oracle's bit for
bit; the slices and gradients match it within the parity tolerances."""
import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from gpu_util import assert_grads_close, assert_render_close, gpu_bins, render_gpu

pytestmark = pytest.mark.gpu


def _gaussians():
    rng = np.random.default_rng(21)
    big = ms.random_gaussians(8, 3, box=(-15, 15), sigma=(7.0, 12.0), aniso=8.0)      # tall and wide rectangles
    thin = ms.random_gaussians(40, 4, box=(-30, 30), sigma=(0.6, 2.0), aniso=12.0)    # thin rotated ellipses
    edge = ms.random_gaussians(30, 5, box=(-40, 40), sigma=(1.0, 4.0), aniso=3.0)     # many cut by the border
    n_needle = 4
    needle = ms.Gaussians(rng.uniform(-10, 10, size=(n_needle, 3)), ms.random_unit_quats(n_needle, rng),
                          np.tile(np.array([[0.15, 0.2, 14.0]]), (n_needle, 1)), np.full(n_needle, 0.7))
    # long thin ellipses lying diagonally in the axial slices: each tile row of their
    # image-wide rectangles touches a few tiles at one end (insets capped at 15)
    th = np.deg2rad(np.array([35.0, 135.0, 150.0]))
    c = np.sqrt(0.5)
    diag = ms.Gaussians(np.array([[0.0, 0.0, 1.0], [2.0, -3.0, -2.5], [-4.0, 1.0, 0.5]]),
                        np.stack([np.full(3, c), -c * np.sin(th), c * np.cos(th), np.zeros(3)], axis=1),
                        np.tile(np.array([[2.0, 2.0, 25.0]]), (3, 1)), np.full(3, 0.8))
    parts = [big, thin, edge, needle, diag]
    return ms.Gaussians(*(np.concatenate([getattr(p, f) for p in parts]) for f in ("mean", "quat", "scale",
                                                                                    "alpha")))


def _stacks():
    rng = np.random.default_rng(8)
    return [ms.make_stack(ms.AXIAL, 6, 176, 168, 0.5, 0.45, 2.0, 3.0),
            ms.make_stack(ms.random_rotations(1, rng)[0], 5, 80, 100, 0.6, 0.6, 1.5, 4.0, psf_u=1.0, psf_v=0.6)]


def test_row_culling_limits_bit_exact_and_parity():
    G, stacks = _gaussians(), _stacks()
    R, out, dev = render_gpu(G, stacks)
    rec = orc.records(G, stacks, 3.0)
    st, (gid, sl, rect, inset, toff, ent) = gpu_bins(R, G.n)
    assert st["status"] == 0 and st["records"] == rec.n
    assert np.array_equal(gid.numpy(), rec.gid) and np.array_equal(sl.numpy(), rec.slice)
    assert np.array_equal(rect.numpy(), rec.rect)
    ins = inset.numpy().view(np.uint64)
    assert np.array_equal(ins, rec.inset)
    # the limits are exercised: tall rectangles, capped insets, culled and unculled records
    heights = rec.rect[:, 3] - rec.rect[:, 1] + 1
    assert (heights > 8).any()
    nib = (ins[:, None] >> (np.arange(16, dtype=np.uint64) * 4)) & np.uint64(15)
    assert (nib == 15).any()
    assert (ins != 0).any() and (ins == 0).sum() > 0
    counts, offs, ids = orc.tile_bins(rec, stacks)
    assert st["entries"] == ids.size and np.array_equal(toff.numpy(), offs)
    e = ent.numpy()
    for t in np.nonzero(counts)[0]:
        assert np.array_equal(np.sort(e[offs[t]:offs[t + 1]]), ids[offs[t]:offs[t + 1]]), t
    want = orc.render(G, stacks, rec)
    assert_render_close(out.cpu().numpy(), want, "row culling limits")
    gout = np.random.default_rng(3).normal(size=want.size).astype(np.float32)
    g = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, stacks, rec, gout.astype(np.float64))
    assert_grads_close(g, ref, G, "row culling limits")
