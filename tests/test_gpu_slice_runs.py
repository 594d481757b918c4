"""Record-count shortcuts on every kind of slice run (Sec. 3.3.1 local set,
the K-sigma slab test of the record predicate): runs of parallel slices
whose plane offsets decrease (a stack stepped against its normal), runs with
equal offsets (a slice repeated), runs crossing the 32-slice window of the
count pass, and moving slices (a screen before the frame terms). Records,
tile rectangles, row insets and tile lists must equal the oracle's bit for
bit, and the slices its render."""
import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from gpu_util import assert_render_close, gpu_bins, render_gpu

pytestmark = pytest.mark.gpu


def _stack_with(st, xf):
    return ms.Stack(xf.shape[0], st.H, st.W, st.dx, st.dy, st.thickness, np.ascontiguousarray(xf, np.float32),
                    st.psf_u, st.psf_v)


def _cases():
    rng = np.random.default_rng(5)
    base = ms.make_stack(ms.random_rotations(1, rng)[0], 40, 33, 29, 1.0, 1.1, 2.5, 1.6)
    reversed_ = _stack_with(base, base.xform[::-1])                       # offsets decrease along the run
    rep = np.concatenate([base.xform[:12], base.xform[11:12], base.xform[11:12], base.xform[12:20]])
    repeated = _stack_with(base, rep)                                      # equal offsets: no monotone run
    moving = ms.make_stack(ms.AXIAL, 20, 30, 30, 1.0, 1.0, 2.0, 1.5, rng=rng, max_rot_deg=4.0, max_trans_mm=1.0)
    return [("window-crossing", [base]), ("reversed", [reversed_]), ("repeated", [repeated]),
            ("moving", [moving]), ("all", [base, reversed_, repeated, moving])]


@pytest.mark.parametrize("name,stacks", _cases(), ids=[c[0] for c in _cases()])
def test_runs_bins_bit_exact(name, stacks):
    G = ms.random_gaussians(600, 77, box=(-22, 22), sigma=(0.5, 3.0), aniso=3.0)
    R, out, dev = render_gpu(G, stacks)
    rec = orc.records(G, stacks, 3.0)
    st, (gid, sl, rect, inset, toff, ent) = gpu_bins(R, G.n)
    assert st["status"] == 0 and st["records"] == rec.n > 0
    assert np.array_equal(gid.numpy(), rec.gid) and np.array_equal(sl.numpy(), rec.slice)
    assert np.array_equal(rect.numpy(), rec.rect)
    assert np.array_equal(inset.numpy().view(np.uint64), rec.inset)
    counts, offs, ids = orc.tile_bins(rec, stacks)
    assert st["entries"] == ids.size and np.array_equal(toff.numpy(), offs)
    e = ent.numpy()
    for t in np.nonzero(counts)[0]:
        assert np.array_equal(np.sort(e[offs[t]:offs[t + 1]]), ids[offs[t]:offs[t + 1]]), t
    assert_render_close(out.cpu().numpy(), orc.render(G, stacks, rec), name)


def test_many_records_per_gaussian_gradients():
    """Gaussians elongated along the normal of an 80-slice stack have a record
    in nearly every slice (more than 64: the chain sums them with the whole
    warp, lane-strided, in a fixed shuffle tree); slices and gradients against
    the oracle (the moments themselves sum by FP32 atomics, so gradients are not
    compared between runs)."""
    from gpu_util import assert_grads_close

    rng = np.random.default_rng(12)
    st = [ms.make_stack(ms.AXIAL, 80, 24, 22, 1.0, 1.0, 1.0, 0.5)]
    n_long = 5
    quat = np.tile(np.array([[1.0, 0.0, 0.0, 0.0]]), (n_long, 1)) + rng.normal(scale=0.05, size=(n_long, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    longs = ms.Gaussians(rng.uniform(-4, 4, size=(n_long, 3)), quat,
                         np.column_stack([rng.uniform(1.5, 3.0, n_long), rng.uniform(1.5, 3.0, n_long),
                                          np.full(n_long, 12.0)]), rng.uniform(0.3, 1.0, n_long))
    short = ms.random_gaussians(60, 13, box=(-10, 10), sigma=(0.6, 2.0), aniso=2.0)
    G = ms.Gaussians(*(np.concatenate([getattr(p, f) for p in (longs, short)]) for f in ("mean", "quat", "scale",
                                                                                         "alpha")))
    R, out, dev = render_gpu(G, st)
    rec = orc.records(G, st, 3.0)
    per_g = np.bincount(rec.gid, minlength=G.n)
    assert (per_g[:n_long] > 64).all(), per_g[:n_long]
    want = orc.render(G, st, rec)
    assert_render_close(out.cpu().numpy(), want, "many records")
    gout = np.random.default_rng(14).normal(size=want.size).astype(np.float32)
    g1 = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, st, rec, gout.astype(np.float64))
    assert_grads_close(g1, ref, G, "many records")
