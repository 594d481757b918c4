"""Pins of the oracle's cell-grid local set (the paper's Eqs. E4-E6): the
binned render equals a brute-force sum over every (Gaussian, voxel) pair
with the membership decided by the paper's cell formula (FP32, written
here with numpy, no records or tiles), equals the full sum when the block
radius covers the grid, and its gradient matches finite differences."""
import types

import numpy as np
import pytest

import mg_synth as ms
import oracle as orc

F32 = np.float32


def _cell(p, c, h, hres):
    t = (F32(p) - F32(c)) / F32(h)
    t = (t + F32(1.0)) * F32(hres)
    t = np.where(np.isnan(t), F32(-1048576.0), np.clip(t, F32(-1048576.0), F32(1048576.0)))
    return np.floor(t).astype(np.int64)


def _voxel_cells(st, cells):
    """[n_slices, H, W, 3] cells of every voxel (FP32, the written order)."""
    hres = F32(0.5 * cells["grid_res"])
    hx, hy = F32(0.5) * F32(st.W - 1), F32(0.5) * F32(st.H - 1)
    u = (np.arange(st.W, dtype=F32) - hx) * F32(st.dx)
    v = (np.arange(st.H, dtype=F32) - hy) * F32(st.dy)
    out = np.zeros((st.n_slices, st.H, st.W, 3), np.int64)
    for k in range(st.n_slices):
        xf = np.asarray(st.xform[k], F32)
        for a in range(3):
            x = (xf[3 * a] * u[None, :] + xf[3 * a + 1] * v[:, None]).astype(F32) + xf[9 + a]
            out[k, :, :, a] = _cell(x, cells["centre"][a], cells["half"], hres)
    return out


def _brute(G, stacks, cells):
    hres = 0.5 * cells["grid_res"]
    gcell = np.stack([_cell(np.asarray(G.mean, F32)[:, a], cells["centre"][a], cells["half"], hres)
                      for a in range(3)], axis=1)
    total = np.zeros(sum(s.n_vox for s in stacks))
    for g in range(G.n):
        one = ms.Gaussians(G.mean[g:g + 1], G.quat[g:g + 1], G.scale[g:g + 1], G.alpha[g:g + 1])
        full = orc.render(one, stacks, exact=True)
        o = 0
        for st in stacks:
            vc = _voxel_cells(st, cells).reshape(-1, 3)
            member = np.all(np.abs(vc - gcell[g]) <= cells["block_radius"], axis=1)
            total[o:o + st.n_vox] += np.where(member, full[o:o + st.n_vox], 0.0)
            o += st.n_vox
    return total


def _case(seed):
    rng = np.random.default_rng(seed)
    G = ms.random_gaussians(40, 900 + seed, box=(-14, 14), sigma=(0.6, 2.5), aniso=3.0, negative_frac=0.2)
    stacks = [ms.make_stack(ms.AXIAL, 3, 21, 26, 1.0, 1.1, 2.5, 3.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 3, 19, 23, 0.9, 1.0, 2.0, 3.0, rng=rng,
                            max_rot_deg=4.0, max_trans_mm=1.0, psf_u=0.8)]
    return G, stacks


@pytest.mark.parametrize("seed,res,radius", [(0, 16, 1), (1, 24, 2), (2, 10, 0)])
def test_cells_render_equals_brute_force_member_sum(seed, res, radius):
    G, stacks = _case(seed)
    cells = dict(grid_res=res, block_radius=radius, centre=(0.3, -0.2, 0.1), half=16.0)
    rec = orc.records(G, stacks, cells=cells)
    got = orc.render(G, stacks, rec, cells=cells)
    want = _brute(G, stacks, cells)
    assert np.abs(want).max() > 0
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


def test_radius_covering_the_grid_gives_the_full_sum():
    G, stacks = _case(3)
    cells = dict(grid_res=8, block_radius=8, centre=(0.0, 0.0, 0.0), half=20.0)
    got = orc.render(G, stacks, orc.records(G, stacks, cells=cells), cells=cells)
    np.testing.assert_allclose(got, orc.render(G, stacks, exact=True), rtol=1e-12, atol=1e-15)


def test_cells_gradient_vs_central_fd():
    G, stacks = _case(4)
    cells = dict(grid_res=16, block_radius=2, centre=(0.0, 0.0, 0.0), half=16.0)
    rec = orc.records(G, stacks, cells=cells)
    rng = np.random.default_rng(4)
    gout = rng.normal(size=sum(s.n_vox for s in stacks))
    gr = orc.grad(G, stacks, rec, gout, cells)

    def g64():
        return types.SimpleNamespace(mean=np.asarray(G.mean, np.float64).copy(),
                                     quat=np.asarray(G.quat, np.float64).copy(),
                                     scale=np.asarray(G.scale, np.float64).copy(),
                                     alpha=np.asarray(G.alpha, np.float64).copy())

    def loss(Gx):
        return float(gout @ orc.render(Gx, stacks, rec, cells=cells))

    for name, width in (("mean", 3), ("quat", 4), ("scale", 3), ("alpha", 1)):
        for _ in range(4):
            g, c = int(rng.integers(G.n)), int(rng.integers(width))
            idx = (g, c) if width > 1 else (g,)
            Gp, Gm = g64(), g64()
            base = float(getattr(Gp, name)[idx])
            hh = 1e-7 * max(1.0, abs(base))   # small: the member sets follow the FP32 mean
            getattr(Gp, name)[idx] = base + hh
            getattr(Gm, name)[idx] = base - hh
            fd = (loss(Gp) - loss(Gm)) / (2 * hh)
            an = float(gr[name][idx])
            scale = max(abs(fd), 1e-3 * float(np.abs(gr[name]).max()))
            assert abs(fd - an) <= 1e-5 * scale, (name, idx, fd, an)
