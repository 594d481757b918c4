"""Pin of the oracle's analytic FP64 gradient: central finite differences of
the FP64 binned render with the records held fixed (the sum is piecewise
constant in the record set, so this is exactly what the adjoint
differentiates)."""
import types

import numpy as np
import pytest

import mg_synth as ms
import oracle as orc


def _g64(G):
    return types.SimpleNamespace(mean=G.mean.astype(np.float64).copy(), quat=G.quat.astype(np.float64).copy(),
                                 scale=G.scale.astype(np.float64).copy(), alpha=G.alpha.astype(np.float64).copy())


@pytest.mark.parametrize("seed", [0, 1])
def test_grad_vs_central_fd(seed):
    G = ms.random_gaussians(25, 70 + seed, box=(-9, 9), sigma=(0.8, 2.5), aniso=3.0, alpha=(-1.0, 1.0))
    rng = np.random.default_rng(seed)
    stacks = [ms.make_stack(ms.AXIAL, 4, 20, 22, 1.0, 1.1, 3.0, 3.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 3, 18, 16, 0.9, 1.0, 2.0, 2.5, rng=rng,
                            max_rot_deg=3.0, max_trans_mm=1.0)]
    rec = orc.records(G, stacks, 3.0)
    assert rec.n > 20
    gout = rng.normal(size=sum(s.n_vox for s in stacks))
    gr = orc.grad(G, stacks, rec, gout)
    G64 = _g64(G)

    def loss(Gx):
        return float(np.dot(gout, orc.render(Gx, stacks, rec)))

    for name, width in (("mean", 3), ("quat", 4), ("scale", 3), ("alpha", 1)):
        for _ in range(6):
            g = int(rng.integers(G.n))
            c = int(rng.integers(width))
            idx = (g, c) if width > 1 else (g,)
            base = float(getattr(G64, name)[idx])
            h = 1e-6 * max(1.0, abs(base))
            Gp, Gm = _g64(G), _g64(G)
            getattr(Gp, name)[idx] = base + h
            getattr(Gm, name)[idx] = base - h
            fd = (loss(Gp) - loss(Gm)) / (2 * h)
            an = float(gr[name][idx])
            scale = max(abs(fd), 1e-3 * float(np.abs(gr[name]).max()))
            assert abs(fd - an) <= 1e-6 * scale, (name, idx, fd, an)
