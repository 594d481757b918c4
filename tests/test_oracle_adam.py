"""Pins of the oracle's Adam step (the optimiser of Sec. 4.1.4)."""
import numpy as np
import torch

from oracle.adam import Adam


def test_matches_torch_adam_float64():
    rng = np.random.default_rng(0)
    p0 = [rng.normal(size=(50, 3)), rng.normal(size=17)]
    lrs = [1e-3, 5e-2]
    ref = Adam(p0, lrs)
    tp = [torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in p0]
    opt = torch.optim.Adam([{"params": [tp[0]], "lr": lrs[0]}, {"params": [tp[1]], "lr": lrs[1]}])
    for _ in range(7):
        gs = [rng.normal(size=x.shape) for x in p0]
        ref.step(gs)
        for t, g in zip(tp, gs):
            t.grad = torch.tensor(g)
        opt.step()
    for a, t in zip(ref.p, tp):
        np.testing.assert_allclose(a, t.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_first_step_and_constant_gradient_closed_form():
    g = np.array([3.0, -0.5, 1e-3, -2e-2])
    lr, eps = 1e-2, 1e-8
    opt = Adam([np.zeros(4)], [lr], eps=eps)
    for t in range(1, 6):
        opt.step([g])
        # a constant gradient keeps m^ = g and v^ = g^2: every step moves by -lr g / (|g| + eps)
        np.testing.assert_allclose(opt.p[0], -t * lr * g / (np.abs(g) + eps), rtol=1e-12)


def test_clamp_and_skip():
    opt = Adam([np.array([0.999, 0.001, 0.5])], [0.1], clamps=[(0.0, 1.0)])
    opt.step([np.array([-1.0, 1.0, 0.0])])
    np.testing.assert_array_equal(opt.p[0][:2], [1.0, 0.0])
    assert opt.p[0][2] == 0.5
    before = [x.copy() for x in (opt.p[0], opt.m[0], opt.v[0])]
    opt.step([np.array([5.0, 5.0, 5.0])], skip=True)
    assert opt.t == 1
    for a, b in zip(before, (opt.p[0], opt.m[0], opt.v[0])):
        np.testing.assert_array_equal(a, b)
