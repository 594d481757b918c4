"""The fused Adam step (mg_adam_step) against the FP64 oracle, its status
predicate, and the device status word of a render whose bins overflow."""
import numpy as np
import pytest
import torch

import mg_synth as ms
from oracle.adam import Adam

pytestmark = pytest.mark.gpu


def _groups(rng, shapes):
    return [rng.normal(size=s).astype(np.float32) for s in shapes]


def test_adam_matches_oracle():
    from paper_2603_00145_b300 import ops

    rng = np.random.default_rng(1)
    shapes = [(1000, 3), (1001,), (37, 4), (4096,)]   # float4 and scalar paths
    lrs = [1e-3, 5e-2, 5e-3, 1e-2]
    clamps = [None, (0.0, 1.0), None, (-0.5, 0.5)]
    p0 = _groups(rng, shapes)
    ref = Adam(p0, lrs, clamps=clamps)
    dev = [torch.from_numpy(x.copy()).cuda() for x in p0]
    m = [torch.zeros_like(x) for x in dev]
    v = [torch.zeros_like(x) for x in dev]
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    for it in range(6):
        gs = _groups(rng, shapes)
        ref.step(gs)
        groups = [{"param": dev[k], "grad": torch.from_numpy(gs[k]).cuda(), "m": m[k], "v": v[k], "lr": lrs[k],
                   "clamp": clamps[k]} for k in range(len(shapes))]
        ops.mg_adam_step(groups, 0.9, 0.999, 1e-8, step)
    torch.cuda.synchronize()
    assert int(step.item()) == 6
    for k in range(len(shapes)):
        got = dev[k].cpu().numpy().astype(np.float64)
        moved = np.abs(ref.p[k] - p0[k]).max()
        err = np.abs(got - ref.p[k]).max()
        assert err <= 1e-5 * moved + 1e-6, (k, err, moved)
        np.testing.assert_allclose(m[k].cpu().numpy(), ref.m[k], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(v[k].cpu().numpy(), ref.v[k], rtol=1e-5, atol=1e-7)
        if clamps[k] is not None:
            assert got.min() >= clamps[k][0] and got.max() <= clamps[k][1]


def test_status_predicate_skips_everything():
    from paper_2603_00145_b300 import ops

    p = torch.ones(64, device="cuda")
    g = torch.full((64,), 0.5, device="cuda")
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    grp = [{"param": p, "grad": g, "m": m, "v": v, "lr": 0.1}]
    status.fill_(2)   # a capacity bit
    ops.mg_adam_step(grp, 0.9, 0.999, 1e-8, step, status)
    assert int(step.item()) == 0 and torch.all(p == 1) and torch.all(m == 0) and torch.all(v == 0)
    status.fill_(16)  # not a failure bit (FP64 geometry in use)
    ops.mg_adam_step(grp, 0.9, 0.999, 1e-8, step, status)
    assert int(step.item()) == 1
    torch.testing.assert_close(p, torch.full_like(p, 1 - 0.1 * 0.5 / (0.5 + 1e-8)))


def test_invalid_arguments():
    from paper_2603_00145_b300 import ops, _lib as L

    p = torch.ones(8, device="cuda")
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    grp = [{"param": p, "grad": p.clone(), "m": torch.zeros_like(p), "v": torch.zeros_like(p), "lr": 0.1}]
    with pytest.raises(L.MgError):
        ops.mg_adam_step(grp, 1.0, 0.999, 1e-8, step)
    with pytest.raises(L.MgError):
        ops.mg_adam_step(grp, 0.9, 0.999, 0.0, step)
    with pytest.raises(L.MgError):
        ops.mg_adam_step(grp * 9, 0.9, 0.999, 1e-8, step)
    assert int(step.item()) == 0 and torch.all(p == 1)


def test_render_status_word_flags_overflow():
    from paper_2603_00145_b300 import SliceRenderer, _lib as L
    from gpu_util import to_dev

    wl = ms.tiny_workload(0)
    G = ms.random_gaussians(500, 3, box=(-20, 20), sigma=(0.8, 2.5), aniso=3.0)
    m, q, s, a = to_dev(G)
    R = SliceRenderer(wl.stacks, check=True)
    R.forward(m, q, s, a)
    need = R.stats()
    assert need["status"] == 0 and int(R.status_word.view(torch.int32).item()) & L.MG_WS_FAIL_BITS == 0
    R.check = False
    R.set_capacity(need["records"] // 2, need["entries"], G.n)
    R.forward(m, q, s, a)
    torch.cuda.synchronize()
    assert int(R.status_word.view(torch.int32).item()) & 1          # records over capacity
    R.set_capacity(need["records"], need["entries"] // 2, G.n)
    R.forward(m, q, s, a)
    torch.cuda.synchronize()
    assert int(R.status_word.view(torch.int32).item()) & 2          # entries over capacity
