"""GPU parity of the neural residual field (Sec. 3.4) against the FP64 oracle.

FP32 precision: forward within relative L2 1e-5, gradients within 1e-4, on
points away from the ReLU kinks of the grid preset (gpu_util.away_from_kinks).
BF16 precision: inputs of every layer are rounded to BF16 (relative error
2^-9 each) and the MLP runs on the tensor cores with FP32 accumulation; the
forward is compared with the oracle evaluated on the same BF16-rounded
activations (relative L2 2e-3: FP32 accumulation order and the approximate
tanh in SiLU), and its error against plain FP64 is bounded by the rounding
budget of 4-5 layers of BF16 activations (relative L2 3e-2).
"""
import numpy as np
import pytest
import torch

import mg_synth as ms
from gpu_util import away_from_kinks
from oracle import nrf as onrf

pytestmark = pytest.mark.gpu

GRID = dict(log2_table=14, n_min=4, n_max=96)


def _rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _nets(preset, precision, seed=0):
    from paper_2603_00145_b300 import NRF

    kw = dict(grid=dict(GRID), table_range=0.5) if preset == "grid" else {}
    W, b, t = ms.nrf_init(preset, seed, bf16=True, last_gain=4.0, **kw)
    spec = onrf.GridSpec(**dict(ms.NRF_GRID, **GRID)) if preset == "grid" else onrf.GridSpec()
    ref = onrf.NRFParams(preset, [w.astype(np.float64) for w in W], [x.astype(np.float64) for x in b],
                         None if t is None else t.astype(np.float64), spec)
    gkw = dict(log2_table=GRID["log2_table"], n_min=GRID["n_min"], n_max=GRID["n_max"]) if preset == "grid" else {}
    net = NRF(preset, precision, W, b, t, **gkw)
    return net, ref


def _points(n, seed):
    x = ms.nrf_points(n, seed)
    x[:8] = np.array([[-1, -1, -1], [1, 1, 1], [0, 0, 0], [1, -1, 0.5], [-1, 1, -0.25], [0.999, 0.5, -1],
                      [0.25, 0.75, -0.75], [-0.5, 0.0, 1.0]], dtype=np.float32)
    return x


def _bf16(a):
    return ms.round_to_bf16(np.asarray(a, np.float32)).astype(np.float64)


@pytest.mark.parametrize("preset", ["paper", "grid"])
def test_nrf_fp32_forward_backward(preset):
    from paper_2603_00145_b300 import mg_nrf_bwd, mg_nrf_fwd

    net, ref = _nets(preset, "fp32")
    x = away_from_kinks(ref, _points(4099, 1))  # ragged tail
    n = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(n, device="cuda")
    mg_nrf_fwd(net, xd, out)
    want = onrf.forward(ref, x.astype(np.float64))
    r = _rel(out.cpu().numpy(), want)
    assert r <= 1e-5, r
    assert np.abs(out.cpu().numpy()).max() <= 0.1
    go = np.random.default_rng(2).normal(size=n).astype(np.float32)
    gp = torch.empty_like(net.params)
    gt = torch.empty_like(net.table) if net.table is not None else None
    mg_nrf_bwd(net, xd, torch.from_numpy(go).cuda(), gp, gt)
    g = onrf.backward(ref, x.astype(np.float64), go.astype(np.float64))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in zip(g["weights"], g["biases"])])
    gpu = gp.cpu().numpy()
    o = 0
    for gw, gb in zip(g["weights"], g["biases"]):
        for part in (gw.ravel(), gb.ravel()):
            rr = _rel(gpu[o:o + part.size], part)
            assert rr <= 1e-4, (o, rr)
            o += part.size
    assert o == flat.size == gpu.size
    if preset == "grid":
        rr = _rel(gt.cpu().numpy().reshape(g["table"].shape), g["table"])
        assert rr <= 1e-4, rr


@pytest.mark.parametrize("preset", ["paper", "grid"])
def test_nrf_bf16_forward(preset):
    from paper_2603_00145_b300 import mg_nrf_fwd

    net, ref = _nets(preset, "bf16")
    n = 8192 + 45
    x = _points(n, 3)
    out = torch.empty(n, device="cuda")
    mg_nrf_fwd(net, torch.from_numpy(x).cuda(), out)
    got = out.cpu().numpy()
    emul = onrf.forward(ref, x.astype(np.float64), round_fn=_bf16)
    exact = onrf.forward(ref, x.astype(np.float64))
    r_emul, r_exact = _rel(got, emul), _rel(got, exact)
    print(f"{preset} bf16: rel-L2 vs BF16-activation oracle {r_emul:.2e}, vs FP64 {r_exact:.2e}")
    assert r_emul <= 2e-3, r_emul
    assert r_exact <= 3e-2, r_exact
    assert np.abs(got).max() <= 0.1


@pytest.mark.parametrize("preset", ["paper", "grid"])
def test_nrf_bf16_backward(preset):
    """BF16 gradients (deltas and activations stored in BF16): relative L2
    within 5e-2 of the FP64 gradient, direction within 0.999 cosine."""
    from paper_2603_00145_b300 import mg_nrf_bwd

    net, ref = _nets(preset, "bf16")
    n = 8192 + 45
    x = _points(n, 4)
    go = np.random.default_rng(5).normal(size=n).astype(np.float32)
    gp = torch.empty_like(net.params)
    gt = torch.empty_like(net.table) if net.table is not None else None
    mg_nrf_bwd(net, torch.from_numpy(x).cuda(), torch.from_numpy(go).cuda(), gp, gt)
    g = onrf.backward(ref, x.astype(np.float64), go.astype(np.float64))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in zip(g["weights"], g["biases"])])
    gpu = gp.cpu().numpy().astype(np.float64)
    r = _rel(gpu, flat)
    cos = float(gpu @ flat / (np.linalg.norm(gpu) * np.linalg.norm(flat)))
    print(f"{preset} bf16 grads: rel-L2 {r:.2e} cos {cos:.6f}")
    assert r <= 5e-2 and cos >= 0.999, (r, cos)
    if preset == "grid":
        # table cells sum few contributions of both signs under a random
        # dL/dr, which magnifies the BF16 rounding of the deltas; check the
        # direction here and the size under a one-signed dL/dr below
        gtn = gt.cpu().numpy().reshape(g["table"].shape).ravel()
        ct = float(gtn @ g["table"].ravel() / (np.linalg.norm(gtn) * np.linalg.norm(g["table"])))
        assert ct >= 0.998, ct
        go1 = (1.0 + 0.25 * np.random.default_rng(6).normal(size=n)).astype(np.float32)
        mg_nrf_bwd(net, torch.from_numpy(x).cuda(), torch.from_numpy(go1).cuda(), gp, gt)
        g1 = onrf.backward(ref, x.astype(np.float64), go1.astype(np.float64))
        rt = _rel(gt.cpu().numpy().reshape(g1["table"].shape), g1["table"])
        print(f"grid bf16 table grads (one-signed dL/dr): rel-L2 {rt:.2e}")
        assert rt <= 2e-2, rt


def test_nrf_zero_last_layer_gives_zero():
    from paper_2603_00145_b300 import NRF, mg_nrf_fwd

    W, b, _ = ms.nrf_init("paper", 7)
    W[-1][:] = 0
    b[-1][:] = 0
    for prec in ("bf16", "fp32"):
        net = NRF("paper", prec, W, b)
        out = torch.empty(1000, device="cuda")
        mg_nrf_fwd(net, torch.from_numpy(ms.nrf_points(1000, 1)).cuda(), out)
        assert float(out.abs().max()) == 0.0


def test_nrf_grid_table_alignment_checked():
    """An entry's two features are read as one 8-byte word, and two
    neighbouring table-gradient entries sharing a 16-byte word take one atomic:
    a table not 8-byte aligned or a table gradient not 16-byte aligned is
    refused before any launch (MG_ERR_INVALID_ARG); a table 8 bytes past a
    16-byte boundary works and gives the same result."""
    from paper_2603_00145_b300 import mg_nrf_bwd, mg_nrf_fwd
    from paper_2603_00145_b300._lib import MG_ERR_INVALID_ARG, MgError

    net, _ = _nets("grid", "fp32")
    m = net.table.numel()
    xyz = torch.from_numpy(_points(256, 3)).cuda()
    out = torch.empty(256, device="cuda")
    buf = torch.zeros(m + 4, device="cuda")
    with pytest.raises(MgError) as ei:
        mg_nrf_fwd(net, xyz, out, table=buf[1:1 + m])  # 4 bytes off
    assert ei.value.status == MG_ERR_INVALID_ARG
    gp = torch.empty(net.params.numel(), device="cuda")
    with pytest.raises(MgError) as ei:
        mg_nrf_bwd(net, xyz, torch.ones(256, device="cuda"), gp, buf[2:2 + m])  # 8 bytes off
    assert ei.value.status == MG_ERR_INVALID_ARG
    shifted = buf[2:2 + m]
    shifted.copy_(net.table.reshape(-1))
    ref = torch.empty(256, device="cuda")
    mg_nrf_fwd(net, xyz, ref)
    mg_nrf_fwd(net, xyz, out, table=shifted)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("preset", ["paper", "grid"])
def test_nrf_at_indexed_rows(preset):
    """The field at a batch of rows of a coordinate table (the training
    step's random voxel batch, Sec. 3.4): acc[idx[i]] += r(coords[idx[i]])
    with repeated rows adding, and the gradients of
    sum_i grad_acc[idx[i]] r(coords[idx[i]]), against the FP64 oracle on the
    gathered points (FP32 field: forward 1e-5, gradients 1e-4)."""
    from paper_2603_00145_b300 import mg_nrf_bwd_at, mg_nrf_fwd_at

    net, ref = _nets(preset, "fp32")
    coords = away_from_kinks(ref, _points(3001, 7))
    rows, n = coords.shape[0], 4099 + 512  # more indices than rows: repeats; ragged tail
    idx = np.random.default_rng(8).integers(0, rows, size=n).astype(np.int64)
    acc0 = np.random.default_rng(9).normal(size=rows).astype(np.float32)
    acc = torch.from_numpy(acc0.copy()).cuda()
    cd, idd = torch.from_numpy(coords).cuda(), torch.from_numpy(idx).cuda()
    mg_nrf_fwd_at(net, cd, idd, n, acc)
    r = onrf.forward(ref, coords[idx].astype(np.float64))
    want = acc0.astype(np.float64) + np.bincount(idx, weights=r, minlength=rows)
    got = acc.cpu().numpy().astype(np.float64)
    assert _rel(got - acc0, want - acc0) <= 1e-5
    # n = 0 and a prefix of the index list
    mg_nrf_fwd_at(net, cd, idd, 0, acc)
    assert np.array_equal(acc.cpu().numpy().astype(np.float64), got)
    acc2 = torch.zeros(rows, device="cuda")
    mg_nrf_fwd_at(net, cd, idd, 100, acc2)
    want2 = np.bincount(idx[:100], weights=r[:100], minlength=rows)
    assert _rel(acc2.cpu().numpy(), want2) <= 1e-5
    ga = np.random.default_rng(10).normal(size=rows).astype(np.float32)
    gp = torch.empty_like(net.params)
    gt = torch.empty_like(net.table) if net.table is not None else None
    mg_nrf_bwd_at(net, cd, idd, n, torch.from_numpy(ga).cuda(), gp, gt)
    g = onrf.backward(ref, coords[idx].astype(np.float64), ga[idx].astype(np.float64))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in zip(g["weights"], g["biases"])])
    assert _rel(gp.cpu().numpy(), flat) <= 1e-4
    if preset == "grid":
        assert _rel(gt.cpu().numpy().reshape(g["table"].shape), g["table"]) <= 1e-4
    # indices outside [0, rows) add nothing
    bad = idd[:64].clone()
    bad[::3] = -1
    bad[1::3] = rows
    acc3 = torch.zeros(rows, device="cuda")
    mg_nrf_fwd_at(net, cd, bad, 64, acc3)
    keep = np.arange(64) % 3 == 2
    want3 = np.bincount(idx[:64][keep], weights=r[:64][keep], minlength=rows)
    assert _rel(acc3.cpu().numpy(), want3) <= 1e-5
    with pytest.raises(ValueError):
        mg_nrf_fwd_at(net, cd, idd.to(torch.int32), n, acc)


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_nrf_encoding_cache(precision):
    """The training pair with the grid-encoding cache (mg_nrf.enc): the forward
    at rows stores each point's features, the backward at the same rows reads
    them instead of gathering the table. The field is bit-identical, the
    gradients equal the uncached ones up to the atomic summation order."""
    from paper_2603_00145_b300 import mg_nrf_bwd_at, mg_nrf_fwd_at

    net, ref = _nets("grid", precision)
    rows, n = 2500, 3000 + 7
    coords = torch.from_numpy(_points(rows, 11)).cuda()
    idx = torch.from_numpy(np.random.default_rng(12).integers(-3, rows + 3, size=n).astype(np.int64)).cuda()
    enc = net.enc_cache(n)
    assert enc is not None and enc.numel() == n * 32 * (2 if precision == "bf16" else 4)
    acc0, acc1 = torch.zeros(rows, device="cuda"), torch.zeros(rows, device="cuda")
    mg_nrf_fwd_at(net, coords, idx, n, acc0)
    mg_nrf_fwd_at(net, coords, idx, n, acc1, enc=enc)
    torch.cuda.synchronize()
    ga = torch.from_numpy(np.random.default_rng(13).normal(size=rows).astype(np.float32)).cuda()
    gp0, gp1 = torch.empty_like(net.params), torch.empty_like(net.params)
    gt0, gt1 = torch.empty_like(net.table), torch.empty_like(net.table)
    mg_nrf_bwd_at(net, coords, idx, n, ga, gp0, gt0)
    mg_nrf_bwd_at(net, coords, idx, n, ga, gp1, gt1, enc=enc)
    torch.cuda.synchronize()
    # the forward adds per point with atomics: compare per row within FP32 order
    assert _rel(acc1.cpu().numpy(), acc0.cpu().numpy()) <= 1e-6
    assert _rel(gp1.cpu().numpy(), gp0.cpu().numpy()) <= 1e-6
    assert _rel(gt1.cpu().numpy(), gt0.cpu().numpy()) <= 1e-6
    with pytest.raises(ValueError):
        mg_nrf_bwd_at(net, coords, idx, n, ga, gp1, gt1, enc=enc[:100])
