"""The adjoint behind torch.autograd (Sec. 3.1, differentiable rendering;
Sec. 3.2 parameterisation; Sec. 3.4 residual field).

``render_slices`` takes the paper's raw parameters (mean, unnormalised
quaternion, log-scale, alpha), normalises and exponentiates them in torch and
renders through ``RenderSlices`` (mg_render_fwd / mg_render_bwd); a scalar loss
and ``.backward()`` then give the raw parameters' gradients. They are checked

* against the oracle's analytic FP64 gradient (records frozen at the GPU's
  own FP32 inputs), chained by hand through q / |q| and exp(s), per group in
  relative L2 and element by element; and
* against central finite differences in FP64 of the oracle's binned render
  (records frozen) on 64 randomly chosen scalar parameters: relative L2 error
  over the 64 <= 1e-4, and each entry within 1e-4 of the largest gradient of
  its parameter group (the element-wise rule of the other gradient tests; a
  single entry's own relative error is not bounded, since with dL/dI of both
  signs one parameter's gradient can be a near-cancelling FP32 sum).

``NRFFunction`` (mg_nrf_fwd / mg_nrf_bwd, FP32 form) is checked the same way
against the FP64 oracle MLP, on a graph that reaches its parameters through
torch operations; points whose FP64 pre-activations lie within FP32 reach of
a ReLU kink are left out (``away_from_kinks``).
"""
import types

import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from gpu_util import away_from_kinks, rel_l2
from oracle import nrf as onrf

pytestmark = pytest.mark.gpu

N_FD = 64
TOL_FD = 1e-4


def _check_fd(got, fd, groups, what):
    """got, fd: [N_FD] gradients; groups: per entry the largest |gradient| of
    its parameter group. Returns (rel-L2, worst entry error / group max,
    median entry error / |fd|)."""
    got, fd = np.asarray(got, np.float64), np.asarray(fd, np.float64)
    err = np.abs(got - fd) / np.asarray(groups, np.float64)
    i = int(np.argmax(err))
    assert err[i] <= TOL_FD, f"{what}: FD entry {i}: got {got[i]:.6e} fd {fd[i]:.6e} err/group-max {err[i]:.2e}"
    r = rel_l2(got, fd)
    assert r <= TOL_FD, f"{what}: FD rel-L2 {r:.2e}"
    med = float(np.median(np.abs(got - fd) / np.maximum(np.abs(fd), 1e-300)))
    return r, float(err.max()), med


def _motion_case(seed):
    """An oblique stack with per-slice motion (rotation <= 3 deg, translation
    <= 1 mm), an orthogonal stack with an in-plane PSF, a zero-thickness stack;
    raw quaternions of random norm, log-scales, alpha of both signs, and a few
    needles on the FP64 geometry path."""
    rng = np.random.default_rng(seed)
    G = ms.random_gaussians(220, 700 + seed, box=(-16, 16), sigma=(0.6, 2.8), aniso=3.0, negative_frac=0.15)
    sc = G.scale.copy()
    sc[::23, 0] *= 140.0
    qraw = (G.quat * rng.uniform(0.4, 2.5, size=(G.n, 1))).astype(np.float32)
    logs = np.log(sc).astype(np.float32)
    stacks = [ms.make_stack(ms.axis_angle_matrix([1, 0, 0], np.deg2rad(30.0)) @ ms.AXIAL, 6, 34, 38, 1.0, 1.0,
                            2.0, 2.0, rng=rng, max_rot_deg=3.0, max_trans_mm=1.0),
              ms.make_stack(ms.CORONAL, 5, 30, 33, 1.1, 1.0, 3.0, 3.0, psf_u=1.2, psf_v=0.7),
              ms.make_stack(ms.SAGITTAL, 3, 25, 21, 1.3, 1.2, 0.0, 4.0)]
    return G.mean.copy(), qraw, logs, G.alpha.copy(), stacks


def _unit_and_scale64(qraw, logs):
    q = np.asarray(qraw, np.float64)
    return q / np.linalg.norm(q, axis=1, keepdims=True), np.exp(np.asarray(logs, np.float64))


@pytest.mark.parametrize("seed", [0, 1])
def test_render_slices_autograd_vs_oracle_and_fd(seed):
    from paper_2603_00145_b300 import SliceRenderer, render_slices

    mean, qraw, logs, alpha, stacks = _motion_case(seed)
    R = SliceRenderer(stacks)
    leaves = [torch.from_numpy(x).cuda().requires_grad_(True) for x in (mean, qraw, logs, alpha)]
    out = render_slices(R, *leaves)
    w = np.random.default_rng(50 + seed).normal(size=out.numel())
    loss = (out * torch.from_numpy(w.astype(np.float32)).cuda()).sum()
    loss.backward()
    got = {k: t.grad.detach().cpu().numpy().astype(np.float64) for k, t in zip(("mean", "qraw", "logs", "alpha"),
                                                                                leaves)}

    # the FP32 values the renderer saw: the records are frozen on exactly these
    with torch.no_grad():
        qn = leaves[1] / leaves[1].norm(dim=1, keepdim=True)
        sc = torch.exp(leaves[2])
    G32 = ms.Gaussians(mean, qn.cpu().numpy(), sc.cpu().numpy(), alpha)
    rec = orc.records(G32, stacks)
    assert R.stats()["records"] == rec.n

    # (1) the oracle's analytic gradient chained through q / |q| and exp(s)
    ref = orc.grad(G32, stacks, rec, w)
    q64, s64 = _unit_and_scale64(qraw, logs)
    nq = np.linalg.norm(np.asarray(qraw, np.float64), axis=1, keepdims=True)
    gq = ref["quat"]
    want = {"mean": ref["mean"], "qraw": (gq - q64 * np.sum(gq * q64, 1, keepdims=True)) / nq,
            "logs": ref["scale"] * s64, "alpha": ref["alpha"]}
    for k in want:
        r = rel_l2(got[k], want[k])
        e = float(np.abs(got[k] - want[k]).max()) / float(np.abs(want[k]).max())
        assert r <= 1e-4 and e <= 1e-4, (k, r, e)

    # (2) central finite differences in FP64 of the binned render, records frozen
    base = {"mean": np.asarray(mean, np.float64), "qraw": np.asarray(qraw, np.float64),
            "logs": np.asarray(logs, np.float64), "alpha": np.asarray(alpha, np.float64)}

    def L(p):
        q, s = _unit_and_scale64(p["qraw"], p["logs"])
        G = types.SimpleNamespace(mean=p["mean"], quat=q, scale=s, alpha=p["alpha"])
        return float(np.dot(w, orc.render(G, stacks, rec)))

    active = np.unique(rec.gid)
    rng = np.random.default_rng(90 + seed)
    names = ["mean", "qraw", "logs", "alpha"]
    g_sel, fd_sel, top = [], [], []
    for _ in range(N_FD):
        k = names[int(rng.integers(4))]
        g = int(rng.choice(active))
        idx = (g,) if k == "alpha" else (g, int(rng.integers(base[k].shape[1])))
        x0 = float(base[k][idx])
        h = 1e-6 * max(1.0, abs(x0))
        pp = {n: v.copy() for n, v in base.items()}
        pm = {n: v.copy() for n, v in base.items()}
        pp[k][idx] = x0 + h
        pm[k][idx] = x0 - h
        fd_sel.append((L(pp) - L(pm)) / (2 * h))
        g_sel.append(got[k][idx])
        top.append(float(np.abs(want[k]).max()))
    r, worst, med = _check_fd(g_sel, fd_sel, top, "render_slices")
    print(f"render_slices autograd vs FD ({N_FD} parameters): rel-L2 {r:.2e}, worst entry {worst:.2e} of its "
          f"group max, median entry {med:.2e} relative")


@pytest.mark.parametrize("preset", ["paper", "grid"])
def test_nrf_function_autograd_vs_oracle_and_fd(preset):
    from paper_2603_00145_b300 import NRF
    from paper_2603_00145_b300.ops import NRFFunction

    grid = dict(log2_table=12, n_min=4, n_max=48)
    kw = dict(grid=dict(grid), table_range=0.5) if preset == "grid" else {}
    W, b, t = ms.nrf_init(preset, 3, bf16=False, last_gain=4.0, **kw)
    spec = onrf.GridSpec(**dict(ms.NRF_GRID, **grid)) if preset == "grid" else onrf.GridSpec()
    gkw = dict(log2_table=grid["log2_table"], n_min=grid["n_min"], n_max=grid["n_max"]) if preset == "grid" else {}
    net = NRF(preset, "fp32", W, b, t, **gkw)
    ref = onrf.NRFParams(preset, [w_.astype(np.float64) for w_ in W], [b_.astype(np.float64) for b_ in b],
                         None if t is None else t.astype(np.float64), spec)
    x = away_from_kinks(ref, ms.nrf_points(3000 + 17, 21))
    n = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    # the parameters reach the field through torch operations (a scale and a
    # shift that autograd must chain through)
    p0 = net.params.detach().clone().requires_grad_(True)
    t0 = net.table.detach().clone().requires_grad_(True) if t is not None else None
    params = p0 * 1.0 + 0.0
    table = t0 * 1.0 if t0 is not None else None
    r = NRFFunction.apply(net, xd, params, table)
    wv = np.random.default_rng(22).normal(size=n)
    loss = (r * torch.from_numpy(wv.astype(np.float32)).cuda()).sum() + 0.5 * (r * r).sum()
    loss.backward()

    x64 = x.astype(np.float64)
    r64 = onrf.forward(ref, x64)
    assert rel_l2(r.detach().cpu().numpy(), r64) <= 1e-5
    gout = wv + r64                      # dL/dr of the loss above
    g = onrf.backward(ref, x64, gout)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in zip(g["weights"], g["biases"])])
    gp = p0.grad.detach().cpu().numpy().astype(np.float64)
    assert rel_l2(gp, flat) <= 1e-4
    assert float(np.abs(gp - flat).max()) <= 1e-4 * float(np.abs(flat).max())
    if t is not None:
        gt = t0.grad.detach().cpu().numpy().astype(np.float64).ravel()
        assert rel_l2(gt, g["table"].ravel()) <= 1e-4

    # central finite differences of the FP64 oracle loss on 64 scalar parameters
    def L(Wl, bl, tab):
        P = onrf.NRFParams(preset, Wl, bl, tab, spec)
        rr = onrf.forward(P, x64)
        return float(np.dot(wv, rr) + 0.5 * np.dot(rr, rr))

    Wl = [w_.astype(np.float64) for w_ in W]
    bl = [b_.astype(np.float64) for b_ in b]
    tab = None if t is None else t.astype(np.float64)
    rng = np.random.default_rng(23)
    offs = np.cumsum([0] + [w_.size + b_.size for w_, b_ in zip(W, b)])
    g_sel, fd_sel, top = [], [], []
    n_table = N_FD // 4 if t is not None else 0
    touched = np.flatnonzero(g["table"].ravel()) if t is not None else None
    for j in range(N_FD):
        h = 1e-6
        if j < n_table:
            i = int(rng.choice(touched))
            tp, tm = tab.copy().ravel(), tab.copy().ravel()
            tp[i] += h
            tm[i] -= h
            fd = (L(Wl, bl, tp.reshape(tab.shape)) - L(Wl, bl, tm.reshape(tab.shape))) / (2 * h)
            g_sel.append(gt[i])
            top.append(float(np.abs(g["table"]).max()))
        else:
            i = int(rng.integers(flat.size))
            li = int(np.searchsorted(offs, i, side="right") - 1)
            o = i - offs[li]
            Wp = [a.copy() for a in Wl]
            bp = [a.copy() for a in bl]
            Wm = [a.copy() for a in Wl]
            bm = [a.copy() for a in bl]
            if o < W[li].size:
                Wp[li].ravel()[o] += h
                Wm[li].ravel()[o] -= h
            else:
                bp[li][o - W[li].size] += h
                bm[li][o - W[li].size] -= h
            fd = (L(Wp, bp, tab) - L(Wm, bm, tab)) / (2 * h)
            g_sel.append(gp[i])
            top.append(float(np.abs(flat[offs[li]:offs[li + 1]]).max()))
        fd_sel.append(fd)
    r, worst, med = _check_fd(g_sel, fd_sel, top, f"NRFFunction {preset}")
    print(f"NRFFunction {preset} vs FD ({N_FD} parameters): rel-L2 {r:.2e}, worst entry {worst:.2e} of its "
          f"group max, median entry {med:.2e} relative")
