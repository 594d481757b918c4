"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on
seeded inputs and put the oracle beside it."""
import numpy as np
import torch

import mg_synth as ms

TOL_REL_L2 = 1e-5        # relative L2 of a rendered slice set vs the FP64 oracle
TOL_MAX_ABS = 1e-4       # maximum absolute error, as a fraction of the oracle's intensity range
TOL_GRAD_REL = 1e-4      # relative L2 of each gradient group vs the oracle's analytic FP64 gradient


def to_dev(G: ms.Gaussians, device="cuda"):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in (G.mean, G.quat, G.scale, G.alpha)]


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_render_close(got, want, what=""):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    rng = float(want.max() - want.min()) if want.size else 0.0
    r = rel_l2(got, want)
    m = float(np.max(np.abs(got - want))) if want.size else 0.0
    assert r <= TOL_REL_L2, f"{what}: rel-L2 {r:.3e} > {TOL_REL_L2}"
    assert m <= TOL_MAX_ABS * max(rng, 1e-30), f"{what}: max-abs {m:.3e} > {TOL_MAX_ABS} * range {rng:.3e}"
    return r, m


def tangent(gq, quat):
    """Remove the component of a quaternion gradient along the quaternion."""
    q = np.asarray(quat, np.float64)
    g = np.asarray(gq, np.float64)
    return g - (np.sum(g * q, axis=1) / np.sum(q * q, axis=1))[:, None] * q


def assert_grads_close(got, ref, G, what=""):
    """got: the library's (mean, quat, scale, alpha) gradients; ref: the
    oracle's dict. The quaternion gradient is compared on the tangent space."""
    out = {}
    for name, x in zip(("mean", "quat", "scale", "alpha"), got):
        x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
        want = ref[name]
        if name == "quat":
            want = tangent(want, G.quat)
        r = rel_l2(x, want)
        out[name] = r
        assert r <= TOL_GRAD_REL, f"{what}: grad {name} rel-L2 {r:.3e} > {TOL_GRAD_REL}"
    return out


def render_gpu(G: ms.Gaussians, stacks, K=3.0, f64_ratio=100.0, caps=None, renderer=None):
    from paper_2603_00145_b300 import SliceRenderer

    R = renderer or SliceRenderer(stacks, cutoff_k=K, f64_ratio=f64_ratio)
    if caps is not None:
        R.set_capacity(caps[0], caps[1], G.n)
    m, q, s, a = to_dev(G)
    out = R.forward(m, q, s, a)
    torch.cuda.synchronize()
    return R, out, (m, q, s, a)


def gpu_bins(R, n):
    """Records and bins read back from the renderer's workspace."""
    from paper_2603_00145_b300.ops import mg_render_ws_layout, read_bins

    st = R.stats()
    lay = mg_render_ws_layout(n, R.dev, R.opts())
    return st, read_bins(R.ws, lay, st["records"], R.dev.n_tiles, st["entries"])


def sub_stacks(stacks, picks):
    return ms.pick_slices(stacks, picks)
