"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on
seeded inputs and put the oracle beside it."""
import numpy as np
import torch

import mg_synth as ms

TOL_REL_L2 = 1e-5        # relative L2 of a rendered slice set vs the FP64 oracle
TOL_MAX_ABS = 1e-4       # maximum absolute error, as a fraction of the oracle's intensity range
TOL_GRAD_REL = 1e-4      # relative L2 of each gradient group vs the oracle's analytic FP64 gradient
TOL_GRAD_ELEM = 1e-4     # max |g - g_ref| of each group, as a fraction of max |g_ref| of that group


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
    oracle's dict. The quaternion gradient is compared on the tangent space.
    Each group must be within TOL_GRAD_REL in relative L2 and, element by
    element, within TOL_GRAD_ELEM of the group's largest reference magnitude
    (so a few badly wrong Gaussians cannot hide under the norm)."""
    out = {}
    for name, x in zip(("mean", "quat", "scale", "alpha"), got):
        x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
        want = ref[name]
        if name == "quat":
            want = tangent(want, G.quat)
        x = np.asarray(x, np.float64).reshape(np.shape(want))
        r = rel_l2(x, want)
        e = float(np.max(np.abs(x - want))) if x.size else 0.0
        top = float(np.max(np.abs(want))) if x.size else 0.0
        out[name] = r
        out[name + "_elem"] = e / top if top > 0 else e
        assert r <= TOL_GRAD_REL, f"{what}: grad {name} rel-L2 {r:.3e} > {TOL_GRAD_REL}"
        if e > TOL_GRAD_ELEM * top:
            i = int(np.argmax(np.abs(x - want)) // (x.size // max(len(x), 1)))
            sc = np.asarray(G.scale[i], np.float64)
            raise AssertionError(f"{what}: grad {name} max-abs {e:.3e} > {TOL_GRAD_ELEM} * max|ref| {top:.3e} "
                                 f"(Gaussian {i}: got {x[i]}, want {want[i]}, scale ratio {sc.max() / sc.min():.1f})")
    return out


def render_gpu(G: ms.Gaussians, stacks, K=3.0, f64_ratio=16.0, caps=None, renderer=None):
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


def away_from_kinks(ref, x, margin=1e-5):
    """The points of ``x`` [n,3] whose FP64 hidden pre-activations all lie
    further than ``margin`` (relative to the sum of the magnitudes that form
    them) from zero. The ReLU mask is an integer decision taken from a
    floating-point value: within FP32 reach of the kink the kernel (FP32) and
    the oracle (FP64) may legitimately take different branches, and one such
    point moves a whole gradient by a step, so parity is checked where both
    sides decide the same way (the decision is then the same in any
    precision). No-op for the smooth (SiLU) preset."""
    from oracle import nrf as onrf

    x = np.asarray(x, np.float32)
    if ref.preset != "grid":
        return x
    _, (cache, zs) = onrf.forward(ref, x.astype(np.float64), return_cache=True)
    keep = np.ones(x.shape[0], dtype=bool)
    for l, z in enumerate(zs[:-1]):
        W = np.abs(np.asarray(ref.weights[l], np.float64))
        scale = np.abs(cache[l]) @ W.T + np.abs(np.asarray(ref.biases[l], np.float64))
        keep &= np.all(np.abs(z) > margin * scale, axis=1)
    return np.ascontiguousarray(x[keep])
