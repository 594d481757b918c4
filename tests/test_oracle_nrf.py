"""Pins of the FP64 neural residual field reference (Sec. 3.4)."""
import numpy as np
import pytest

import mg_synth as ms
from oracle import nrf


def _params(preset, seed, **kw):
    W, b, t = ms.nrf_init(preset, seed, **kw)
    spec = nrf.GridSpec(**ms.NRF_GRID) if preset == "grid" else nrf.GridSpec()
    if preset == "grid" and "grid" in kw:
        spec = nrf.GridSpec(**dict(ms.NRF_GRID, **kw["grid"]))
    return nrf.NRFParams(preset, [w.astype(np.float64) for w in W], [x.astype(np.float64) for x in b],
                         None if t is None else t.astype(np.float64), spec)


def test_fourier_encoding_at_known_angles():
    """x = 1/4: the bands see angles pi/4, pi/2, pi, 2pi, 4pi, 8pi."""
    x = np.array([[0.25, 0.0, -0.5]])
    e = nrf.fourier_encode(x)[0]
    assert e.shape == (39,)
    assert np.allclose(e[:3], [0.25, 0.0, -0.5])
    # band j at offset 3 + 6j: sin(x0..x2), then cos(x0..x2)
    exp_sin0 = [np.sqrt(0.5), 1.0, 0.0, 0.0, 0.0, 0.0]
    exp_cos0 = [np.sqrt(0.5), 0.0, -1.0, 1.0, 1.0, 1.0]
    for j in range(6):
        assert abs(e[3 + 6 * j + 0] - exp_sin0[j]) < 1e-12
        assert abs(e[3 + 6 * j + 3] - exp_cos0[j]) < 1e-12
        assert abs(e[3 + 6 * j + 1]) < 1e-12 and abs(e[3 + 6 * j + 4] - 1.0) < 1e-12  # x1 = 0
    # x2 = -1/2: sin(-pi/2) = -1 at j = 0, cos(-pi) = -1 at j = 1
    assert abs(e[3 + 2] + 1.0) < 1e-12 and abs(e[3 + 6 + 5] + 1.0) < 1e-12


def test_grid_levels_and_dense_linear_reproduction():
    spec = nrf.GridSpec(levels=4, feats=2, log2_table=14, n_min=4, n_max=32)
    res = spec.resolutions()
    assert res[0] == 4 and res[-1] == 32
    # a table holding a linear function of the (dense) vertex coordinates is
    # reproduced exactly by trilinear interpolation at any point
    rng = np.random.default_rng(0)
    table = np.zeros((4, spec.table_size, 2))
    a = rng.normal(size=(2, 3))
    c0 = rng.normal(size=2)
    for l, N in enumerate(res):
        if (N + 1) ** 3 > spec.table_size:
            continue
        for idx in range((N + 1) ** 3):
            v = np.array([idx % (N + 1), (idx // (N + 1)) % (N + 1), idx // (N + 1) ** 2]) / N
            table[l, idx] = a @ v + c0
    x = rng.uniform(-1, 1, size=(50, 3))
    enc = nrf.grid_encode(x, table, spec)
    p = (x + 1) / 2
    for l, N in enumerate(res):
        if (N + 1) ** 3 > spec.table_size:
            continue
        assert np.allclose(enc[:, 2 * l:2 * l + 2], p @ a.T + c0, atol=1e-12)


def test_grid_hash_axis_vertices():
    """Hashed levels: vertex (1,0,0) -> 1, (0,1,0) -> 2654435761 mod T, (0,0,1) -> 805459861 mod T."""
    spec = nrf.GridSpec(levels=2, feats=1, log2_table=10, n_min=64, n_max=128)
    T = spec.table_size
    N = spec.resolutions()[0]
    # query points exactly on vertices (f = 0 -> all weight on corner 0)
    for v, want in (((1, 0, 0), 1 % T), ((0, 1, 0), 2654435761 % T), ((0, 0, 1), 805459861 % T), ((0, 0, 0), 0)):
        x = np.array([[2.0 * v[0] / N - 1, 2.0 * v[1] / N - 1, 2.0 * v[2] / N - 1]])
        (idx, w), _ = nrf._grid_corners(x, spec)
        assert idx[0, 0] == want and abs(w[0, 0] - 1.0) < 1e-12


@pytest.mark.parametrize("preset", ["paper", "grid"])
def test_bound_and_zero_weights(preset):
    kw = {"grid": dict(log2_table=12, n_max=64), "table_range": 1.0} if preset == "grid" else {}
    P = _params(preset, 1, last_gain=50.0, **kw)
    x = ms.nrf_points(200, 2).astype(np.float64)
    r = nrf.forward(P, x)
    assert np.all(np.abs(r) <= 0.1) and np.abs(r).max() > 0.09
    P.weights[-1][:] = 0
    P.biases[-1][:] = 0
    assert np.all(nrf.forward(P, x) == 0.0)


@pytest.mark.parametrize("preset", ["paper", "grid"])
def test_backward_vs_central_fd(preset):
    kw = {"grid": dict(log2_table=12, n_max=64), "table_range": 0.5} if preset == "grid" else {}
    P = _params(preset, 3, **kw)
    x = ms.nrf_points(64, 4).astype(np.float64)
    rng = np.random.default_rng(5)
    go = rng.normal(size=64)
    g = nrf.backward(P, x, go)

    def L():
        return float(np.dot(go, nrf.forward(P, x)))

    h = 1e-6
    for l in range(len(P.weights)):
        for _ in range(4):
            i, j = rng.integers(P.weights[l].shape[0]), rng.integers(P.weights[l].shape[1])
            w0 = P.weights[l][i, j]
            P.weights[l][i, j] = w0 + h
            lp = L()
            P.weights[l][i, j] = w0 - h
            lm = L()
            P.weights[l][i, j] = w0
            assert abs((lp - lm) / (2 * h) - g["weights"][l][i, j]) <= 1e-6 * max(1.0, abs(g["weights"][l][i, j]))
        i = rng.integers(P.biases[l].shape[0])
        b0 = P.biases[l][i]
        P.biases[l][i] = b0 + h
        lp = L()
        P.biases[l][i] = b0 - h
        lm = L()
        P.biases[l][i] = b0
        assert abs((lp - lm) / (2 * h) - g["biases"][l][i]) <= 1e-6 * max(1.0, abs(g["biases"][l][i]))
    if preset == "grid":
        nz = np.argwhere(np.abs(g["table"]) > 1e-8)
        for t in nz[rng.choice(len(nz), 6, replace=False)]:
            t = tuple(t)
            v0 = P.table[t]
            P.table[t] = v0 + h
            lp = L()
            P.table[t] = v0 - h
            lm = L()
            P.table[t] = v0
            assert abs((lp - lm) / (2 * h) - g["table"][t]) <= 1e-6 * max(1.0, abs(g["table"][t]))
