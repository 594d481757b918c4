"""FP64 reference of the neural residual field (NRF), Sec. 3.4 / Eq. E8.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's field: Fourier positional encoding with 6 frequency bands, 4
hidden layers of 64 SiLU units, output bounded by a scaled tanh to
[-0.1, 0.1]; I_final(x) = I(x) + r(x) (Sec. 3.4, Sec. 4.1.4).

Two presets are defined (the paper's and a multiresolution-grid variant):

* ``paper``: enc(x) = [x, sin(2^j pi x), cos(2^j pi x)], j = 0..5, laid out as
  x0 x1 x2, then per band j: sin(2^j pi x0..x2), cos(2^j pi x0..x2)  (39
  features) -> 4 x (64, SiLU) -> 1 -> 0.1 tanh. Including raw x and the base
  2^j pi are readings (the paper states neither).
* ``grid``: a 16-level multiresolution hash-grid encoding with 2 features per
  level (Mueller et al. 2022, "Instant neural graphics primitives"), restated
  here: level l has resolution N_l = floor(N_min * b^l), b = exp((ln N_max -
  ln N_min)/(L-1)); p = (x+1)/2 clamped to [0,1]; pos = p N_l; cell i0 =
  min(floor(pos), N_l - 1); f = pos - i0; the 8 corners v = i0 + c are looked
  up densely (v_x + v_y (N_l+1) + v_z (N_l+1)^2) when (N_l+1)^3 <= T, else by
  the spatial hash (v_x * 1 ^ v_y * 2654435761 ^ v_z * 805459861) mod 2^32 mod
  T; trilinear weights. 32 features -> 2 x (64, ReLU) -> 1 -> 0.1 tanh.

Parity: pinned by the tests (finite differences of this FP64 code, the
bound |r| <= 0.1, zero weights -> r = 0, the encoding at angles where sin/cos
are known exactly, and exact trilinear reproduction of linear fields).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

N_BANDS = 6
HASH_P1 = np.uint64(1)
HASH_P2 = np.uint64(2654435761)
HASH_P3 = np.uint64(805459861)


@dataclass
class GridSpec:
    levels: int = 16
    feats: int = 2
    log2_table: int = 19
    n_min: int = 16
    n_max: int = 512

    def resolutions(self) -> List[int]:
        b = np.exp((np.log(self.n_max) - np.log(self.n_min)) / (self.levels - 1))
        return [int(np.floor(self.n_min * b ** l)) for l in range(self.levels)]

    @property
    def table_size(self) -> int:
        return 1 << self.log2_table


# ---------------------------------------------------------------------------
# encodings
# ---------------------------------------------------------------------------


def fourier_encode(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    parts = [x]
    for j in range(N_BANDS):
        a = (2.0 ** j) * np.pi * x
        parts.append(np.sin(a))
        parts.append(np.cos(a))
    return np.concatenate(parts, axis=1)


def _grid_corners(x: np.ndarray, spec: GridSpec):
    """Per level: corner indices [n,8] and trilinear weights [n,8] (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    p = np.clip((x + 1.0) * 0.5, 0.0, 1.0)
    T = spec.table_size
    out = []
    for N in spec.resolutions():
        pos = p * N
        i0 = np.minimum(np.floor(pos), N - 1).astype(np.int64)
        f = pos - i0
        idx = np.zeros((x.shape[0], 8), dtype=np.int64)
        w = np.ones((x.shape[0], 8), dtype=np.float64)
        dense = (N + 1) ** 3 <= T
        for c in range(8):
            cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
            v = i0 + np.array([cx, cy, cz])
            if dense:
                idx[:, c] = v[:, 0] + v[:, 1] * (N + 1) + v[:, 2] * (N + 1) ** 2
            else:
                vu = v.astype(np.uint64)
                h = (vu[:, 0] * HASH_P1) ^ (vu[:, 1] * HASH_P2) ^ (vu[:, 2] * HASH_P3)
                h = h & np.uint64(0xFFFFFFFF)
                idx[:, c] = (h % np.uint64(T)).astype(np.int64)
            for d, cd in enumerate((cx, cy, cz)):
                w[:, c] *= f[:, d] if cd else (1.0 - f[:, d])
        out.append((idx, w))
    return out


def grid_encode(x: np.ndarray, table: np.ndarray, spec: GridSpec) -> np.ndarray:
    """table: [levels, T, feats]."""
    feats = []
    for l, (idx, w) in enumerate(_grid_corners(x, spec)):
        feats.append(np.einsum("nc,ncf->nf", w, table[l][idx]))
    return np.concatenate(feats, axis=1)


# ---------------------------------------------------------------------------
# MLP
# ---------------------------------------------------------------------------


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def relu(z):
    return np.maximum(z, 0.0)


def relu_grad(z):
    return (z > 0).astype(np.float64)


@dataclass
class NRFParams:
    preset: str                     # "paper" or "grid"
    weights: List[np.ndarray]       # W_l [out, in]
    biases: List[np.ndarray]        # b_l [out]
    table: np.ndarray | None = None  # grid preset: [levels, T, feats]
    spec: GridSpec = field(default_factory=GridSpec)
    out_scale: float = 0.1


def _act(preset):
    return (silu, silu_grad) if preset == "paper" else (relu, relu_grad)


def encode(P: NRFParams, x):
    return fourier_encode(x) if P.preset == "paper" else grid_encode(x, P.table, P.spec)


def forward(P: NRFParams, x, return_cache: bool = False, round_fn=None):
    """r(x) = out_scale * tanh(MLP(enc(x))) in FP64. Returns [n].
    ``round_fn`` (optional) is applied to the encoding and to every hidden
    activation, to model a lower-precision storage of activations."""
    act, _ = _act(P.preset)
    h = encode(P, x)
    if round_fn is not None:
        h = round_fn(h)
    cache = [h]
    zs = []
    nl = len(P.weights)
    for l in range(nl):
        W = np.asarray(P.weights[l], np.float64)
        b = np.asarray(P.biases[l], np.float64)
        z = h @ W.T + b
        zs.append(z)
        h = act(z) if l < nl - 1 else z
        if round_fn is not None and l < nl - 1:
            h = round_fn(h)
        cache.append(h)
    y = P.out_scale * np.tanh(h[:, 0])
    if return_cache:
        return y, (cache, zs)
    return y


def backward(P: NRFParams, x, grad_out):
    """Gradients of sum(grad_out * r(x)) w.r.t. weights, biases (and table)."""
    _, dact = _act(P.preset)
    y, (cache, zs) = forward(P, x, return_cache=True)
    nl = len(P.weights)
    g = np.asarray(grad_out, np.float64) * P.out_scale * (1.0 - np.tanh(cache[-1][:, 0]) ** 2)
    g = g[:, None]
    gW = [None] * nl
    gb = [None] * nl
    for l in range(nl - 1, -1, -1):
        if l < nl - 1:
            g = g * dact(zs[l])
        gW[l] = g.T @ cache[l]
        gb[l] = g.sum(axis=0)
        g = g @ np.asarray(P.weights[l], np.float64)
    out = {"weights": gW, "biases": gb}
    if P.preset == "grid":
        gt = np.zeros_like(np.asarray(P.table, np.float64))
        F = P.spec.feats
        for l, (idx, w) in enumerate(_grid_corners(x, P.spec)):
            gl = g[:, l * F:(l + 1) * F]
            for c in range(8):
                np.add.at(gt[l], idx[:, c], w[:, c:c + 1] * gl)
        out["table"] = gt
    return out


def layer_dims(preset: str) -> List[tuple]:
    if preset == "paper":
        return [(64, 3 + 6 * N_BANDS), (64, 64), (64, 64), (64, 64), (1, 64)]
    return [(64, 32), (64, 64), (1, 64)]
