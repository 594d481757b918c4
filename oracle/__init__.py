"""CPU reference ("oracle") for the Magnetic Gaussian slice renderer.

TEST INFRASTRUCTURE ONLY. Imported by ``tests/``, by ``__graft_entry__.smoke()``
and by ``bench.py``'s CPU-baseline leg; the product path never imports it and
shares no code with it. It is plain and slow on purpose:

* ``mg_oracle.c`` (plain C, built with ``-ffp-contract=off``): the FP32 record
  predicate as written in its header, and FP64 evaluation of each Gaussian's
  slice-profile integral from the 3x3 profile-convolved covariance (Sec. 3.2
  Eq. E3, Sec. 3.3.2 Eq. E7 with a Gaussian slice profile), the analytic FP64
  gradient, and ellipsoid pair counts.
* ``nrf.py``: the neural residual field (Sec. 3.4, Eq. E8) in FP64 numpy.
* ``metrics.py``: losses (Sec. 3.5.2) and PSNR in FP64 numpy.

Parity status of each function is stated in its docstring; the pins live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libmgoracle.so")
TILE = 8
FWHM2VAR = 0.18033688011112042  # 1 / (8 ln 2)


def build(force: bool = False) -> str:
    """Compile ``mg_oracle.c`` with gcc (FP32 predicate needs -ffp-contract=off)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.or_make_records.restype = i64
        L.or_make_records.argtypes = [i64, p, p, p, ctypes.c_int, p, p, p, p, p, p, p, p, ctypes.c_float, i64, p, p,
                                      p, p]
        L.or_render.restype = None
        L.or_render.argtypes = [i64, p, p, p, p, ctypes.c_int, p, p, p, p, p, p, p, p, i64, p, p, p, p, ctypes.c_int,
                                p, p, p]
        L.or_grad.restype = None
        L.or_grad.argtypes = [i64, p, p, p, p, ctypes.c_int, p, p, p, p, p, p, p, p, i64, p, p, p, p, p, p, p, p,
                              p, p, p]
        L.or_make_records_cells.restype = i64
        L.or_make_records_cells.argtypes = [i64, p, ctypes.c_int, p, p, p, p, p, p, p, p, p, p, i64, p, p, p]
        L.or_pair_counts.restype = None
        L.or_pair_counts.argtypes = [i64, p, p, p, p, ctypes.c_int, p, p, p, p, p, p, p, p, i64, p, p, p, p,
                                     ctypes.c_double, p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _StackArgs:
    """Flat per-stack arrays for the C calls (kept alive while in use). The
    record predicate takes FP32 geometry, the FP64 evaluation takes FP64
    geometry (the FP32 inputs converted exactly, or FP64 inputs as given)."""

    def __init__(self, stacks, dtype=np.float32):
        self.n = len(stacks)
        self.nsl = np.array([s.n_slices for s in stacks], dtype=np.int32)
        self.H = np.array([s.H for s in stacks], dtype=np.int32)
        self.W = np.array([s.W for s in stacks], dtype=np.int32)
        self.dx = np.array([s.dx for s in stacks], dtype=dtype)
        self.dy = np.array([s.dy for s in stacks], dtype=dtype)
        self.thk = np.array([s.thickness for s in stacks], dtype=dtype)
        self.psf = np.array([[getattr(s, "psf_u", 0.0), getattr(s, "psf_v", 0.0)] for s in stacks],
                            dtype=dtype).reshape(-1)
        self.xf = np.ascontiguousarray(np.concatenate([np.asarray(s.xform).reshape(-1, 12) for s in stacks])
                                       .astype(dtype))

    def args(self):
        return [self.n, _ptr(self.nsl), _ptr(self.H), _ptr(self.W), _ptr(self.dx), _ptr(self.dy), _ptr(self.thk),
                _ptr(self.psf), _ptr(self.xf)]


def _cells_args(cells):
    """(int32 [res, radius], float32 [cx, cy, cz, half]) of the cell-grid local set, kept alive by the caller."""
    if cells is None:
        return None, None
    ci = np.array([int(cells["grid_res"]), int(cells["block_radius"])], dtype=np.int32)
    cf = np.array([*[float(np.float32(v)) for v in cells["centre"]], float(np.float32(cells["half"]))],
                  dtype=np.float32)
    return ci, cf


def _gargs(G, dtype=np.float32):
    arrs = [np.ascontiguousarray(a, dtype=dtype) for a in (G.mean, G.quat, G.scale, G.alpha)]
    return arrs, [int(arrs[0].shape[0])] + [_ptr(a) for a in arrs]


@dataclass
class Records:
    """(Gaussian, slice) records, slice-major then ascending Gaussian id."""
    slice: np.ndarray   # [m] int32 global slice index
    gid: np.ndarray     # [m] int32
    rect: np.ndarray    # [m,4] int32 tile rectangle tx0, ty0, tx1, ty1 (inclusive)
    inset: np.ndarray | None = None  # [m] uint64 row insets of the rectangle (None: no culling)

    @property
    def n(self):
        return int(self.slice.shape[0])

    def _args(self):
        if self.inset is not None:
            self.inset = np.ascontiguousarray(self.inset, dtype=np.uint64)
        return [self.n, _ptr(self.slice), _ptr(self.gid), _ptr(self.rect),
                None if self.inset is None else _ptr(self.inset)]

    def row_tiles(self, r: int):
        """The (tx, ty) tiles record r lists: its rectangle, each of the first
        eight tile rows narrowed by the insets (low 4 bits from the left, high
        4 bits from the right)."""
        tx0, ty0, tx1, ty1 = (int(v) for v in self.rect[r])
        ins = 0 if self.inset is None else int(self.inset[r])
        out = []
        for ty in range(ty0, ty1 + 1):
            n = ty - ty0
            b = (ins >> (8 * n)) & 0xFF if n < 8 else 0
            out.extend((tx, ty) for tx in range(tx0 + (b & 15), tx1 - (b >> 4) + 1))
        return out


def records(G, stacks, K: float = 3.0, cells=None) -> Records:
    """Records by the FP32 record predicate (bit-exact specification): the
    K-sigma slab and cut-ellipse rule, or with ``cells`` (dict grid_res,
    block_radius, centre, half) the paper's cell-grid rule (Eqs. E4-E6),
    whose records bound the member voxels. Parity: pinned by brute-force
    conservativeness/tightness tests and, for cells, a brute-force member sum."""
    L = lib()
    sa = _StackArgs(stacks)
    keep, ga = _gargs(G)
    if cells is not None:
        ci, cf = _cells_args(cells)
        a = sa.args()
        total = L.or_make_records_cells(ga[0], ga[1], *a, _ptr(ci), _ptr(cf), 0, None, None, None)
        sl = np.zeros(total, dtype=np.int32)
        gid = np.zeros(total, dtype=np.int32)
        rect = np.zeros((total, 4), dtype=np.int32)
        L.or_make_records_cells(ga[0], ga[1], *a, _ptr(ci), _ptr(cf), total, _ptr(sl), _ptr(gid), _ptr(rect))
        return Records(sl, gid, rect, np.zeros(total, dtype=np.uint64))  # no row culling for cells
    total = L.or_make_records(*ga[:4], *sa.args(), ctypes.c_float(K), 0, None, None, None, None)
    sl = np.zeros(total, dtype=np.int32)
    gid = np.zeros(total, dtype=np.int32)
    rect = np.zeros((total, 4), dtype=np.int32)
    inset = np.zeros(total, dtype=np.uint64)
    L.or_make_records(*ga[:4], *sa.args(), ctypes.c_float(K), total, _ptr(sl), _ptr(gid), _ptr(rect), _ptr(inset))
    return Records(sl, gid, rect, inset)


def slice_table(stacks):
    """Per global slice: (stack index, H, W, TX, TY, output offset, first global tile)."""
    rows = []
    off = 0
    tile = 0
    for si, s in enumerate(stacks):
        TX = (s.W + TILE - 1) // TILE
        TY = (s.H + TILE - 1) // TILE
        for _ in range(s.n_slices):
            rows.append((si, s.H, s.W, TX, TY, off, tile))
            off += s.H * s.W
            tile += TX * TY
    return rows, tile


def tile_bins(rec: Records, stacks):
    """Per global tile (stacks, slices, then ty*TX+tx): the record count and the
    sorted record ids (CSR). Brute force over every record's listed tiles."""
    rows, n_tiles = slice_table(stacks)
    lists = [[] for _ in range(n_tiles)]
    for r in range(rec.n):
        k = int(rec.slice[r])
        _, _, _, TX, _, _, tb = rows[k]
        for tx, ty in rec.row_tiles(r):
            lists[tb + ty * TX + tx].append(r)
    counts = np.array([len(l) for l in lists], dtype=np.int64)
    offs = np.zeros(n_tiles + 1, dtype=np.int64)
    np.cumsum(counts, out=offs[1:])
    ids = np.array([r for l in lists for r in l], dtype=np.int64)
    return counts, offs, ids


def render(G, stacks, rec: Records | None = None, exact: bool = False, K: float = 3.0, cells=None) -> np.ndarray:
    """FP64 slice values, all stacks concatenated (flat). ``exact``: every
    Gaussian at every pixel (the untruncated sum S); otherwise the binned sum
    S^bin over ``rec``. Parity: pinned by quadrature, closed forms, mass
    conservation and rigid equivariance tests."""
    L = lib()
    sa = _StackArgs(stacks, np.float64)
    keep, ga = _gargs(G, np.float64)
    total = sum(s.n_vox for s in stacks)
    out = np.zeros(total, dtype=np.float64)
    if exact:
        dummy = Records(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros((0, 4), np.int32))
        rr = dummy
    else:
        rr = rec if rec is not None else records(G, stacks, K, cells)
    ci, cf = _cells_args(None if exact else cells)
    L.or_render(*ga, *sa.args(), *rr._args(), 1 if exact else 0, _ptr(out), None if ci is None else _ptr(ci),
                None if cf is None else _ptr(cf))
    return out


def split(flat: np.ndarray, stacks) -> List[np.ndarray]:
    """Split a flat concatenated slice array into per-stack [n_slices,H,W]."""
    out, o = [], 0
    for s in stacks:
        out.append(flat[o:o + s.n_vox].reshape(s.n_slices, s.H, s.W))
        o += s.n_vox
    return out


def grad(G, stacks, rec: Records, gout: np.ndarray, cells=None):
    """Analytic FP64 gradient of sum(gout * S^bin) with the records frozen.
    Returns dict mean[n,3], quat[n,4], scale[n,3], alpha[n]. Parity: pinned by
    central finite differences of ``render``."""
    L = lib()
    sa = _StackArgs(stacks, np.float64)
    keep, ga = _gargs(G, np.float64)
    go = np.ascontiguousarray(gout, dtype=np.float64).reshape(-1)
    n = int(np.asarray(G.mean).reshape(-1, 3).shape[0])
    gm = np.zeros((n, 3))
    gq = np.zeros((n, 4))
    gs = np.zeros((n, 3))
    gaa = np.zeros(n)
    ci, cf = _cells_args(cells)
    L.or_grad(*ga, *sa.args(), *rec._args(), _ptr(go), _ptr(gm), _ptr(gq), _ptr(gs), _ptr(gaa),
              None if ci is None else _ptr(ci), None if cf is None else _ptr(cf))
    return {"mean": gm, "quat": gq, "scale": gs, "alpha": gaa}


def pose_grad(G, stacks, rec: Records, gout: np.ndarray, cells=None) -> np.ndarray:
    """Gradient of sum(gout * S^bin) with respect to each slice pose, records
    frozen: [S, 6] = (dL/dt world, dL/domega) per slice, the rotation perturbed
    as R (I + [omega]x) with omega in the slice frame (columns of R).

    Moving a slice rigidly is the same, for that slice's values, as moving
    every Gaussian by the inverse motion about the slice centre: a shift by
    dt is mu -> mu - dt, a rotation R exp([omega]x) is mu -> t + W (mu - t)
    and q -> w (x) q with W = R exp(-[omega]x) R^T, whose unit quaternion is
    w = (1, -R omega / 2) to first order. So the pose gradient of slice k is
    the chain of the Gaussian gradients of that slice alone (``grad`` on the
    one-slice stack) through those motions. Expects unit quaternions.
    Parity: pinned by central finite differences of ``render`` in the slice
    transform (tests/test_oracle_pose.py)."""
    import types

    mu = np.asarray(G.mean, np.float64).reshape(-1, 3)
    q = np.asarray(G.quat, np.float64).reshape(-1, 4)
    go = np.asarray(gout, np.float64).reshape(-1)
    S = sum(int(s.n_slices) for s in stacks)
    out = np.zeros((S, 6))
    k = 0
    off = 0
    for s in stacks:
        xf_all = np.asarray(s.xform, np.float64).reshape(-1, 12)
        for j in range(int(s.n_slices)):
            xf = xf_all[j]
            npx = int(s.H) * int(s.W)
            sub = types.SimpleNamespace(n_slices=1, H=s.H, W=s.W, dx=s.dx, dy=s.dy, thickness=s.thickness,
                                        psf_u=getattr(s, "psf_u", 0.0), psf_v=getattr(s, "psf_v", 0.0),
                                        xform=xf[None, :].copy(), n_vox=npx)
            sel = rec.slice == k
            rk = Records(np.zeros(int(sel.sum()), np.int32), rec.gid[sel].copy(), rec.rect[sel].copy(),
                         None if rec.inset is None else rec.inset[sel].copy())
            gr = grad(G, [sub], rk, go[off:off + npx], cells)
            R = xf[:9].reshape(3, 3)
            t = xf[9:]
            gmu, gq = gr["mean"], gr["quat"]
            out[k, :3] = -gmu.sum(axis=0)
            d = (mu - t) @ R                      # d_i = R^T (mu_i - t), row-wise
            out[k, 3:] = np.cross(gmu @ R, d).sum(axis=0)
            qw, qv = q[:, 0], q[:, 1:]
            for a in range(3):
                v = -0.5 * R[:, a]                # vector part of the first-order quaternion of W
                dq_w = -(qv @ v)
                dq_v = qw[:, None] * v[None, :] + np.cross(np.broadcast_to(v, qv.shape), qv)
                out[k, 3 + a] += float((gq[:, 0] * dq_w).sum() + (gq[:, 1:] * dq_v).sum())
            k += 1
            off += npx
    return out


def pair_counts(G, stacks, rec: Records, K: float = 3.0):
    """(pairs inside the K-sigma ellipsoid of Sigma' in FP64, evaluated pairs)."""
    L = lib()
    sa = _StackArgs(stacks, np.float64)
    keep, ga = _gargs(G, np.float64)
    c = np.zeros(2, dtype=np.int64)
    L.or_pair_counts(*ga, *sa.args(), *rec._args(), ctypes.c_double(K), _ptr(c))
    return int(c[0]), int(c[1])


def volume_planes(G_dim: int, spacing: float, centre=(0.0, 0.0, 0.0)):
    """The isotropic target grid as G_dim z-planes of G_dim x G_dim voxels, no
    slice profile: voxel (c, j, i) sits at (cx + u_i, cy + v_j, z_c) with
    u_i = (i - (G-1)/2) h, v_j = (j - (G-1)/2) h and the plane height
    z_c = float32(cz + h (c - (G-1)/2)) evaluated in double; centre and h are
    taken as float32 values."""
    import types

    cx, cy, cz = (float(np.float32(v)) for v in centre)
    h = float(np.float32(spacing))
    xf = np.zeros((G_dim, 12), dtype=np.float64)
    for c in range(G_dim):
        xf[c, :9] = np.eye(3).reshape(-1)
        xf[c, 9:] = (cx, cy, float(np.float32(cz + h * (c - 0.5 * (G_dim - 1)))))
    return types.SimpleNamespace(n_slices=G_dim, H=G_dim, W=G_dim, dx=h, dy=h, thickness=0.0, xform=xf,
                                 n_vox=G_dim ** 3)


def sample_volume(G, G_dim: int, spacing: float, centre=(0.0, 0.0, 0.0), K: float = 3.0, exact: bool = False,
                  cells=None):
    """Inference sampling (Sec. 3.1, Fig. 1c): the Gaussian mixture of Eq. E7
    (no slice profile) on the isotropic grid, binned like the slices.
    Returns [G,G,G] (z,y,x) FP64."""
    st = volume_planes(G_dim, spacing, centre)
    return render(G, [st], None, exact=exact, K=K, cells=cells).reshape(G_dim, G_dim, G_dim)
