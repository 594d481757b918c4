"""Pins of the oracle's FP32 record predicate (the K-sigma slab test plus the
tile rectangle of the cut ellipse) against brute force in FP64.

* conservativeness: every slice pixel inside the K-sigma ellipsoid of the
  profile-convolved covariance lies in a listed tile of that Gaussian's
  record for the slice;
* tightness: the tile rectangle equals the one obtained from the FP64 extents
  of the cut ellipse, found here by an eigen-decomposition of the in-plane
  quadratic form (a different route from the Schur complement the predicate
  uses), up to an FP32 margin;
* existence: a record exists exactly when the K-sigma slab test passes; its
  tile rectangle is empty when the cut ellipse misses the image;
* row culling: every tile holding a pixel inside the ellipse stays listed;
  each listed tile row of a rectangle wider than one tile reaches no further
  than the FP64 extent of the ellipse over that tile row's pixel band (dense
  boundary samples plus the band's chords) grown by the stated margin; and
  the listed tiles number within a few percent of the tiles that hold an
  inside pixel.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import mg_synth as ms
import oracle as orc

FWHM2VAR = 1.0 / (8.0 * np.log(2.0))
TILE = 8


def _plane_quadratic(mu, q, s, xf, psf_var):
    """q(u,v) = y^T Sigma'^-1 y for y = R_k (u,v,0) + t_k - mu as (A [2x2], b [2], c);
    Sigma' = Sigma + R_k diag(psf_var) R_k^T (in-plane PSF and slice profile)."""
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sg = R @ np.diag(np.asarray(s, np.float64) ** 2) @ R.T
    Rk = xf[:9].reshape(3, 3)
    P = np.linalg.inv(Sg + Rk @ np.diag(psf_var) @ Rk.T)
    B = Rk[:, :2]               # world = B (u,v) + t
    d0 = xf[9:] - mu            # y = B uv + d0
    A = B.T @ P @ B
    b = B.T @ P @ d0
    c = d0 @ P @ d0
    return A, b, c


def _fp64_tile_rect(A, b, c, K, st, margin_px):
    """Tile rectangle of the ellipse {uv : q(uv) <= K^2} from its FP64 extents,
    extents grown by ``margin_px`` pixels (negative shrinks). None if empty."""
    ctr = -np.linalg.solve(A, b)
    qmin = c + b @ ctr
    r2 = K * K - qmin
    if r2 < 0:
        return None
    w, V = np.linalg.eigh(A)
    th = np.linspace(0, 2 * np.pi, 4001)
    pts = ctr[:, None] + V @ (np.sqrt(r2 / w)[:, None] * np.stack([np.cos(th), np.sin(th)]))
    hx, hy = 0.5 * (st.W - 1), 0.5 * (st.H - 1)
    fx = pts[0] / st.dx + hx
    fy = pts[1] / st.dy + hy
    il, ih = np.ceil(fx.min() - margin_px), np.floor(fx.max() + margin_px)
    jl, jh = np.ceil(fy.min() - margin_px), np.floor(fy.max() + margin_px)
    if il > ih or jl > jh or il > st.W - 1 or ih < 0 or jl > st.H - 1 or jh < 0:
        return None
    il, jl = max(il, 0), max(jl, 0)
    ih, jh = min(ih, st.W - 1), min(jh, st.H - 1)
    return (int(il) // TILE, int(jl) // TILE, int(ih) // TILE, int(jh) // TILE)


def _row_extent(A, b, c, K, st, y0, y1):
    """FP64 pixel-x extent of {q <= K^2} over pixel rows y in [y0, y1]
    (continuous), or None: boundary samples inside the band plus the chords
    at its two edges."""
    ctr = -np.linalg.solve(A, b)
    r2 = K * K - (c + b @ ctr)
    if r2 <= 0:
        return None
    w, V = np.linalg.eigh(A)
    th = np.linspace(0, 2 * np.pi, 20001)
    pts = ctr[:, None] + V @ (np.sqrt(r2 / w)[:, None] * np.stack([np.cos(th), np.sin(th)]))
    hx, hy = 0.5 * (st.W - 1), 0.5 * (st.H - 1)
    fx, fy = pts[0] / st.dx + hx, pts[1] / st.dy + hy
    xs = list(fx[(fy >= y0) & (fy <= y1)])
    for yb in (y0, y1):
        v = (yb - hy) * st.dy  # chord: A00 du^2 + 2 A01 du dv + A11 dv^2 = r2, dv = v - ctr_v
        dv = v - ctr[1]
        disc = (A[0, 1] * dv) ** 2 - A[0, 0] * (A[1, 1] * dv * dv - r2)
        if disc >= 0:
            for sg in (-1.0, 1.0):
                du = (-A[0, 1] * dv + sg * np.sqrt(disc)) / A[0, 0]
                xs.append((ctr[0] + du) / st.dx + hx)
    if not xs:
        return None
    return min(xs), max(xs), np.sqrt(r2 / w).max()


def _contains(outer, inner):
    if inner is not None and (inner[0] > inner[2] or inner[1] > inner[3]):
        inner = None  # a record whose pixel box is empty lists no tile
    if outer is not None and (outer[0] > outer[2] or outer[1] > outer[3]):
        outer = None
    if inner is None:
        return True
    if outer is None:
        return False
    return outer[0] <= inner[0] and outer[1] <= inner[1] and outer[2] >= inner[2] and outer[3] >= inner[3]


@pytest.mark.parametrize("seed,K", [(0, 3.0), (1, 3.0), (2, 2.0), (3, 4.5)])
def test_records_vs_brute_force(seed, K):
    rng = np.random.default_rng(seed)
    G = ms.random_gaussians(80, 50 + seed, box=(-26, 26), sigma=(0.6, 4.0), aniso=4.0)
    stacks = [ms.make_stack(ms.AXIAL, 5, 40, 37, 1.0, 1.2, 3.0, 2.5),
              ms.make_stack(ms.random_rotations(1, rng)[0], 4, 33, 50, 0.8, 0.9, 2.0, 3.0,
                            rng=rng, max_rot_deg=5.0, max_trans_mm=1.0, psf_u=1.6, psf_v=0.9),
              ms.make_stack(ms.SAGITTAL, 3, 20, 20, 1.5, 1.5, 0.0, 4.0)]
    rec = orc.records(G, stacks, K)
    have = {(int(k), int(g)): tuple(int(v) for v in r) for k, g, r in zip(rec.slice, rec.gid, rec.rect)}
    where = {(int(k), int(g)): r for r, (k, g) in enumerate(zip(rec.slice, rec.gid))}
    n_listed = n_ideal = 0
    # slice-major, ascending Gaussian id
    key = rec.slice.astype(np.int64) * G.n + rec.gid
    assert np.all(np.diff(key) > 0)
    k0 = 0
    for st in stacks:
        psf_var = np.array([st.psf_u ** 2, st.psf_v ** 2, st.thickness ** 2]) * FWHM2VAR
        ii, jj = np.meshgrid(np.arange(st.W), np.arange(st.H), indexing="xy")
        uv = np.stack([(ii - 0.5 * (st.W - 1)) * st.dx, (jj - 0.5 * (st.H - 1)) * st.dy], axis=-1)
        for k in range(st.n_slices):
            xf = st.xform[k].astype(np.float64)
            for g in range(G.n):
                q = G.quat[g].astype(np.float64)
                q /= np.linalg.norm(q)
                A, b, c = _plane_quadratic(G.mean[g].astype(np.float64), q, G.scale[g], xf, psf_var)
                qv = np.einsum("hwi,ij,hwj->hw", uv, A, uv) + 2 * uv @ b + c
                got = have.get((k0 + k, g))
                inside = qv <= K * K * (1 - 1e-5)
                if inside.any():
                    assert got is not None, (k, g)
                    jin, iin = np.nonzero(inside)
                    tx, ty = iin // TILE, jin // TILE
                    assert got[0] <= tx.min() and got[2] >= tx.max() and got[1] <= ty.min() and got[3] >= ty.max()
                if got is not None:
                    r = where[(k0 + k, g)]
                    listed = set(rec.row_tiles(r))
                    n_listed += len(listed)
                    # every tile with an inside pixel is listed
                    need = {(int(a), int(b_)) for a, b_ in zip(*np.nonzero(inside.T))}
                    need = {(a // TILE, b_ // TILE) for a, b_ in need}
                    n_ideal += len(need)
                    assert need <= listed, (k, g, sorted(need - listed))
                    # each culled row reaches no further than the FP64 extent over the tile band
                    ins = int(rec.inset[r])
                    for ty_ in range(got[1], got[3] + 1):
                        nrow = ty_ - got[1]
                        bits = (ins >> (8 * nrow)) & 0xFF if nrow < 8 else 0
                        if nrow >= 8 or (bits & 15) == 15 or (bits >> 4) == 15 or got[0] == got[2]:
                            continue  # rows the rule leaves unculled
                        row = sorted(tx_ for tx_, t_ in listed if t_ == ty_)
                        if not row:
                            continue
                        ext = _row_extent(A, b, c, K * (1 + 1e-5), st, TILE * ty_, min(TILE * ty_ + TILE - 1,
                                                                                         st.H - 1))
                        assert ext is not None, (k, g, ty_)
                        lo, hi, rmax = ext
                        m_px = (rmax / 256 + st.dx / 1024) / st.dx + 1e-3
                        assert TILE * row[0] + TILE - 1 >= np.ceil(lo - m_px), (k, g, ty_, row, lo)
                        assert TILE * row[-1] <= np.floor(hi + m_px), (k, g, ty_, row, hi)
                # slab test in FP64: w0^2 / Sww vs K^2 (margin for FP32 rounding)
                q_min = c - b @ np.linalg.solve(A, b)  # min over the plane of q
                # q_min is w0^2/Sww (the plane minimum of the convolved form)
                if q_min < K * K * (1 - 1e-5):
                    assert got is not None, ("slab record missing", k, g)
                elif q_min > K * K * (1 + 1e-5):
                    assert got is None, ("record outside the slab", k, g)
                lo = _fp64_tile_rect(A, b, c, K * (1 - 1e-5), st, -1e-3)
                hi = _fp64_tile_rect(A, b, c, K * (1 + 1e-5), st, 1e-3)
                assert _contains(got, lo), (k, g, got, lo)
                assert _contains(hi, got), (k, g, got, hi)
        k0 += st.n_slices
    # the culled lists are close to the ideal tile sets
    assert n_listed <= 1.03 * n_ideal + 5, (n_listed, n_ideal)
    assert int(np.count_nonzero(rec.inset)) > 0


def test_record_count_and_tile_bins_consistent():
    G = ms.random_gaussians(50, 9, box=(-15, 15), sigma=(0.8, 3.0), aniso=3.0)
    stacks = [ms.make_stack(ms.CORONAL, 6, 35, 48, 1.0, 1.0, 3.0, 3.0)]
    rec = orc.records(G, stacks, 3.0)
    counts, offs, ids = orc.tile_bins(rec, stacks)
    assert counts.sum() == sum(len(rec.row_tiles(r)) for r in range(rec.n)) == ids.size
    areas = (rec.rect[:, 2] - rec.rect[:, 0] + 1) * (rec.rect[:, 3] - rec.rect[:, 1] + 1)
    assert counts.sum() <= areas[areas > 0].sum()
    for t in range(counts.size):
        seg = ids[offs[t]:offs[t + 1]]
        assert np.all(np.diff(seg) > 0)


@pytest.mark.parametrize("seed,K", [(0, 3.0), (5, 2.5)])
def test_pair_counts_vs_brute_force(seed, K):
    """Pin of ``pair_counts`` (the metric's numerator P and the evaluated
    pairs): the inside count equals the number of (record, pixel) pairs with
    y^T Sigma'^-1 y <= K^2 found here over EVERY pixel of every slice by the
    scipy-rotation plane quadratic (another route than the oracle's 3x3
    inverse), up to the pixels in the 1e-5 boundary band; the evaluated count
    equals the pixels of the listed tiles, counted tile by tile with the image
    border clipping them."""
    rng = np.random.default_rng(100 + seed)
    G = ms.random_gaussians(60, 300 + seed, box=(-20, 20), sigma=(0.6, 3.5), aniso=4.0, negative_frac=0.2)
    stacks = [ms.make_stack(ms.AXIAL, 4, 37, 30, 1.0, 1.2, 3.0, 2.5),
              ms.make_stack(ms.random_rotations(1, rng)[0], 4, 29, 41, 0.8, 0.9, 2.0, 3.0,
                            rng=rng, max_rot_deg=5.0, max_trans_mm=1.0, psf_u=1.4, psf_v=0.7),
              ms.make_stack(ms.CORONAL, 3, 21, 19, 1.5, 1.5, 0.0, 4.0)]
    rec = orc.records(G, stacks, K)
    got_in, got_ev = orc.pair_counts(G, stacks, rec, K)
    where = {(int(k), int(g)): r for r, (k, g) in enumerate(zip(rec.slice, rec.gid))}
    lo = hi = ev = 0
    k0 = 0
    for st in stacks:
        psf_var = np.array([st.psf_u ** 2, st.psf_v ** 2, st.thickness ** 2]) * FWHM2VAR
        ii, jj = np.meshgrid(np.arange(st.W), np.arange(st.H), indexing="xy")
        uv = np.stack([(ii - 0.5 * (st.W - 1)) * st.dx, (jj - 0.5 * (st.H - 1)) * st.dy], axis=-1)
        for k in range(st.n_slices):
            xf = st.xform[k].astype(np.float64)
            for g in range(G.n):
                r = where.get((k0 + k, g))
                if r is None:
                    continue
                q = G.quat[g].astype(np.float64)
                q /= np.linalg.norm(q)
                A, b, c = _plane_quadratic(G.mean[g].astype(np.float64), q, G.scale[g], xf, psf_var)
                qv = np.einsum("hwi,ij,hwj->hw", uv, A, uv) + 2 * uv @ b + c
                lo += int(np.count_nonzero(qv <= K * K * (1 - 1e-5)))
                hi += int(np.count_nonzero(qv <= K * K * (1 + 1e-5)))
                for tx, ty in rec.row_tiles(r):
                    ev += min(TILE, st.W - TILE * tx) * min(TILE, st.H - TILE * ty)
        k0 += st.n_slices
    assert lo <= got_in <= hi, (lo, got_in, hi)
    assert hi - lo <= max(3, 1e-3 * lo)  # the band is thin: the count is pinned, not merely bracketed
    assert got_ev == ev, (got_ev, ev)
    assert 0 < got_in < got_ev
