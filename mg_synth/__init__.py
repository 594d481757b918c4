"""Seeded synthetic inputs for the Magnetic Gaussian slice renderer.

This module is shared by the tests, the oracle side and the CUDA side. It holds
the input containers and the generators of seeded synthetic workloads: Gaussian
sets, stack geometries, ellipsoid phantoms, simulated thick-slice stacks. It
does NOT hold any arithmetic of the method itself (no Gaussian evaluation, no
slice-profile integral of a Gaussian, no binning): those live separately in the
oracle (CPU reference) and in the CUDA library.

Conventions (the same ones the C boundary documents):

* Gaussians: ``mean`` [n,3] world mm, ``quat`` [n,4] unit quaternion (w,x,y,z),
  ``scale`` [n,3] standard deviations in mm (> 0), ``alpha`` [n] intensity.
  All float32, C-contiguous.
* Stack: ``n_slices`` slices of ``H`` x ``W`` pixels at ``dx`` x ``dy`` mm, slice
  profile FWHM ``thickness`` mm (0 = point sampling). ``xform`` [n_slices,12]
  float32 = rotation R (3x3 row-major, columns e_u, e_v, e_n) then translation
  t: world = R (u, v, w)^T + t, the slice plane is w = 0. Pixel (i, j)
  (column i, row j) sits at u = (i - (W-1)/2) dx, v = (j - (H-1)/2) dy.
  Rendered slices are stored [n_slices, H, W].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------


@dataclass
class Gaussians:
    mean: np.ndarray   # [n,3] float32, mm
    quat: np.ndarray   # [n,4] float32, unit (w,x,y,z)
    scale: np.ndarray  # [n,3] float32, mm (std-dev along the principal axes)
    alpha: np.ndarray  # [n]   float32

    def __post_init__(self):
        self.mean = np.ascontiguousarray(self.mean, dtype=np.float32).reshape(-1, 3)
        self.quat = np.ascontiguousarray(self.quat, dtype=np.float32).reshape(-1, 4)
        self.scale = np.ascontiguousarray(self.scale, dtype=np.float32).reshape(-1, 3)
        self.alpha = np.ascontiguousarray(self.alpha, dtype=np.float32).reshape(-1)
        n = self.mean.shape[0]
        assert self.quat.shape[0] == n and self.scale.shape[0] == n and self.alpha.shape[0] == n

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def subset(self, idx) -> "Gaussians":
        return Gaussians(self.mean[idx], self.quat[idx], self.scale[idx], self.alpha[idx])

    def copy(self) -> "Gaussians":
        return Gaussians(self.mean.copy(), self.quat.copy(), self.scale.copy(), self.alpha.copy())


@dataclass
class Stack:
    n_slices: int
    H: int
    W: int
    dx: float
    dy: float
    thickness: float          # slice-profile FWHM in mm; 0 = point sampling
    xform: np.ndarray         # [n_slices,12] float32
    psf_u: float = 0.0        # in-plane PSF FWHM (mm) along e_u; 0 = none
    psf_v: float = 0.0        # in-plane PSF FWHM (mm) along e_v

    def __post_init__(self):
        self.xform = np.ascontiguousarray(self.xform, dtype=np.float32).reshape(self.n_slices, 12)

    @property
    def n_vox(self) -> int:
        return self.n_slices * self.H * self.W


def total_slices(stacks: Sequence[Stack]) -> int:
    return sum(s.n_slices for s in stacks)


def total_voxels(stacks: Sequence[Stack]) -> int:
    return sum(s.n_vox for s in stacks)


# --------------------------------------------------------------------------
# small geometry helpers (rotations used to lay out stacks and phantoms)
# --------------------------------------------------------------------------


def random_unit_quats(n: int, rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def axis_angle_matrix(axis, angle: float) -> np.ndarray:
    """Rodrigues rotation matrix (float64) about ``axis`` by ``angle`` radians."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def random_rotations(n: int, rng: np.random.Generator) -> np.ndarray:
    """Uniformly random rotation matrices [n,3,3] (float64) from the QR
    decomposition of Gaussian matrices (sign-fixed, det = +1); used only to
    orient phantom ellipsoids and stacks."""
    out = np.empty((n, 3, 3))
    for i in range(n):
        A = rng.normal(size=(3, 3))
        Qm, Rm = np.linalg.qr(A)
        Qm = Qm * np.sign(np.diag(Rm))
        if np.linalg.det(Qm) < 0:
            Qm[:, 0] *= -1
        out[i] = Qm
    return out


# orientation frames (columns e_u, e_v, e_n; right-handed) of the three
# orthogonal clinical stacks
AXIAL = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)      # n = +z
CORONAL = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], dtype=np.float64)   # u=x, v=z, n=-y
SAGITTAL = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], dtype=np.float64)   # u=y, v=z, n=x


def make_stack(frame: np.ndarray, n_slices: int, H: int, W: int, dx: float, dy: float,
               thickness: float, spacing: float, centre=(0.0, 0.0, 0.0),
               rng: np.random.Generator | None = None, max_rot_deg: float = 0.0,
               max_trans_mm: float = 0.0, psf_u: float = 0.0, psf_v: float = 0.0) -> Stack:
    """A stack of parallel slices along ``frame``'s third column, ``spacing`` mm apart,
    centred on ``centre``; optional per-slice rigid motion (random axis, angle up
    to ``max_rot_deg``; translation uniform in a ball of ``max_trans_mm``)."""
    frame = np.asarray(frame, dtype=np.float64)
    c = np.asarray(centre, dtype=np.float64)
    xf = np.zeros((n_slices, 12), dtype=np.float64)
    for k in range(n_slices):
        Rk = frame.copy()
        tk = c + (k - (n_slices - 1) / 2.0) * spacing * frame[:, 2]
        if rng is not None and (max_rot_deg > 0 or max_trans_mm > 0):
            ang = np.deg2rad(max_rot_deg) * rng.uniform(0, 1)
            M = axis_angle_matrix(rng.normal(size=3), ang)
            Rk = M @ Rk
            d = rng.normal(size=3)
            d *= max_trans_mm * rng.uniform(0, 1) ** (1 / 3) / np.linalg.norm(d)
            tk = tk + d
        xf[k, :9] = Rk.reshape(-1)
        xf[k, 9:] = tk
    return Stack(n_slices, H, W, float(dx), float(dy), float(thickness), xf.astype(np.float32), float(psf_u),
                 float(psf_v))


def volume_stack(G: int, spacing: float, centre=(0.0, 0.0, 0.0)) -> Stack:
    """The isotropic target grid seen as G axial z-planes of G x G voxels with no
    slice profile (used only to build inputs for tests)."""
    return make_stack(AXIAL, G, G, G, spacing, spacing, 0.0, spacing, centre)


# --------------------------------------------------------------------------
# Gaussian sets
# --------------------------------------------------------------------------


def random_gaussians(n: int, seed: int, box=(-20.0, 20.0), sigma=(0.8, 2.5),
                     aniso: float = 2.0, alpha=(0.2, 1.0), negative_frac: float = 0.0) -> Gaussians:
    """Random anisotropic Gaussians in a cube: means uniform in ``box`` (mm),
    random unit quaternions, per-axis std-devs log-uniform in ``sigma`` times an
    anisotropy factor up to ``aniso``, intensities uniform in ``alpha`` (a
    fraction ``negative_frac`` made negative)."""
    rng = np.random.default_rng(seed)
    mean = rng.uniform(box[0], box[1], size=(n, 3))
    quat = random_unit_quats(n, rng)
    base = np.exp(rng.uniform(np.log(sigma[0]), np.log(sigma[1]), size=(n, 1)))
    ratio = np.exp(rng.uniform(-np.log(aniso) / 2, np.log(aniso) / 2, size=(n, 3)))
    scale = base * ratio
    a = rng.uniform(alpha[0], alpha[1], size=n)
    if negative_frac > 0:
        neg = rng.uniform(size=n) < negative_frac
        a[neg] *= -1
    return Gaussians(mean.astype(np.float32), quat.astype(np.float32), scale.astype(np.float32),
                     a.astype(np.float32))


def grid_gaussians(res: int, fov_mm: float, seed: int, keep=None, sigma_factor: float = 1.0,
                   jitter: float = 0.0, alpha_fn=None, max_n: int | None = None) -> Gaussians:
    """Gaussians on a ``res``^3 grid spanning a cube of side ``fov_mm`` centred on
    the origin (the paper's low-resolution uniform initialisation), isotropic
    std-dev = spacing * ``sigma_factor``, identity rotation. ``keep(points)`` may
    drop background points; ``alpha_fn(points)`` sets intensities."""
    rng = np.random.default_rng(seed)
    h = fov_mm / res
    ax = (np.arange(res) - (res - 1) / 2.0) * h
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    if jitter > 0:
        pts = pts + rng.uniform(-jitter, jitter, size=pts.shape) * h
    if keep is not None:
        pts = pts[keep(pts)]
    if max_n is not None and pts.shape[0] > max_n:
        sel = np.sort(rng.choice(pts.shape[0], size=max_n, replace=False))
        pts = pts[sel]
    n = pts.shape[0]
    quat = np.zeros((n, 4))
    quat[:, 0] = 1.0
    scale = np.full((n, 3), h * sigma_factor)
    a = alpha_fn(pts) if alpha_fn is not None else np.full(n, 0.5)
    return Gaussians(pts.astype(np.float32), quat.astype(np.float32), scale.astype(np.float32),
                     np.asarray(a, dtype=np.float32))


# --------------------------------------------------------------------------
# ellipsoid phantoms (stand-ins for the fetal / adult brain volumes)
# --------------------------------------------------------------------------


@dataclass
class Phantom:
    centres: np.ndarray     # [m,3] mm
    axes: np.ndarray        # [m,3] semi-axes mm
    rots: np.ndarray        # [m,3,3]
    values: np.ndarray      # [m]
    mode: str = "paint"     # "paint": later ellipsoids overwrite; "sum": summed then clipped to [0,1]
    fov_mm: float = 48.0
    spacing: float = 1.0

    def evaluate(self, pts: np.ndarray) -> np.ndarray:
        """Phantom intensity at world points [p,3] (float64)."""
        pts = np.asarray(pts, dtype=np.float64)
        out = np.zeros(pts.shape[0])
        for c, a, R, v in zip(self.centres, self.axes, self.rots, self.values):
            loc = (pts - c) @ R  # coordinates in the ellipsoid frame
            inside = np.sum((loc / a) ** 2, axis=1) <= 1.0
            if self.mode == "sum":
                out[inside] += v
            else:
                out[inside] = v
        if self.mode == "sum":
            np.clip(out, 0.0, 1.0, out=out)
        return out

    def volume_torch(self, G: int | None = None, spacing: float | None = None, device: str = "cpu"):
        """Same as ``volume`` evaluated with torch on ``device`` (float32
        coordinates; returns a float32 tensor [z,y,x])."""
        import torch

        h = self.spacing if spacing is None else spacing
        G = int(round(self.fov_mm / h)) if G is None else G
        ax = (torch.arange(G, device=device, dtype=torch.float32) - (G - 1) / 2.0) * h
        out = torch.zeros(G, G, G, device=device, dtype=torch.float32)
        zz, yy, xx = torch.meshgrid(ax, ax, ax, indexing="ij")
        for c, a, R, v in zip(self.centres, self.axes, self.rots, self.values):
            Rt = torch.as_tensor(R, dtype=torch.float32, device=device)
            ct = torch.as_tensor(c, dtype=torch.float32, device=device)
            at = torch.as_tensor(a, dtype=torch.float32, device=device)
            d0, d1, d2 = xx - ct[0], yy - ct[1], zz - ct[2]
            r = torch.zeros_like(out)
            for j in range(3):  # coordinates in the ellipsoid frame: (x - c) @ R
                l = d0 * Rt[0, j] + d1 * Rt[1, j] + d2 * Rt[2, j]
                r += (l / at[j]) ** 2
            inside = r <= 1.0
            if self.mode == "sum":
                out += inside.to(out.dtype) * float(v)
            else:
                out = torch.where(inside, torch.full_like(out, float(v)), out)
        if self.mode == "sum":
            out.clamp_(0.0, 1.0)
        return out

    def volume(self, G: int | None = None, spacing: float | None = None) -> np.ndarray:
        """Phantom sampled at voxel centres of a G^3 grid centred on the origin,
        stored [z,y,x]."""
        h = self.spacing if spacing is None else spacing
        G = int(round(self.fov_mm / h)) if G is None else G
        ax = (np.arange(G) - (G - 1) / 2.0) * h
        zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
        pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
        return self.evaluate(pts).reshape(G, G, G)


def random_phantom(m: int, fov_mm: float, seed: int, values=(0.2, 1.0), nested: bool = False,
                   spacing: float = 1.0) -> Phantom:
    """``m`` random ellipsoids inside a cube of side ``fov_mm``. ``nested`` builds
    a brain-like layering: a large outer shell (CSF-like), a brain body, then
    progressively smaller structures (ventricles, nuclei) inside it, painted in
    that order."""
    rng = np.random.default_rng(seed)
    half = fov_mm / 2.0
    cs, ax, Rs, vs = [], [], [], []
    Rall = random_rotations(m, rng)
    for i in range(m):
        if nested:
            frac = i / max(m - 1, 1)
            size = half * (0.82 - 0.7 * frac) * rng.uniform(0.6, 1.0, size=3)
            size = np.maximum(size, 1.5)
            reach = max(half * 0.8 - size.max(), 0.0) * min(1.0, 0.2 + frac)
            c = rng.uniform(-reach, reach, size=3) * 0.6
        else:
            size = rng.uniform(0.08, 0.3, size=3) * fov_mm
            c = rng.uniform(-half * 0.55, half * 0.55, size=3)
        cs.append(c)
        ax.append(size)
        Rs.append(Rall[i])
        vs.append(rng.uniform(values[0], values[1]))
    return Phantom(np.array(cs), np.array(ax), np.array(Rs), np.array(vs),
                   mode="paint" if nested else "sum", fov_mm=fov_mm, spacing=spacing)


# --------------------------------------------------------------------------
# thick-slice stack simulation from a phantom volume (data generation)
# --------------------------------------------------------------------------


def slice_points(stack: Stack) -> np.ndarray:
    """World positions [n_slices,H,W,3] (float64) of the stack's pixel centres."""
    xf = stack.xform.astype(np.float64)
    i = np.arange(stack.W)
    j = np.arange(stack.H)
    u = (i - (stack.W - 1) / 2.0) * stack.dx
    v = (j - (stack.H - 1) / 2.0) * stack.dy
    vv, uu = np.meshgrid(v, u, indexing="ij")
    out = np.empty((stack.n_slices, stack.H, stack.W, 3))
    for k in range(stack.n_slices):
        R = xf[k, :9].reshape(3, 3)
        t = xf[k, 9:]
        out[k] = uu[..., None] * R[:, 0] + vv[..., None] * R[:, 1] + t
    return out


def simulate_stack(vol: np.ndarray, vol_spacing: float, stack: Stack, seed: int,
                   noise_sigma: float = 0.0, n_quad: int = 64, device: str = "cpu"):
    """Acquire ``stack`` from a phantom volume [z,y,x] centred on the origin: each
    pixel integrates the trilinearly interpolated volume along the slice normal
    against a unit-integral Gaussian profile of FWHM ``thickness`` (``n_quad``
    points over +-3 sigma), then Rician noise of level ``noise_sigma``.
    Returns float32 [n_slices,H,W] (torch tensor on ``device``)."""
    import torch
    import torch.nn.functional as F

    dev = torch.device(device)
    V = torch.as_tensor(vol, dtype=torch.float32, device=dev)[None, None]
    G = vol.shape[0]
    half_extent = (G - 1) / 2.0 * vol_spacing
    xf = torch.as_tensor(stack.xform, dtype=torch.float64, device=dev)
    sig = stack.thickness / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    if sig > 0:
        ts = np.linspace(-3 * sig, 3 * sig, n_quad)
        w = np.exp(-0.5 * (ts / sig) ** 2)
        w /= w.sum()
    else:
        ts, w = np.zeros(1), np.ones(1)
    i = torch.arange(stack.W, dtype=torch.float64, device=dev)
    j = torch.arange(stack.H, dtype=torch.float64, device=dev)
    u = (i - (stack.W - 1) / 2.0) * stack.dx
    v = (j - (stack.H - 1) / 2.0) * stack.dy
    vv, uu = torch.meshgrid(v, u, indexing="ij")
    out = torch.zeros(stack.n_slices, stack.H, stack.W, dtype=torch.float32, device=dev)
    tq = torch.as_tensor(ts, dtype=torch.float64, device=dev)
    wq = torch.as_tensor(w, dtype=torch.float64, device=dev)
    for k in range(stack.n_slices):
        R = xf[k, :9].reshape(3, 3)
        t = xf[k, 9:]
        base = uu[..., None] * R[:, 0] + vv[..., None] * R[:, 1] + t
        p = base[None] + tq[:, None, None, None] * R[:, 2]  # [n_quad, H, W, 3]
        g = (p / half_extent).to(torch.float32)[None]  # grid_sample order is (x,y,z)
        s = F.grid_sample(V, g, mode="bilinear", padding_mode="zeros", align_corners=True)[0, 0]
        out[k] = (s.to(torch.float64) * wq[:, None, None]).sum(0).to(torch.float32)
    if noise_sigma > 0:
        gen = torch.Generator(device="cpu").manual_seed(int(seed))
        n1 = torch.randn(out.shape, generator=gen, dtype=torch.float32).to(dev) * noise_sigma
        n2 = torch.randn(out.shape, generator=gen, dtype=torch.float32).to(dev) * noise_sigma
        out = torch.sqrt((out + n1) ** 2 + n2 ** 2)
    return out


def pick_slices(stacks: Sequence[Stack], picks):
    """Stacks holding only the picked slices ((stack index, slice index) pairs),
    in order, and each pick's [start, end) range in the flat output of the
    full stacks."""
    bases, base = [], 0
    for s in stacks:
        bases.append(base)
        base += s.n_vox
    out, ranges = [], []
    for si, k in picks:
        s = stacks[si]
        out.append(Stack(1, s.H, s.W, s.dx, s.dy, s.thickness, s.xform[k:k + 1], s.psf_u, s.psf_v))
        o = bases[si] + k * s.H * s.W
        ranges.append((o, o + s.H * s.W))
    return out, ranges


def devoxelised_gaussians(stacks: Sequence[Stack], data: Sequence[np.ndarray], n: int, seed: int,
                          jitter_mm: float = 0.5, sigma_mm: float = 1.0,
                          fg_threshold: float = 0.05) -> Gaussians:
    """Point-cloud initialisation: pick ``n`` foreground stack pixels (value >
    ``fg_threshold``) at random across all stacks, place a Gaussian at each
    pixel centre jittered by +-``jitter_mm``, isotropic std-dev ``sigma_mm``,
    identity rotation, intensity = the pixel value."""
    rng = np.random.default_rng(seed)
    pts, vals = [], []
    for st, d in zip(stacks, data):
        d = np.asarray(d, dtype=np.float64)
        P = slice_points(st)
        m = d > fg_threshold
        pts.append(P[m])
        vals.append(d[m])
    pts = np.concatenate(pts)
    vals = np.concatenate(vals)
    sel = rng.choice(pts.shape[0], size=n, replace=pts.shape[0] < n)
    mean = pts[sel] + rng.uniform(-jitter_mm, jitter_mm, size=(n, 3))
    quat = np.zeros((n, 4))
    quat[:, 0] = 1.0
    scale = np.full((n, 3), sigma_mm)
    return Gaussians(mean.astype(np.float32), quat.astype(np.float32), scale.astype(np.float32),
                     vals[sel].astype(np.float32))


# --------------------------------------------------------------------------
# the workloads (shapes of the paper's fetal-brain / adult-brain settings)
# --------------------------------------------------------------------------


@dataclass
class Workload:
    name: str
    phantom: Phantom
    stacks: List[Stack]
    noise_sigma: float
    n_gaussians: int
    target_G: int
    target_spacing: float
    extra: dict = field(default_factory=dict)


def tiny_workload(seed: int = 0) -> Workload:
    """48^3 phantom at 1 mm (12 summed ellipsoids, U[0.2,1]); 3 orthogonal stacks
    of 16 slices, 48x48 at 1 mm, 3 mm profile FWHM (slice spacing 3 mm);
    Rician sigma 0.01; 2048 devoxelised Gaussians."""
    ph = random_phantom(12, 48.0, seed, values=(0.2, 1.0), nested=False, spacing=1.0)
    stacks = [make_stack(F, 16, 48, 48, 1.0, 1.0, 3.0, 3.0) for F in (AXIAL, CORONAL, SAGITTAL)]
    return Workload("tiny-48^3-3x16x48^2-2048g", ph, stacks, 0.01, 2048, 48, 1.0)


def feta_workload(seed: int = 0, n_gaussians: int = 200_000) -> Workload:
    """256^3 phantom at 0.5 mm (60 nested ellipsoids, U[0,1]); 3 orthogonal
    stacks of 64 slices, 256x256 at 0.5 mm, 2 mm slice thickness (2 mm
    spacing); Rician sigma 0.02; 200k Gaussians; 256^3 0.5 mm target grid."""
    ph = random_phantom(60, 128.0, seed, values=(0.0, 1.0), nested=True, spacing=0.5)
    stacks = [make_stack(F, 64, 256, 256, 0.5, 0.5, 2.0, 2.0) for F in (AXIAL, CORONAL, SAGITTAL)]
    return Workload("feta-256^3-3x64x256^2-200kg", ph, stacks, 0.02, n_gaussians, 256, 0.5)


def motion_workload(seed: int = 0, n_gaussians: int = 500_000) -> Workload:
    """The 256^3 phantom with 4 stacks (3 orthogonal + 1 oblique at 30 deg) and
    known per-slice rigid motion (rotation <= 3 deg, translation <= 1 mm)."""
    ph = random_phantom(60, 128.0, seed, values=(0.0, 1.0), nested=True, spacing=0.5)
    rng = np.random.default_rng(seed + 1000)
    frames = [AXIAL, CORONAL, SAGITTAL, axis_angle_matrix([1, 0, 0], np.deg2rad(30.0)) @ AXIAL]
    stacks = [make_stack(F, 64, 256, 256, 0.5, 0.5, 2.0, 2.0, rng=rng, max_rot_deg=3.0,
                         max_trans_mm=1.0) for F in frames]
    return Workload("motion-256^3-4x64x256^2-500kg", ph, stacks, 0.02, n_gaussians, 256, 0.5)


def stress_workload(seed: int = 0, n_gaussians: int = 2_000_000) -> Workload:
    """384^3 phantom at 0.4 mm (100 ellipsoids); 5 stacks at random
    orientations, 96 slices of 384x384 at 0.4 mm, 1.6 mm thickness, per-slice
    motion <= 5 deg; 2M Gaussians; 384^3 target."""
    ph = random_phantom(100, 153.6, seed, values=(0.0, 1.0), nested=True, spacing=0.4)
    rng = np.random.default_rng(seed + 2000)
    frames = []
    for _ in range(5):
        frames.append(random_rotations(1, rng)[0])
    stacks = [make_stack(F, 96, 384, 384, 0.4, 0.4, 1.6, 1.6, rng=rng, max_rot_deg=5.0,
                         max_trans_mm=1.0) for F in frames]
    return Workload("stress-384^3-5x96x384^2-2Mg", ph, stacks, 0.02, n_gaussians, 384, 0.4)


def phantom_init_gaussians(wl: Workload, seed: int, res: int | None = None,
                           sigma_factor: float = 1.0) -> Gaussians:
    """Uniform-grid initialisation over the phantom's foreground with about
    ``wl.n_gaussians`` Gaussians: grid spacing h = (V_fg / N)^(1/3), std-dev
    h * ``sigma_factor``, intensity = phantom value at the point."""
    ph = wl.phantom
    rng = np.random.default_rng(seed)
    probe = rng.uniform(-ph.fov_mm / 2, ph.fov_mm / 2, size=(200_000, 3))
    fg_frac = float(np.mean(ph.evaluate(probe) > 0))
    v_fg = fg_frac * ph.fov_mm ** 3
    h = (v_fg / wl.n_gaussians) ** (1.0 / 3.0)
    if res is None:
        res = int(np.ceil(ph.fov_mm / h))
    return grid_gaussians(res, res * h, seed, keep=lambda p: ph.evaluate(p) > 0, sigma_factor=sigma_factor,
                          jitter=0.25, alpha_fn=lambda p: ph.evaluate(p), max_n=wl.n_gaussians)


# --------------------------------------------------------------------------
# neural residual field parameters (seeded initial weights)
# --------------------------------------------------------------------------


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """float32 values rounded to the nearest bfloat16 (ties to even), returned
    as float32, so that a BF16 copy of them is exact."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16) << np.uint64(16)
    return (u & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).reshape(a.shape)


NRF_LAYERS = {
    # preset -> [(out, in)] per linear layer
    "paper": [(64, 39), (64, 64), (64, 64), (64, 64), (1, 64)],
    "grid": [(64, 32), (64, 64), (1, 64)],
}
NRF_GRID = dict(levels=16, feats=2, log2_table=19, n_min=16, n_max=512)


def nrf_init(preset: str, seed: int, bf16: bool = True, table_range: float = 1e-4,
             last_gain: float = 1.0, grid: dict | None = None):
    """Seeded NRF parameters: uniform fan-in init per layer, biases small,
    optional BF16-representable weights; for the grid preset a feature table
    [levels, 2^log2_table, feats] uniform in +-``table_range``.
    Returns (weights list [out,in], biases list [out], table or None)."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    layers = NRF_LAYERS[preset]
    for li, (o, i) in enumerate(layers):
        lim = np.sqrt(6.0 / i) if li < len(layers) - 1 else np.sqrt(3.0 / i) * last_gain
        W = rng.uniform(-lim, lim, size=(o, i)).astype(np.float32)
        b = rng.uniform(-0.05, 0.05, size=o).astype(np.float32)
        if bf16:
            W = round_to_bf16(W)
        Ws.append(W)
        bs.append(b)
    table = None
    if preset == "grid":
        g = dict(NRF_GRID, **(grid or {}))
        table = rng.uniform(-table_range, table_range,
                            size=(g["levels"], 1 << g["log2_table"], g["feats"])).astype(np.float32)
    return Ws, bs, table


def nrf_points(n: int, seed: int) -> np.ndarray:
    """Query coordinates uniform in the canonical cube [-1,1]^3, float32 [n,3]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
