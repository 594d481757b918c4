"""Reconstruction driver (Sec. 3.1, 3.5): fit Magnetic Gaussians, and
optionally the neural residual field, to multi-stack thick-slice data, then
sample the isotropic volume.

The hot path (record pass, binning, forward and adjoint render, NRF, FP64
loss) runs in the C-ABI library; this module holds the optimiser loop.
Parameterisation follows Sec. 3.2: means in canonical coordinates
[-1,1]^3 (mm = centre + half_extent * mean_c), unnormalised quaternions,
log-scales and intensities; Adam with the learning rates of Sec. 4.1.4.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import torch

from . import ops


@dataclass
class FitConfig:
    iterations: int = 2000
    lr_position: float = 1e-3   # canonical units (Sec. 4.1.4)
    lr_intensity: float = 5e-2
    lr_scale: float = 5e-3
    lr_rotation: float = 1e-3
    lambda_aniso: float = 0.1   # Eq. E12
    lambda_r: float = 1.5       # Eq. E13
    loss: str = "l1l2"          # the plain-fit slice loss
    cutoff_k: float = 3.0
    nrf: Optional[str] = None   # None, "paper" or "grid"
    nrf_precision: str = "bf16"
    nrf_start: int = 1000       # delayed activation (Sec. 3.4)
    nrf_batch: int = 1 << 20    # voxels per iteration seen by the NRF
    lr_nrf: float = 1e-4        # Sec. 4.1.4
    lr_table: float = 1e-2
    nrf_seed: int = 0
    log_every: int = 0
    seed: int = 0


class LossL1L2(torch.autograd.Function):
    """mean |r| + mean r^2 in FP64 (mg_loss_l1l2) with its gradient."""

    @staticmethod
    def forward(ctx, pred, target, ws):
        grad = torch.empty_like(pred)
        out = torch.empty(2, dtype=torch.float64, device=pred.device)
        ops.mg_loss_l1l2(pred.detach().contiguous(), target, grad, out, ws)
        ctx.save_for_backward(grad)
        return out[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g.to(grad.dtype), None, None


def voxel_coords(stacks: Sequence, centre, half_extent: float, device="cuda") -> torch.Tensor:
    """Canonical coordinates [n_vox, 3] of every slice voxel (stacks
    concatenated, [n_slices, H, W] order)."""
    out = []
    c = torch.as_tensor(np.asarray(centre, np.float64), device=device)
    for s in stacks:
        xf = torch.as_tensor(np.asarray(s.xform, np.float64), device=device)
        u = (torch.arange(s.W, device=device, dtype=torch.float64) - (s.W - 1) / 2.0) * s.dx
        v = (torch.arange(s.H, device=device, dtype=torch.float64) - (s.H - 1) / 2.0) * s.dy
        vv, uu = torch.meshgrid(v, u, indexing="ij")
        for k in range(s.n_slices):
            R = xf[k, :9].reshape(3, 3)
            p = uu[..., None] * R[:, 0] + vv[..., None] * R[:, 1] + xf[k, 9:]
            out.append(((p - c) / half_extent).reshape(-1, 3).to(torch.float32))
    return torch.cat(out).contiguous()


class Model(torch.nn.Module):
    def __init__(self, G, centre, half_extent: float, device="cuda"):
        super().__init__()
        self.centre = torch.as_tensor(np.asarray(centre, np.float32), device=device)
        self.half = float(half_extent)
        m = (torch.as_tensor(G.mean, device=device) - self.centre) / self.half
        self.mean_c = torch.nn.Parameter(m.contiguous())
        self.quat = torch.nn.Parameter(torch.as_tensor(G.quat, device=device).clone())
        self.log_scale = torch.nn.Parameter(torch.log(torch.as_tensor(G.scale, device=device)).contiguous())
        self.alpha = torch.nn.Parameter(torch.as_tensor(G.alpha, device=device).clone())

    def gaussians(self):
        mean = self.centre + self.half * self.mean_c
        q = self.quat / self.quat.norm(dim=1, keepdim=True)
        return mean, q, torch.exp(self.log_scale), self.alpha

    def aniso(self, lam_r: float):
        s = torch.exp(self.log_scale)
        return torch.clamp(s.max(dim=1).values / s.min(dim=1).values - lam_r, min=0).mean()


def make_nrf(preset: str, precision: str, seed: int, device="cuda"):
    import mg_synth as ms

    W, b, t = ms.nrf_init(preset, seed, bf16=(precision == "bf16"), last_gain=0.1)
    return ops.NRF(preset, precision, W, b, t, device=device)


def fit(stacks, target, G_init, centre, half_extent, cfg: FitConfig, device="cuda", log=None):
    """Returns (model, nrf or None, stats). ``target``: flat device tensor of
    all slice voxels."""
    torch.manual_seed(cfg.seed)
    model = Model(G_init, centre, half_extent, device)
    R = ops.SliceRenderer(stacks, device=device, cutoff_k=cfg.cutoff_k, check=True)
    opt = torch.optim.Adam([
        {"params": [model.mean_c], "lr": cfg.lr_position},
        {"params": [model.alpha], "lr": cfg.lr_intensity},
        {"params": [model.log_scale], "lr": cfg.lr_scale},
        {"params": [model.quat], "lr": cfg.lr_rotation}])
    ws = torch.empty(ops.mg_reduce_workspace_size(target.numel()), dtype=torch.uint8, device=device)
    nrf = None
    nrf_opt = None
    coords = None
    nrf_params = nrf_table = None
    gen = torch.Generator(device=device).manual_seed(cfg.seed + 17)
    n_vox = target.numel()
    hist = []
    t0 = time.perf_counter()
    for it in range(cfg.iterations):
        if cfg.nrf and it == cfg.nrf_start:
            nrf = make_nrf(cfg.nrf, cfg.nrf_precision, cfg.nrf_seed, device)
            nrf_params = torch.nn.Parameter(nrf.params.clone())
            groups = [{"params": [nrf_params], "lr": cfg.lr_nrf}]
            if nrf.table is not None:
                nrf_table = torch.nn.Parameter(nrf.table.clone())
                groups.append({"params": [nrf_table], "lr": cfg.lr_table})
            nrf_opt = torch.optim.Adam(groups)
            coords = voxel_coords(stacks, centre, half_extent, device)
        mean, q, s, a = model.gaussians()
        pred = ops.RenderSlices.apply(R, mean, q, s, a)  # checks capacity every iteration (grows on overflow)
        if nrf is not None:
            idx = torch.randint(0, n_vox, (min(cfg.nrf_batch, n_vox),), device=device, generator=gen)
            r = ops.NRFFunction.apply(nrf, coords[idx], nrf_params, nrf_table)
            pred = pred.index_add(0, idx, r)
        loss = LossL1L2.apply(pred, target, ws)
        total = loss.float() + cfg.lambda_aniso * model.aniso(cfg.lambda_r)
        opt.zero_grad(set_to_none=True)
        if nrf_opt:
            nrf_opt.zero_grad(set_to_none=True)
        total.backward()
        opt.step()
        if nrf_opt:
            nrf_opt.step()
        with torch.no_grad():
            model.alpha.clamp_(0.0, 1.0)  # alpha in [0, 1] (Sec. 3.2)
        if cfg.log_every and (it % cfg.log_every == 0 or it == cfg.iterations - 1):
            hist.append((it, float(loss.detach())))
            if log:
                log(f"it {it} loss {hist[-1][1]:.6e}")
    torch.cuda.synchronize()
    st = R.stats()
    if st["status"] != 0:
        raise RuntimeError(f"render status {st['status']} during the fit")
    if nrf is not None:
        nrf.params = nrf_params.detach().contiguous()
        if nrf_table is not None:
            nrf.table = nrf_table.detach().contiguous()
    return model, nrf, {"seconds": time.perf_counter() - t0, "history": hist, "final_loss": float(loss.detach())}


def sample(model: Model, nrf, G_dim: int, spacing: float, centre=(0.0, 0.0, 0.0), cutoff_k: float = 3.0,
           batch: int = 1 << 22):
    """The isotropic G^3 volume (z, y, x): Gaussian mixture (Eq. E7) plus the
    NRF residual at the voxel centres (Eq. E8)."""
    with torch.no_grad():
        mean, q, s, a = model.gaussians()
        S = ops.VolumeSampler(G_dim, spacing, centre, device=mean.device, cutoff_k=cutoff_k)
        vol = S(mean.contiguous(), q.contiguous(), s.contiguous(), a.contiguous()).clone()
        if nrf is not None:
            dev = mean.device
            ax = (torch.arange(G_dim, device=dev, dtype=torch.float64) - (G_dim - 1) / 2.0) * spacing
            c = torch.as_tensor(np.asarray(centre, np.float64), device=dev)
            flat = vol.view(-1)
            out = torch.empty(min(batch, G_dim ** 3), device=dev)
            zz = ax + c[2]
            for start in range(0, G_dim ** 3, batch):
                n = min(batch, G_dim ** 3 - start)
                lin = torch.arange(start, start + n, device=dev)
                iz, rem = lin // (G_dim * G_dim), lin % (G_dim * G_dim)
                iy, ix = rem // G_dim, rem % G_dim
                xyz = torch.stack([ax[ix] + c[0], ax[iy] + c[1], zz[iz]], dim=1)
                xyz = ((xyz - model.centre.double()) / model.half).to(torch.float32).contiguous()
                ops.mg_nrf_fwd(nrf, xyz, out[:n])
                flat[start:start + n] += out[:n]
        return vol


def psnr(vol: torch.Tensor, ref: torch.Tensor, max_val: float = 1.0) -> float:
    """10 log10(max^2 / MSE) with the squared differences summed in FP64 on the device."""
    a = vol.reshape(-1).contiguous().float()
    b = ref.reshape(-1).contiguous().float().to(a.device)
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    ws = torch.empty(ops.mg_reduce_workspace_size(a.numel()), dtype=torch.uint8, device=a.device)
    ops.mg_sq_diff_sum(a, b, out, ws)
    mse = float(out) / a.numel()
    return float("inf") if mse == 0 else 10.0 * np.log10(max_val * max_val / mse)
