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
    loss: str = "l1l2"          # "l1l2" (mean |r| + mean r^2) or "paper" (smooth L1 + lambda_ssim SSIM, Sec. 3.5.2)
    local_set: str = "ksigma"   # "ksigma" (K-sigma tiles) or "cells" (the paper's cell grid, Eqs. E4-E6)
    grid_res: int = 0           # cells: cells per axis of the canonical cube
    block_radius: int = 5       # cells: the paper's default (Sec. 4.1.4)
    lambda_ssim: float = 0.5    # Sec. 4.1.4
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
    graph: bool = True          # replay each phase's iteration as a CUDA graph
    check_every: int = 100      # graph replays between host checks of the step counter
    headroom: float = 1.5       # bin capacity over the warm-up iteration's need (graph mode)


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


def cells_of(cfg: FitConfig, centre, half_extent):
    """The cell-grid local set of the fit's canonical cube, or None."""
    if cfg.local_set == "ksigma":
        return None
    if cfg.local_set != "cells" or cfg.grid_res < 1:
        raise ValueError("local_set must be 'ksigma', or 'cells' with grid_res >= 1")
    return dict(grid_res=cfg.grid_res, block_radius=cfg.block_radius, centre=tuple(float(c) for c in centre),
                half=float(half_extent))


class _Trainer:
    """One training iteration of the fit as a sequence of stream-ordered
    launches with no host synchronisation (so it can be captured in a CUDA
    graph): render (mg_render_fwd), optional NRF residual on a random voxel
    batch, FP64 loss, backward (mg_render_bwd, mg_nrf_bwd) and the Adam step
    (mg_adam_step), predicated on the forward's device status word."""

    def __init__(self, stacks, target, G_init, centre, half_extent, cfg: FitConfig, device):
        self.cfg, self.device, self.target = cfg, device, target
        self.stacks, self.centre, self.half = stacks, centre, half_extent
        self.model = Model(G_init, centre, half_extent, device)
        self.cells = cells_of(cfg, centre, half_extent)
        self.R = ops.SliceRenderer(stacks, device=device, cutoff_k=cfg.cutoff_k, check=True, cells=self.cells)
        m = self.model
        self.adam = ops.DeviceAdam([
            {"param": m.mean_c, "lr": cfg.lr_position},
            {"param": m.alpha, "lr": cfg.lr_intensity, "clamp": (0.0, 1.0)},  # alpha in [0, 1] (Sec. 3.2)
            {"param": m.log_scale, "lr": cfg.lr_scale},
            {"param": m.quat, "lr": cfg.lr_rotation}])
        if cfg.loss not in ("l1l2", "paper"):
            raise ValueError(f"unknown loss {cfg.loss!r}")
        if cfg.loss == "paper":
            self.ws = torch.empty(ops.mg_loss_recon_workspace_size(self.R.dev), dtype=torch.uint8, device=device)
        else:
            self.ws = torch.empty(ops.mg_reduce_workspace_size(target.numel()), dtype=torch.uint8, device=device)
        self.nrf = self.nrf_adam = self.coords = None
        self.nrf_params = self.nrf_table = None
        self.nrf_enc = None  # grid encoding of the current NRF batch (forward stores, backward reads)
        # device buffers of the parameterisation (mg_params_fwd / _bwd)
        n = m.mean_c.shape[0]
        f32 = dict(dtype=torch.float32, device=device)
        self.mean, self.q, self.s = torch.empty(n, 3, **f32), torch.empty(n, 4, **f32), torch.empty(n, 3, **f32)
        self.g_mc, self.g_qr, self.g_ls = torch.empty(n, 3, **f32), torch.empty(n, 4, **f32), torch.empty(n, 3, **f32)
        self.aniso = torch.zeros(1, dtype=torch.float64, device=device)
        self.ws_p = torch.empty(ops.mg_params_workspace_size(n), dtype=torch.uint8, device=device)
        self.pred = torch.empty(self.R.dev.n_vox, **f32)

    def enable_nrf(self):
        cfg = self.cfg
        self.nrf = make_nrf(cfg.nrf, cfg.nrf_precision, cfg.nrf_seed, self.device)
        self.nrf_params = torch.nn.Parameter(self.nrf.params.clone())
        groups = [{"param": self.nrf_params, "lr": cfg.lr_nrf}]
        if self.nrf.table is not None:
            self.nrf_table = torch.nn.Parameter(self.nrf.table.clone())
            groups.append({"param": self.nrf_table, "lr": cfg.lr_table})
        self.nrf_adam = ops.DeviceAdam(groups)
        self.coords = voxel_coords(self.stacks, self.centre, self.half, self.device)
        torch.cuda.manual_seed(cfg.seed + 17)  # voxel batches come from the default CUDA generator

    def zero_grad(self):
        self.adam.zero_grad()
        if self.nrf_adam is not None:
            self.nrf_adam.zero_grad()

    def iteration(self):
        """One step, all in this library's kernels; the NRF's random voxel
        batch (Sec. 3.4) is drawn by torch's generator and passed in as row
        indices."""
        cfg, m = self.cfg, self.model
        with torch.no_grad():
            ops.mg_params_fwd(m.mean_c, m.quat, m.log_scale, self.centre, self.half, cfg.lambda_r, self.mean, self.q,
                              self.s, self.aniso, self.ws_p)
            fused = cfg.loss != "paper" and self.nrf is None
            if fused:
                # the L1 + L2 loss and its gradient fused into the forward's writes
                grad = torch.empty_like(self.pred)
                out = torch.empty(2, dtype=torch.float64, device=self.device)
                pred = self.R.forward_l1l2(self.mean, self.q, self.s, m.alpha, self.target, self.pred, grad, out)
            else:
                pred = self.R.forward(self.mean, self.q, self.s, m.alpha, out=self.pred)
            if self.nrf is not None:
                n_vox = self.target.numel()
                idx = torch.randint(0, n_vox, (min(cfg.nrf_batch, n_vox),), device=self.device)
                if self.nrf_enc is None:
                    self.nrf_enc = self.nrf.enc_cache(idx.numel())
                ops.mg_nrf_fwd_at(self.nrf, self.coords, idx, idx.numel(), pred, self.nrf_params, self.nrf_table,
                                  enc=self.nrf_enc)
            # the loss (FP64 sums) and its gradient dL/dpred in one kernel
            if cfg.loss == "paper":
                grad = torch.empty_like(pred)
                out = torch.empty(3, dtype=torch.float64, device=pred.device)
                ops.mg_loss_recon(pred, self.target, self.R.dev, cfg.lambda_ssim, grad, out, self.ws)
            elif not fused:
                grad = torch.empty_like(pred)
                out = torch.empty(2, dtype=torch.float64, device=pred.device)
                ops.mg_loss_l1l2(pred, self.target, grad, out, self.ws)
            if self.nrf is not None:
                gp = torch.empty_like(self.nrf_params)
                gt = torch.empty_like(self.nrf_table) if self.nrf_table is not None else None
                ops.mg_nrf_bwd_at(self.nrf, self.coords, idx, idx.numel(), grad, gp, gt, self.nrf_params,
                                  self.nrf_table, enc=self.nrf_enc)
                self.nrf_params.grad = gp
                if gt is not None:
                    self.nrf_table.grad = gt
            gm, gq, gs, ga = self.R.backward(self.mean, self.q, self.s, m.alpha, grad)
            ops.mg_params_bwd(m.quat, m.log_scale, self.half, cfg.lambda_r, cfg.lambda_aniso, gm, gq, gs, self.g_mc,
                              self.g_qr, self.g_ls)
            m.mean_c.grad, m.quat.grad, m.log_scale.grad, m.alpha.grad = self.g_mc, self.g_qr, self.g_ls, ga
            status = self.R.status_word
            self.adam.step(status=status)
            if self.nrf_adam is not None:
                self.nrf_adam.step(status=status)
        return out[0]

    def done(self) -> int:
        return self.adam.steps

    def size_bins(self, factor: float, keep_larger: bool = True):
        """Capacity = factor x the last forward's record and entry counts
        (never below the current capacity when ``keep_larger``)."""
        st = self.R.stats()
        if st["status"] == ops.L.MG_ERR_NOT_FINITE:
            raise ops.L.MgError(ops.L.MG_ERR_NOT_FINITE, "fit: non-finite Gaussian parameters")
        n = self.model.mean_c.shape[0]
        r, e = int(st["records"] * factor) + 1, int(st["entries"] * factor) + 1
        if keep_larger:
            r, e = max(r, self.R.caps[0]), max(e, self.R.caps[1])
        self.R.set_capacity(r, e, n)

    def finish(self):
        if self.nrf is not None:
            self.nrf.params = self.nrf_params.detach().contiguous()
            if self.nrf_table is not None:
                self.nrf.table = self.nrf_table.detach().contiguous()


def _phase_end(cfg: FitConfig, done: int) -> int:
    if cfg.nrf and done < cfg.nrf_start:
        return min(cfg.nrf_start, cfg.iterations)
    return cfg.iterations


def fit(stacks, target, G_init, centre, half_extent, cfg: FitConfig, device="cuda", log=None):
    """Returns (model, nrf or None, stats). ``target``: flat device tensor of
    all slice voxels.

    With ``cfg.graph`` each phase (before / after the NRF starts) runs two
    eager iterations on a side stream (they size the bins, with 1.5x
    headroom), then captures one iteration in a CUDA graph and replays it,
    checking the device step counter every ``cfg.check_every`` iterations. An
    iteration whose bins overflow changes nothing (the Adam step is
    predicated on the render status), so on a lag the workspace grows, the
    graph is captured again and the missing iterations are run."""
    torch.manual_seed(cfg.seed)
    t0 = time.perf_counter()
    T = _Trainer(stacks, target, G_init, centre, half_extent, cfg, device)
    hist = []
    captures = 0
    t_eager = t_capture = t_replay = 0.0
    loss = None
    if not cfg.graph:
        for it in range(cfg.iterations):
            if cfg.nrf and it == cfg.nrf_start:
                T.enable_nrf()
            T.zero_grad()
            loss = T.iteration()  # the renderer checks capacity every iteration (grows on overflow)
            if cfg.log_every and (it % cfg.log_every == 0 or it == cfg.iterations - 1):
                hist.append((it, float(loss.detach())))
                if log:
                    log(f"it {it} loss {hist[-1][1]:.6e}")
    else:
        done = 0
        while done < cfg.iterations:
            if cfg.nrf and done >= cfg.nrf_start and T.nrf is None:
                T.enable_nrf()
            end = _phase_end(cfg, done)
            # eager warm-up on a side stream: sizes the bins and initialises lazily created state
            T.R.check = True
            ta = time.perf_counter()
            side = torch.cuda.Stream(device=device)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                for _ in range(min(2, end - done)):
                    T.zero_grad()
                    loss = T.iteration()
                    if cfg.log_every and done % cfg.log_every == 0:
                        hist.append((done, float(loss)))
                    done += 1
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            t_eager += time.perf_counter() - ta
            if done >= end:
                continue
            T.size_bins(cfg.headroom, keep_larger=False)
            graph = None
            lags = 0
            while done < end:
                if graph is None:
                    ta = time.perf_counter()
                    T.R.check = False
                    T.zero_grad()
                    graph = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(graph):
                        loss = T.iteration()
                    captures += 1
                    t_capture += time.perf_counter() - ta
                ta = time.perf_counter()
                k = min(cfg.check_every, end - done)
                for _ in range(k):
                    graph.replay()
                now = T.done()  # synchronises
                t_replay += time.perf_counter() - ta
                if now < done + k:  # an iteration's bins overflowed: it was a no-op
                    lags += 1
                    if lags > 8:
                        raise RuntimeError("fit: the bins keep overflowing after growing the workspace")
                    graph = None
                    T.size_bins(1.5)
                if cfg.log_every:
                    hist.append((now - 1, float(loss.detach())))
                    if log:
                        log(f"it {now - 1} loss {hist[-1][1]:.6e}")
                done = now
            del graph
        T.R.check = True
    torch.cuda.synchronize()
    st = T.R.stats()
    if st["status"] != 0:
        raise RuntimeError(f"render status {st['status']} during the fit")
    T.finish()
    seconds = time.perf_counter() - t0
    return T.model, T.nrf, {"seconds": seconds, "history": hist, "final_loss": float(loss.detach()),
                            "graph_captures": captures, "iterations": T.done(),
                            "seconds_eager": t_eager, "seconds_capture": t_capture, "seconds_replay": t_replay}


def _rotvec_to_matrix(w: torch.Tensor) -> torch.Tensor:
    """Rodrigues' formula, [S,3] -> [S,3,3] (FP64)."""
    th = torch.linalg.norm(w, dim=1, keepdim=True)
    k = w / th.clamp_min(1e-30)
    K = torch.zeros(w.shape[0], 3, 3, dtype=w.dtype, device=w.device)
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 0] = -k[:, 2], k[:, 1], k[:, 2]
    K[:, 1, 2], K[:, 2, 0], K[:, 2, 1] = -k[:, 0], -k[:, 1], k[:, 0]
    s, c = torch.sin(th)[:, :, None], torch.cos(th)[:, :, None]
    eye = torch.eye(3, dtype=w.dtype, device=w.device).expand_as(K)
    return eye + s * K + (1 - c) * (K @ K)


def register_slices(renderer: ops.SliceRenderer, mean, quat, scale, alpha, target, iterations: int = 100,
                    lr_t: float = 0.05, lr_r: float = 0.01, lr_final: float = 0.02):
    """Slice-to-volume registration against fixed Gaussians: the slice poses
    T_k (Sec. 3.3.2) are corrected by Adam (mg_adam_step) on the pose
    gradient of the L1+L2 slice loss (mg_render_pose_grad), the learning
    rates decaying exponentially to ``lr_final`` of their start. Each pose is
    composed from the starting transform as t = t0 + dt, R = R0 Exp(omega);
    the pose gradient is taken at the current pose (omega in the slice
    frame). The renderer's transforms are updated in place. Returns the loss
    history."""
    dev = mean.device
    D = renderer.dev
    x0 = D.poses().double()
    S = x0.shape[0]
    R0, t0 = x0[:, :9].reshape(S, 3, 3), x0[:, 9:]
    dt = torch.zeros(S, 3, dtype=torch.float32, device=dev)
    om = torch.zeros(S, 3, dtype=torch.float32, device=dev)
    adam = ops.DeviceAdam([{"param": dt, "lr": lr_t}, {"param": om, "lr": lr_r}])
    n = target.numel()
    grad = torch.empty(n, dtype=torch.float32, device=dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    ws = torch.empty(ops.mg_reduce_workspace_size(n), dtype=torch.uint8, device=dev)

    def apply():
        R = R0 @ _rotvec_to_matrix(om.double())
        D.set_poses(torch.cat([R.reshape(S, 9), t0 + dt.double()], dim=1).float())

    hist = []
    for it in range(iterations):
        decay = lr_final ** (it / max(iterations - 1, 1))
        adam.groups[0]["lr"], adam.groups[1]["lr"] = lr_t * decay, lr_r * decay
        apply()
        pred = renderer.forward(mean, quat, scale, alpha)
        ops.mg_loss_l1l2(pred, target, grad, out, ws)
        renderer.backward(mean, quat, scale, alpha, grad)
        g = renderer.pose_grad(mean, quat, scale, alpha)
        dt.grad = g[:, :3].contiguous()
        om.grad = g[:, 3:].contiguous()
        adam.step()
        hist.append(float(out[0]))
    apply()
    return hist


def sample(model: Model, nrf, G_dim: int, spacing: float, centre=(0.0, 0.0, 0.0), cutoff_k: float = 3.0,
           batch: int = 1 << 22, cells=None):
    """The isotropic G^3 volume (z, y, x): Gaussian mixture (Eq. E7) plus the
    NRF residual at the voxel centres (Eq. E8); ``cells``: the cell-grid local
    set of the fit (``cells_of``), None for the K-sigma set."""
    with torch.no_grad():
        mean, q, s, a = model.gaussians()
        S = ops.VolumeSampler(G_dim, spacing, centre, device=mean.device, cutoff_k=cutoff_k, cells=cells)
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
