"""Python binding of the mgauss C ABI over torch CUDA tensors.

The functions ``mg_*`` below carry the names and arguments of include/mgauss.h
and only marshal arguments (tensor -> device pointer, stream handle); every
step of the computation runs in the library's CUDA kernels. PyTorch provides
device memory, streams and autograd glue.

``SliceRenderer`` owns a workspace and grows it when the device reports a
capacity overflow; ``RenderSlices`` is the autograd Function whose backward
is ``mg_render_bwd``.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence

import torch

from . import _lib as L

_F32 = torch.float32


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype=_F32, numel=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _gauss(mean, quat, scale, alpha) -> L.MgGaussians:
    n = mean.shape[0] if mean.dim() == 2 else mean.numel() // 3
    return L.MgGaussians(n, _dev(mean, "mean", numel=3 * n), _dev(quat, "quat", numel=4 * n),
                         _dev(scale, "scale", numel=3 * n), _dev(alpha, "alpha", numel=n))


def _opts(cutoff_k=3.0, f64_ratio=16.0, cap_records=0, cap_entries=0, cells=None) -> L.MgOpts:
    """``cells``: None for the K-sigma local set, or a dict(grid_res, block_radius,
    centre (mm, 3), half (mm)) for the paper's cell-grid local set (Eqs. E4-E6)."""
    o = L.MgOpts(float(cutoff_k), float(f64_ratio), int(cap_records), int(cap_entries))
    o.local_set = L.MG_LOCAL_KSIGMA
    o.block_radius = 5
    if cells is not None:
        o.local_set = L.MG_LOCAL_CELLS
        o.grid_res = int(cells["grid_res"])
        o.block_radius = int(cells["block_radius"])
        for a in range(3):
            o.grid_centre[a] = float(cells["centre"][a])
        o.grid_half = float(cells["half"])
    return o


class DeviceStacks:
    """Stack geometry resident on the device (transforms uploaded once)."""

    def __init__(self, stacks: Sequence, device="cuda"):
        self.stacks = list(stacks)
        self.xforms = [torch.as_tensor(s.xform, dtype=_F32).reshape(s.n_slices, 12).contiguous().to(device)
                       for s in self.stacks]
        arr = (L.MgStack * len(self.stacks))()
        for i, (s, x) in enumerate(zip(self.stacks, self.xforms)):
            arr[i] = L.MgStack(int(s.n_slices), int(s.H), int(s.W), float(s.dx), float(s.dy), float(s.thickness),
                               x.data_ptr(), float(getattr(s, "psf_u", 0.0)), float(getattr(s, "psf_v", 0.0)))
        self.arr = arr
        self.n = len(self.stacks)
        self.n_vox = sum(int(s.n_slices) * int(s.H) * int(s.W) for s in self.stacks)
        self.n_slices = sum(int(s.n_slices) for s in self.stacks)
        T = L.MG_TILE_EDGE
        self.n_tiles = sum(int(s.n_slices) * ((int(s.W) + T - 1) // T) * ((int(s.H) + T - 1) // T) for s in self.stacks)

    def set_poses(self, xform_all: torch.Tensor):
        """Overwrite the slice transforms in place (device [slices, 12], all
        stacks in order); the device pointers the renderer holds stay valid."""
        o = 0
        for x in self.xforms:
            x.copy_(xform_all[o:o + x.shape[0]])
            o += x.shape[0]

    def poses(self) -> torch.Tensor:
        return torch.cat(self.xforms)


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------

def mg_render_workspace_size(n: int, stacks: DeviceStacks, opts: L.MgOpts) -> int:
    g = L.MgGaussians(int(n), None, None, None, None)
    return int(L.lib().mg_render_workspace_size(ctypes.byref(g), stacks.arr, stacks.n, ctypes.byref(opts)))


def mg_render_fwd(mean, quat, scale, alpha, stacks: DeviceStacks, opts: L.MgOpts, out, ws, stream=None):
    g = _gauss(mean, quat, scale, alpha)
    _dev(out, "out", numel=stacks.n_vox)
    _dev(ws, "ws", dtype=torch.uint8)
    st = L.lib().mg_render_fwd(ctypes.byref(g), stacks.arr, stacks.n, ctypes.byref(opts), out.data_ptr(),
                               ws.data_ptr(), ws.numel(), _stream_handle(stream))
    L.check(st, "mg_render_fwd")


def mg_render_fwd_l1l2(mean, quat, scale, alpha, stacks: DeviceStacks, opts: L.MgOpts, target, out, grad, loss_out,
                       ws, stream=None):
    """mg_render_fwd with the L1 + L2 slice loss fused (loss_out: device
    float64[2] = {loss, sum r^2}; grad may be None)."""
    g = _gauss(mean, quat, scale, alpha)
    _dev(target, "target", numel=stacks.n_vox)
    _dev(out, "out", numel=stacks.n_vox)
    if grad is not None:
        _dev(grad, "grad", numel=stacks.n_vox)
    _dev(loss_out, "loss_out", dtype=torch.float64, numel=2)
    _dev(ws, "ws", dtype=torch.uint8)
    st = L.lib().mg_render_fwd_l1l2(ctypes.byref(g), stacks.arr, stacks.n, ctypes.byref(opts), target.data_ptr(),
                                    out.data_ptr(), grad.data_ptr() if grad is not None else None,
                                    loss_out.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(stream))
    L.check(st, "mg_render_fwd_l1l2")


def mg_render_bwd(mean, quat, scale, alpha, stacks: DeviceStacks, opts: L.MgOpts, grad_out, g_mean, g_quat,
                  g_scale, g_alpha, ws, stream=None, raise_on_error=True) -> int:
    g = _gauss(mean, quat, scale, alpha)
    n = g.n
    _dev(grad_out, "grad_out", numel=stacks.n_vox)
    ptrs = [_dev(g_mean, "g_mean", numel=3 * n), _dev(g_quat, "g_quat", numel=4 * n),
            _dev(g_scale, "g_scale", numel=3 * n), _dev(g_alpha, "g_alpha", numel=n)]
    st = L.lib().mg_render_bwd(ctypes.byref(g), stacks.arr, stacks.n, ctypes.byref(opts), grad_out.data_ptr(),
                               *ptrs, ws.data_ptr(), ws.numel(), _stream_handle(stream))
    if raise_on_error:
        L.check(st, "mg_render_bwd")
    return st


def mg_render_pose_grad(mean, quat, scale, alpha, stacks: DeviceStacks, opts: L.MgOpts, g_pose, ws, stream=None):
    """g_pose: device FP32 [slices, 6] = (dL/dt world, dL/domega slice frame) per slice."""
    g = _gauss(mean, quat, scale, alpha)
    _dev(g_pose, "g_pose", numel=6 * stacks.n_slices)
    L.check(L.lib().mg_render_pose_grad(ctypes.byref(g), stacks.arr, stacks.n, ctypes.byref(opts), g_pose.data_ptr(),
                                        ws.data_ptr(), ws.numel(), _stream_handle(stream)), "mg_render_pose_grad")


def mg_render_ws_layout(n: int, stacks: DeviceStacks, opts: L.MgOpts) -> dict:
    g = L.MgGaussians(int(n), None, None, None, None)
    lay = L.MgWsLayout()
    L.check(L.lib().mg_render_ws_layout(ctypes.byref(g), stacks.arr, stacks.n, ctypes.byref(opts), ctypes.byref(lay)),
            "mg_render_ws_layout")
    return {k: int(getattr(lay, k)) for k, _ in L.MgWsLayout._fields_}


def mg_sample_ws_layout(n: int, G: int, opts: L.MgOpts) -> dict:
    lay = L.MgWsLayout()
    L.check(L.lib().mg_sample_ws_layout(int(n), int(G), ctypes.byref(opts), ctypes.byref(lay)), "mg_sample_ws_layout")
    return {k: int(getattr(lay, k)) for k, _ in L.MgWsLayout._fields_}


def read_bins(ws, layout: dict, n_records: int, n_tiles: int, n_entries: int):
    """Copies of the records (gid, slice, rect, row insets) and tile bins from a workspace."""
    def view(off, count, dtype, width=1):
        nbytes = count * width * torch.tensor([], dtype=dtype).element_size()
        return ws[off:off + nbytes].view(dtype).reshape(count, width).cpu()
    gid = view(layout["rec_gid"], n_records, torch.int32)[:, 0]
    sl = view(layout["rec_slice"], n_records, torch.int32)[:, 0]
    tiles = view(layout["rec_rect"], n_records, torch.int16, 8)  # 16-byte records: rect, row insets
    rect = tiles[:, :4].to(torch.int32) & 0xFFFF
    inset = tiles[:, 4:].contiguous().view(torch.int64)[:, 0]
    toff = view(layout["tile_off"], n_tiles + 1, torch.int32)[:, 0].to(torch.int64) & 0xFFFFFFFF
    ent = view(layout["entries"], n_entries, torch.int32)[:, 0].to(torch.int64) & 0xFFFFFFFF
    return gid, sl, rect, inset, toff, ent


def mg_render_stats_get(ws, stream=None) -> dict:
    s = L.MgRenderStats()
    st = L.lib().mg_render_stats_get(ws.data_ptr(), ws.numel(), ctypes.byref(s), _stream_handle(stream))
    if st not in (L.MG_OK, L.MG_ERR_CAPACITY, L.MG_ERR_NOT_FINITE):
        L.check(st, "mg_render_stats_get")
    return {"records": s.records, "entries": s.entries, "tiles": s.tiles, "cap_records": s.cap_records,
            "cap_entries": s.cap_entries, "status": s.status}


def mg_sample_workspace_size(n: int, G: int, opts: L.MgOpts) -> int:
    return int(L.lib().mg_sample_workspace_size(int(n), int(G), ctypes.byref(opts)))


def mg_sample_volume(mean, quat, scale, alpha, centre, spacing: float, G: int, opts: L.MgOpts, out, ws, stream=None):
    g = _gauss(mean, quat, scale, alpha)
    _dev(out, "out", numel=G ** 3)
    c = (ctypes.c_float * 3)(*[float(v) for v in centre])
    st = L.lib().mg_sample_volume(ctypes.byref(g), c, float(spacing), int(G), ctypes.byref(opts), out.data_ptr(),
                                  ws.data_ptr(), ws.numel(), _stream_handle(stream))
    L.check(st, "mg_sample_volume")


def mg_reduce_workspace_size(n: int) -> int:
    return int(L.lib().mg_reduce_workspace_size(int(n)))


def mg_loss_l1l2(pred, target, grad, loss_out, ws, stream=None):
    n = pred.numel()
    _dev(target, "target", numel=n)
    gp = _dev(grad, "grad", numel=n) if grad is not None else None
    _dev(loss_out, "loss_out", dtype=torch.float64, numel=2)
    st = L.lib().mg_loss_l1l2(_dev(pred, "pred"), target.data_ptr(), n, gp, loss_out.data_ptr(), ws.data_ptr(),
                              ws.numel(), _stream_handle(stream))
    L.check(st, "mg_loss_l1l2")


def mg_sq_diff_sum(a, b, out, ws, stream=None):
    n = a.numel()
    _dev(b, "b", numel=n)
    _dev(out, "out", dtype=torch.float64, numel=1)
    st = L.lib().mg_sq_diff_sum(_dev(a, "a"), b.data_ptr(), n, out.data_ptr(), ws.data_ptr(), ws.numel(),
                                _stream_handle(stream))
    L.check(st, "mg_sq_diff_sum")


def mg_loss_recon_workspace_size(stacks: DeviceStacks) -> int:
    return int(L.lib().mg_loss_recon_workspace_size(stacks.arr, stacks.n))


def mg_loss_recon(pred, target, stacks: DeviceStacks, lambda_ssim: float, grad, loss_out, ws, stream=None):
    """Smooth-L1 + lambda_ssim (1 - mean SSIM) over the slices of ``stacks``;
    loss_out: device double[3] = {loss, mean smooth-L1, mean SSIM}."""
    n = stacks.n_vox
    _dev(pred, "pred", numel=n)
    _dev(target, "target", numel=n)
    gp = _dev(grad, "grad", numel=n) if grad is not None else None
    _dev(loss_out, "loss_out", dtype=torch.float64, numel=3)
    _dev(ws, "ws", dtype=torch.uint8)
    L.check(L.lib().mg_loss_recon(pred.data_ptr(), target.data_ptr(), stacks.arr, stacks.n, float(lambda_ssim), gp,
                                  loss_out.data_ptr(), ws.data_ptr(), ws.numel(), _stream_handle(stream)),
            "mg_loss_recon")


def mg_render_pair_count(mean, quat, scale, alpha, stacks: DeviceStacks, opts: L.MgOpts, ws, stream=None):
    g = _gauss(mean, quat, scale, alpha)
    c = (ctypes.c_int64 * 2)()
    L.check(L.lib().mg_render_pair_count(ctypes.byref(g), stacks.arr, stacks.n, ctypes.byref(opts), ws.data_ptr(),
                                         ws.numel(), c, _stream_handle(stream)), "mg_render_pair_count")
    return int(c[0]), int(c[1])


def mg_adam_step(groups: Sequence[dict], beta1: float, beta2: float, eps: float, step, status=None,
                 status_mask: int = L.MG_WS_FAIL_BITS, stream=None):
    """groups: dicts with param, grad, m, v (device FP32 tensors of one size),
    lr and optional clamp (lo, hi). ``step``: device int32 [1]; ``status``:
    a device tensor whose first 32-bit word predicates the update, or None."""
    arr = (L.MgAdamGroup * len(groups))()
    for i, g in enumerate(groups):
        n = g["param"].numel()
        lo, hi = g.get("clamp") or (1.0, 0.0)
        arr[i] = L.MgAdamGroup(_dev(g["param"], "param"), _dev(g["grad"], "grad", numel=n),
                               _dev(g["m"], "m", numel=n), _dev(g["v"], "v", numel=n), n, float(g["lr"]),
                               float(lo), float(hi))
    sp = _dev(step, "step", dtype=torch.int32, numel=1)
    stp = None
    if status is not None:
        if not status.is_cuda or status.numel() * status.element_size() < 4:
            raise ValueError("status must be a CUDA tensor of at least 4 bytes")
        stp = status.data_ptr()
    L.check(L.lib().mg_adam_step(arr, len(groups), float(beta1), float(beta2), float(eps), sp, stp,
                                 int(status_mask), _stream_handle(stream)), "mg_adam_step")


def mg_params_workspace_size(n: int) -> int:
    return int(L.lib().mg_params_workspace_size(int(n)))


def mg_params_fwd(mean_c, quat_raw, log_scale, centre, half: float, lambda_r: float, mean, quat, scale,
                  aniso_out=None, ws=None, stream=None):
    n = mean_c.numel() // 3
    args = [_dev(mean_c, "mean_c", numel=3 * n), _dev(quat_raw, "quat_raw", numel=4 * n),
            _dev(log_scale, "log_scale", numel=3 * n)]
    c = (ctypes.c_float * 3)(*[float(v) for v in centre])
    outs = [_dev(mean, "mean", numel=3 * n), _dev(quat, "quat", numel=4 * n), _dev(scale, "scale", numel=3 * n)]
    ap = _dev(aniso_out, "aniso_out", dtype=torch.float64, numel=1) if aniso_out is not None else None
    wp = _dev(ws, "ws", dtype=torch.uint8) if ws is not None else None
    L.check(L.lib().mg_params_fwd(n, *args, c, float(half), float(lambda_r), *outs, ap, wp,
                                  ws.numel() if ws is not None else 0, _stream_handle(stream)), "mg_params_fwd")


def mg_params_bwd(quat_raw, log_scale, half: float, lambda_r: float, lambda_aniso: float, g_mean, g_quat, g_scale,
                  g_mean_c, g_quat_raw, g_log_scale, stream=None):
    n = quat_raw.numel() // 4
    L.check(L.lib().mg_params_bwd(n, _dev(quat_raw, "quat_raw", numel=4 * n), _dev(log_scale, "log_scale", numel=3 * n),
                                  float(half), float(lambda_r), float(lambda_aniso),
                                  _dev(g_mean, "g_mean", numel=3 * n), _dev(g_quat, "g_quat", numel=4 * n),
                                  _dev(g_scale, "g_scale", numel=3 * n), _dev(g_mean_c, "g_mean_c", numel=3 * n),
                                  _dev(g_quat_raw, "g_quat_raw", numel=4 * n),
                                  _dev(g_log_scale, "g_log_scale", numel=3 * n), _stream_handle(stream)),
            "mg_params_bwd")


def mg_profile_enable(on: bool = True):
    L.check(L.lib().mg_profile_enable(1 if on else 0), "mg_profile_enable")


def mg_profile_stages(names):
    """Time only the named stages (the others launch without events)."""
    lib = L.lib()
    all_names = [lib.mg_profile_stage_name(i).decode() for i in range(lib.mg_profile_stage_count())]
    mask = 0
    for n in names:
        mask |= 1 << all_names.index(n)
    L.check(lib.mg_profile_stages(mask), "mg_profile_stages")


def mg_profile_read(reset: bool = True) -> dict:
    """{stage name: (milliseconds, calls)} accumulated since the last reset."""
    lib = L.lib()
    n = lib.mg_profile_stage_count()
    ms = (ctypes.c_double * n)()
    calls = (ctypes.c_int64 * n)()
    L.check(lib.mg_profile_read(ms, calls, 1 if reset else 0), "mg_profile_read")
    return {lib.mg_profile_stage_name(i).decode(): (ms[i], int(calls[i])) for i in range(n)}


def mg_version() -> str:
    return L.lib().mg_version().decode()


# ---------------------------------------------------------------------------
# workspace management and autograd
# ---------------------------------------------------------------------------


class SliceRenderer:
    """Renders a fixed set of stacks; keeps the workspace between calls.

    Capacity: starts from ``records_per_gaussian`` records per Gaussian (or the
    exact bound n * slices when smaller) and 8 entries per record; when the
    device reports an overflow the forward is repeated with 1.25x the
    reported need. ``check`` reads the device counters after every forward
    (one stream synchronisation)."""

    def __init__(self, stacks: Sequence, device="cuda", cutoff_k: float = 3.0, f64_ratio: float = 16.0,
                 records_per_gaussian: int = 32, entries_per_record: int = 8, check: bool = True, cells=None):
        self.cells = cells
        self.dev = DeviceStacks(stacks, device)
        self.device = device
        self.K = cutoff_k
        self.f64_ratio = f64_ratio
        self.rpg = records_per_gaussian
        self.epr = entries_per_record
        self.check = check
        self.caps = None
        self.ws = None
        self.last_stats = None
        self._n = None

    def opts(self) -> L.MgOpts:
        return _opts(self.K, self.f64_ratio, self.caps[0], self.caps[1], self.cells)

    def _ensure(self, n: int):
        if self.caps is None or self._n != n:
            cr = max(1, min(n * self.dev.n_slices, self.rpg * n))
            self.caps = (cr, self.epr * cr)
            self._n = n
        need = mg_render_workspace_size(n, self.dev, self.opts())
        if self.ws is None or self.ws.numel() < need:
            self.ws = None
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)

    def set_capacity(self, records: int, entries: int, n: int):
        self.caps = (max(1, int(records)), max(1, int(entries)))
        self._n = n
        self._ensure(n)

    def forward(self, mean, quat, scale, alpha, out=None, stream=None):
        n = int(mean.shape[0])
        if out is None:
            out = torch.empty(self.dev.n_vox, dtype=_F32, device=mean.device)
        for _ in range(4):
            self._ensure(n)
            mg_render_fwd(mean, quat, scale, alpha, self.dev, self.opts(), out, self.ws, stream)
            if not self.check:
                return out
            st = mg_render_stats_get(self.ws, stream)
            self.last_stats = st
            if st["status"] == L.MG_OK:
                return out
            if st["status"] == L.MG_ERR_NOT_FINITE:
                raise L.MgError(L.MG_ERR_NOT_FINITE, "mg_render_fwd")
            self.caps = (max(self.caps[0], int(st["records"] * 1.25) + 1),
                         max(self.caps[1], int(st["entries"] * 1.25) + 1))
        raise L.MgError(L.MG_ERR_CAPACITY, "mg_render_fwd (after growing the workspace)")

    def forward_l1l2(self, mean, quat, scale, alpha, target, out, grad, loss_out, stream=None):
        """forward() with the L1 + L2 slice loss and its gradient fused into
        the evaluation kernel (same growth on capacity overflow)."""
        n = int(mean.shape[0])
        for _ in range(4):
            self._ensure(n)
            mg_render_fwd_l1l2(mean, quat, scale, alpha, self.dev, self.opts(), target, out, grad, loss_out, self.ws,
                               stream)
            if not self.check:
                return out
            st = mg_render_stats_get(self.ws, stream)
            self.last_stats = st
            if st["status"] == L.MG_OK:
                return out
            if st["status"] == L.MG_ERR_NOT_FINITE:
                raise L.MgError(L.MG_ERR_NOT_FINITE, "mg_render_fwd_l1l2")
            self.caps = (max(self.caps[0], int(st["records"] * 1.25) + 1),
                         max(self.caps[1], int(st["entries"] * 1.25) + 1))
        raise L.MgError(L.MG_ERR_CAPACITY, "mg_render_fwd_l1l2 (after growing the workspace)")

    def stats(self, stream=None) -> dict:
        return mg_render_stats_get(self.ws, stream)

    @property
    def status_word(self) -> torch.Tensor:
        """The device status word of the workspace (its first 32 bits)."""
        return self.ws[:4]

    def pair_count(self, mean, quat, scale, alpha, stream=None):
        """(pairs inside the K-sigma ellipsoid, evaluated pairs) of the last forward."""
        return mg_render_pair_count(mean, quat, scale, alpha, self.dev, self.opts(), self.ws, stream)

    def backward(self, mean, quat, scale, alpha, grad_out, stream=None, out=None):
        """dL/d(mean, quat, scale, alpha) for dL/dI = grad_out; ``out``: four
        contiguous FP32 tensors of shapes [n,3], [n,4], [n,3], [n] to write
        into (for example views of one flat buffer), else new ones."""
        n = int(mean.shape[0])
        if out is None:
            g = [torch.empty(n, 3, dtype=_F32, device=mean.device), torch.empty(n, 4, dtype=_F32, device=mean.device),
                 torch.empty(n, 3, dtype=_F32, device=mean.device), torch.empty(n, dtype=_F32, device=mean.device)]
        else:
            g = list(out)
            for t_, shp in zip(g, ((n, 3), (n, 4), (n, 3), (n,))):
                if tuple(t_.shape) != shp or t_.dtype != _F32 or not t_.is_contiguous() or t_.device != mean.device:
                    raise ValueError(f"backward(out=...): expected contiguous float32 {shp} on {mean.device}")
        st = mg_render_bwd(mean, quat, scale, alpha, self.dev, self.opts(), grad_out.contiguous(), *g, self.ws,
                           stream, raise_on_error=False)
        if st == L.MG_ERR_STALE_WORKSPACE:
            # the workspace was reused by another forward: rebuild its bins
            self.forward(mean, quat, scale, alpha)
            st = mg_render_bwd(mean, quat, scale, alpha, self.dev, self.opts(), grad_out.contiguous(), *g, self.ws,
                               stream, raise_on_error=False)
        L.check(st, "mg_render_bwd")
        return g

    def pose_grad(self, mean, quat, scale, alpha):
        """dL/d(slice pose) [slices, 6] of the loss whose dL/dI the last
        backward received: (dL/dt world, dL/domega slice frame)."""
        return _slice_pose_grad(self, mean, quat, scale, alpha)


class DeviceAdam:
    """Adam over parameter groups with the whole update in mg_adam_step (one
    launch, moments and step counter on the device, optional clamp and a
    device status predicate). Parameters keep their torch ``.grad``."""

    def __init__(self, groups: Sequence[dict], betas=(0.9, 0.999), eps: float = 1e-8):
        if not 1 <= len(groups) <= L.MG_ADAM_MAX_GROUPS:
            raise ValueError("1..8 parameter groups")
        self.groups = []
        for g in groups:
            p = g["param"]
            if not (p.is_cuda and p.dtype == _F32 and p.is_contiguous()):
                raise ValueError("parameters must be contiguous CUDA FP32 tensors")
            self.groups.append({"param": p, "lr": float(g["lr"]), "clamp": g.get("clamp"),
                                "m": torch.zeros_like(p), "v": torch.zeros_like(p)})
        self.betas, self.eps = (float(betas[0]), float(betas[1])), float(eps)
        self.step_t = torch.zeros(1, dtype=torch.int32, device=groups[0]["param"].device)

    def zero_grad(self):
        for g in self.groups:
            g["param"].grad = None

    def step(self, status=None, stream=None):
        gs = []
        for g in self.groups:
            p = g["param"]
            if p.grad is None:
                raise RuntimeError("a parameter has no gradient")
            gs.append({"param": p.data, "grad": p.grad.contiguous(), "m": g["m"], "v": g["v"], "lr": g["lr"],
                       "clamp": g["clamp"]})
        mg_adam_step(gs, self.betas[0], self.betas[1], self.eps, self.step_t, status, stream=stream)

    @property
    def steps(self) -> int:
        return int(self.step_t.item())


def _slice_pose_grad(renderer, mean, quat, scale, alpha):
    g = torch.empty(renderer.dev.n_slices, 6, dtype=_F32, device=mean.device)
    mg_render_pose_grad(mean, quat, scale, alpha, renderer.dev, renderer.opts(), g, renderer.ws)
    return g


class RenderSlices(torch.autograd.Function):
    """Slices of all stacks from Gaussians (mean, unit quat, scale, alpha)."""

    @staticmethod
    def forward(ctx, renderer: SliceRenderer, mean, quat, scale, alpha):
        mean, quat, scale, alpha = (t.detach().contiguous() for t in (mean, quat, scale, alpha))
        out = renderer.forward(mean, quat, scale, alpha)
        ctx.renderer = renderer
        ctx.save_for_backward(mean, quat, scale, alpha)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        mean, quat, scale, alpha = ctx.saved_tensors
        gm, gq, gs, ga = ctx.renderer.backward(mean, quat, scale, alpha, grad_out)
        return None, gm, gq, gs, ga


def render_slices(renderer: SliceRenderer, mean, quat_raw, log_scale, alpha):
    """The paper's parameterisation (Sec. 3.2): unnormalised quaternion and
    log-scale; normalisation and exp are taken in torch so autograd chains
    through them."""
    q = quat_raw / quat_raw.norm(dim=1, keepdim=True)
    return RenderSlices.apply(renderer, mean, q, torch.exp(log_scale), alpha)


class VolumeSampler:
    """Inference sampling onto the isotropic G^3 grid (mg_sample_volume)."""

    def __init__(self, G: int, spacing: float, centre=(0.0, 0.0, 0.0), device="cuda", cutoff_k: float = 3.0,
                 f64_ratio: float = 16.0, records_per_gaussian: int = 64, cells=None):
        self.cells = cells
        self.G, self.h, self.centre = int(G), float(spacing), tuple(float(c) for c in centre)
        self.device, self.K, self.f64 = device, cutoff_k, f64_ratio
        self.rpg = records_per_gaussian
        self.caps = None
        self.ws = None

    def __call__(self, mean, quat, scale, alpha, out=None, stream=None):
        n = int(mean.shape[0])
        if out is None:
            out = torch.empty(self.G ** 3, dtype=_F32, device=mean.device)
        if self.caps is None:
            cr = max(1, min(n * self.G, self.rpg * n))
            self.caps = (cr, 8 * cr)
        for _ in range(4):
            o = _opts(self.K, self.f64, *self.caps, cells=self.cells)
            need = mg_sample_workspace_size(n, self.G, o)
            if self.ws is None or self.ws.numel() < need:
                self.ws = None
                self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            mg_sample_volume(mean, quat, scale, alpha, self.centre, self.h, self.G, o, out, self.ws, stream)
            st = mg_render_stats_get(self.ws, stream)
            if st["status"] == L.MG_OK:
                self.last_stats = st
                return out.view(self.G, self.G, self.G)
            if st["status"] == L.MG_ERR_NOT_FINITE:
                raise L.MgError(L.MG_ERR_NOT_FINITE, "mg_sample_volume")
            self.caps = (max(self.caps[0], int(st["records"] * 1.25) + 1),
                         max(self.caps[1], int(st["entries"] * 1.25) + 1))
        raise L.MgError(L.MG_ERR_CAPACITY, "mg_sample_volume (after growing the workspace)")


# ---------------------------------------------------------------------------
# neural residual field
# ---------------------------------------------------------------------------
ENCODINGS = {"paper": L.MG_NRF_FOURIER, "grid": L.MG_NRF_GRID}
PRECISIONS = {"bf16": L.MG_NRF_BF16, "fp32": L.MG_NRF_FP32}


def mg_nrf_param_count(encoding: str) -> int:
    return int(L.lib().mg_nrf_param_count(ENCODINGS[encoding]))


class NRF:
    """Device parameters of a neural residual field (FP32 master copies) and
    the C-ABI calls on them. ``encoding``: "paper" (Fourier, 4 x 64 SiLU) or
    "grid" (hash grid, 2 x 64 ReLU); ``precision``: "bf16" or "fp32"."""

    def __init__(self, encoding: str, precision: str, weights, biases, table=None, device="cuda",
                 log2_table: int = 19, n_min: int = 16, n_max: int = 512, out_scale: float = 0.1):
        self.encoding, self.precision = encoding, precision
        flat = []
        for W, b in zip(weights, biases):
            flat.append(torch.as_tensor(W, dtype=_F32).reshape(-1))
            flat.append(torch.as_tensor(b, dtype=_F32).reshape(-1))
        self.params = torch.cat(flat).to(device).contiguous()
        if self.params.numel() != mg_nrf_param_count(encoding):
            raise ValueError(f"{encoding}: {self.params.numel()} parameters, expected {mg_nrf_param_count(encoding)}")
        self.table = None
        if encoding == "grid":
            self.table = torch.as_tensor(table, dtype=_F32).to(device).contiguous()
            if self.table.numel() != 16 * 2 * (1 << log2_table):
                raise ValueError("table must be [16, 2^log2_table, 2]")
        self.log2_table, self.n_min, self.n_max, self.out_scale = log2_table, n_min, n_max, out_scale

    def struct(self, params=None, table=None, enc=None, enc_mode: int = 0) -> L.MgNrf:
        p = self.params if params is None else params
        t = self.table if table is None else table
        return L.MgNrf(ENCODINGS[self.encoding], PRECISIONS[self.precision], _dev(p, "params"),
                       _dev(t, "table") if t is not None else None, self.log2_table, self.n_min, self.n_max,
                       float(self.out_scale), _dev(enc, "enc", torch.uint8) if enc is not None else None,
                       enc_mode if enc is not None else L.MG_NRF_ENC_NONE)

    def enc_cache(self, n: int, device=None):
        """A device buffer for the grid encoding of n points (None for the
        Fourier encoding): a forward call at rows stores the features into it,
        the backward call at the same rows reads them back instead of
        gathering the table again (mg_nrf.enc / enc_mode)."""
        s = self.struct()
        nb = int(L.lib().mg_nrf_enc_bytes(ctypes.byref(s), int(n)))
        if nb == 0:
            return None
        return torch.empty(nb, dtype=torch.uint8, device=device or self.params.device)


def mg_nrf_fwd(net: NRF, xyz, out, params=None, table=None, stream=None):
    n = xyz.numel() // 3
    _dev(xyz, "xyz", numel=3 * n)
    _dev(out, "out", numel=n)
    s = net.struct(params, table)
    L.check(L.lib().mg_nrf_fwd(ctypes.byref(s), xyz.data_ptr(), n, out.data_ptr(), _stream_handle(stream)),
            "mg_nrf_fwd")


def mg_nrf_bwd(net: NRF, xyz, grad_out, g_params, g_table=None, params=None, table=None, stream=None):
    n = xyz.numel() // 3
    _dev(xyz, "xyz", numel=3 * n)
    _dev(grad_out, "grad_out", numel=n)
    gp = _dev(g_params, "g_params", numel=mg_nrf_param_count(net.encoding))
    gt = _dev(g_table, "g_table") if g_table is not None else None
    s = net.struct(params, table)
    L.check(L.lib().mg_nrf_bwd(ctypes.byref(s), xyz.data_ptr(), n, grad_out.data_ptr(), gp, gt,
                               _stream_handle(stream)), "mg_nrf_bwd")


def _check_enc(net: NRF, enc, n: int):
    if enc is not None:
        need = int(L.lib().mg_nrf_enc_bytes(ctypes.byref(net.struct()), int(n)))
        if enc.numel() * enc.element_size() < need:
            raise ValueError(f"encoding cache holds {enc.numel() * enc.element_size()} bytes, {need} needed")


def mg_nrf_fwd_at(net: NRF, coords, idx, n: int, acc, params=None, table=None, stream=None, enc=None):
    """acc[idx[i]] += r(coords[idx[i]]) for i < n (the field at a batch of
    rows; indices outside [0, rows) are skipped). ``enc`` (NRF.enc_cache):
    the points' grid encoding is also stored there for mg_nrf_bwd_at."""
    rows = coords.numel() // 3
    _dev(coords, "coords", numel=3 * rows)
    _dev(acc, "acc", numel=rows)
    ip = _dev_idx(idx, n)
    _check_enc(net, enc, n)
    s = net.struct(params, table, enc, L.MG_NRF_ENC_STORE)
    L.check(L.lib().mg_nrf_fwd_at(ctypes.byref(s), coords.data_ptr(), rows, ip, n, acc.data_ptr(),
                                  _stream_handle(stream)), "mg_nrf_fwd_at")


def mg_nrf_bwd_at(net: NRF, coords, idx, n: int, grad_acc, g_params, g_table=None, params=None, table=None,
                  stream=None, enc=None):
    """Gradients of sum_i grad_acc[idx[i]] r(coords[idx[i]]) for the field's
    parameters (and table). ``enc``: the encoding a mg_nrf_fwd_at call stored
    for the same rows, read instead of gathering the table again."""
    rows = coords.numel() // 3
    _dev(coords, "coords", numel=3 * rows)
    _dev(grad_acc, "grad_acc", numel=rows)
    ip = _dev_idx(idx, n)
    gp = _dev(g_params, "g_params", numel=mg_nrf_param_count(net.encoding))
    gt = _dev(g_table, "g_table") if g_table is not None else None
    _check_enc(net, enc, n)
    s = net.struct(params, table, enc, L.MG_NRF_ENC_LOAD)
    L.check(L.lib().mg_nrf_bwd_at(ctypes.byref(s), coords.data_ptr(), rows, ip, n, grad_acc.data_ptr(), gp, gt,
                                  _stream_handle(stream)), "mg_nrf_bwd_at")


def _dev_idx(idx, n: int) -> int:
    if not (isinstance(idx, torch.Tensor) and idx.is_cuda and idx.dtype == torch.int64 and idx.is_contiguous()
            and idx.numel() >= n):
        raise ValueError(f"idx must be a contiguous CUDA int64 tensor with at least {n} entries")
    return idx.data_ptr()


class NRFFunction(torch.autograd.Function):
    """r = NRF(xyz) with gradients for the parameter vector (and grid table)."""

    @staticmethod
    def forward(ctx, net: NRF, xyz, params, table):
        xyz = xyz.detach().contiguous()
        out = torch.empty(xyz.numel() // 3, dtype=_F32, device=xyz.device)
        mg_nrf_fwd(net, xyz, out, params.detach(), None if table is None else table.detach())
        ctx.net = net
        ctx.save_for_backward(xyz, params, table if table is not None else torch.empty(0, device=xyz.device))
        ctx.has_table = table is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        xyz, params, table = ctx.saved_tensors
        table = table if ctx.has_table else None
        gp = torch.empty_like(params)
        gt = torch.empty_like(table) if table is not None else None
        mg_nrf_bwd(ctx.net, xyz, grad_out.contiguous(), gp, gt, params.detach(),
                   None if table is None else table.detach())
        return None, None, gp, gt
