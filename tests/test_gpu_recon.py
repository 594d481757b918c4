"""End-to-end reconstruction on the GPU (Sec. 3.1, 3.4, 3.5): the fit
lowers the slice loss and reaches a volume PSNR against the phantom; the
neural residual field trained on the Gaussian render's residuals raises it;
the BF16 field matches the FP32 one."""
import numpy as np
import pytest
import torch

import mg_synth as ms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    wl = ms.tiny_workload(0)
    vol = wl.phantom.volume_torch(device="cuda")
    data = [ms.simulate_stack(vol, 1.0, s, seed=i, noise_sigma=wl.noise_sigma, device="cuda")
            for i, s in enumerate(wl.stacks)]
    target = torch.cat([d.reshape(-1) for d in data]).contiguous()
    G = ms.devoxelised_gaussians(wl.stacks, [d.cpu().numpy() for d in data], wl.n_gaussians, seed=0)
    return wl, vol, target, G


def _run(tiny, **kw):
    from paper_2603_00145_b300 import recon

    wl, vol, target, G = tiny
    cfg = recon.FitConfig(iterations=600, log_every=100, **kw)
    m, nrf, st = recon.fit(wl.stacks, target, G, (0, 0, 0), wl.phantom.fov_mm / 2, cfg)
    V = recon.sample(m, nrf, 48, 1.0)
    return recon.psnr(V, vol), st


def test_fit_lowers_loss_and_reconstructs(tiny):
    p, st = _run(tiny)
    losses = [l for _, l in st["history"]]
    assert losses[-1] < 0.5 * losses[0], losses
    assert p > 22.0, p


def test_nrf_gain_and_bf16_matches_fp32(tiny):
    """What the residual field adds: the same 600 iterations with the field
    switched on at 300 (hash-grid encoding, trained on the residuals of the
    Gaussian render) against the Gaussians alone."""
    p_plain, _ = _run(tiny)
    p_bf16, _ = _run(tiny, nrf="grid", nrf_start=300, nrf_batch=1 << 16)
    p_fp32, _ = _run(tiny, nrf="grid", nrf_precision="fp32", nrf_start=300, nrf_batch=1 << 16)
    print(f"volume PSNR: Gaussians {p_plain:.3f} dB, + NRF BF16 {p_bf16:.3f} dB, + NRF FP32 {p_fp32:.3f} dB")
    assert p_bf16 > p_plain + 0.2, (p_plain, p_bf16)
    assert abs(p_bf16 - p_fp32) < 0.1, (p_bf16, p_fp32)
