"""GPU parity of the volume sampler and of the FP64 loss reductions."""
import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from oracle import metrics
from gpu_util import assert_render_close, to_dev

pytestmark = pytest.mark.gpu


def _sample(G, Gd, h, centre, K=3.0):
    from paper_2603_00145_b300 import VolumeSampler

    S = VolumeSampler(Gd, h, centre, cutoff_k=K)
    V = S(*to_dev(G))
    torch.cuda.synchronize()
    return S, V


@pytest.mark.parametrize("Gd,h", [(40, 0.8), (37, 1.1)])
def test_sampler_parity(Gd, h):
    G = ms.random_gaussians(400, 31, box=(-14, 14), sigma=(0.6, 2.5), aniso=3.0, negative_frac=0.1)
    centre = (0.3, -0.7, 1.1)
    S, V = _sample(G, Gd, h, centre)
    want = orc.sample_volume(G, Gd, h, centre)
    assert_render_close(V.cpu().numpy(), want, "sampler")
    # bins bit-exact
    from paper_2603_00145_b300.ops import mg_sample_ws_layout, read_bins, _opts

    st = S.last_stats
    lay = mg_sample_ws_layout(G.n, Gd, _opts(3.0, 100.0, *S.caps))
    gid, sl, rect, inset, toff, ent = read_bins(S.ws, lay, st["records"], st["tiles"], st["entries"])
    rec = orc.records(G, [orc.volume_planes(Gd, h, centre)])
    assert np.array_equal(gid.numpy(), rec.gid) and np.array_equal(sl.numpy(), rec.slice)
    assert np.array_equal(rect.numpy(), rec.rect)
    assert np.array_equal(inset.numpy().view(np.uint64), rec.inset)


def test_sampler_is_e7_and_conserves_mass():
    """With K = 6 the binned sampler equals the untruncated Eq. E7 mixture and
    h^3 * sum V equals the total mass (spacing <= sigma / 2)."""
    G = ms.random_gaussians(20, 8, box=(-3, 3), sigma=(1.2, 2.0), aniso=1.5)
    Gd, h = 64, 0.5
    S, V = _sample(G, Gd, h, (0.0, 0.0, 0.0), K=6.0)
    want = orc.sample_volume(G, Gd, h, (0.0, 0.0, 0.0), exact=True)
    assert_render_close(V.cpu().numpy(), want, "sampler K=6 vs exact")
    mass = sum(float(G.alpha[g]) * (2 * np.pi) ** 1.5 * float(np.prod(G.scale[g].astype(np.float64)))
               for g in range(G.n))
    assert abs(float(V.double().sum()) * h ** 3 / mass - 1.0) < 1e-5


@pytest.mark.parametrize("n", [1, 17, 4096 + 3, 1_000_003])
def test_loss_l1l2_parity(n):
    from paper_2603_00145_b300 import mg_loss_l1l2, mg_reduce_workspace_size

    rng = np.random.default_rng(n)
    p = rng.uniform(-0.5, 1.0, n).astype(np.float32)
    t = rng.uniform(0.0, 1.0, n).astype(np.float32)
    pd, td = torch.from_numpy(p).cuda(), torch.from_numpy(t).cuda()
    grad = torch.empty_like(pd)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    ws = torch.empty(mg_reduce_workspace_size(n), dtype=torch.uint8, device="cuda")
    mg_loss_l1l2(pd, td, grad, out, ws)
    loss, g = metrics.l1_l2(p, t)
    assert abs(float(out[0]) - loss) <= 2e-6 * abs(loss)
    assert np.max(np.abs(grad.cpu().numpy() - g)) <= 4 * np.finfo(np.float32).eps * np.max(np.abs(g))
    out2 = torch.empty_like(out)
    mg_loss_l1l2(pd, td, None, out2, ws)
    assert torch.equal(out, out2)  # deterministic


def test_sq_diff_sum_and_psnr():
    from paper_2603_00145_b300 import mg_reduce_workspace_size, mg_sq_diff_sum

    n = 64 ** 3 + 5
    rng = np.random.default_rng(3)
    a = rng.uniform(0, 1, n).astype(np.float32)
    b = (a + rng.normal(0, 0.01, n)).astype(np.float32)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(mg_reduce_workspace_size(n), dtype=torch.uint8, device="cuda")
    mg_sq_diff_sum(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), out, ws)
    ref = metrics.mse(a, b) * n
    assert abs(float(out[0]) - ref) <= 2e-6 * ref
    psnr = 10 * np.log10(1.0 / (float(out[0]) / n))
    assert abs(psnr - metrics.psnr(a, b)) < 1e-4
