"""GPU parity of the slice renderer (C ABI) against the FP64 oracle.

Records and tile bins must match the oracle bit for bit; rendered slices
within relative L2 1e-5 and max-abs 1e-4 of the intensity range; the adjoint
within relative L2 1e-4 per parameter group.
"""
import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from gpu_util import (assert_grads_close, assert_render_close, gpu_bins, render_gpu, sub_stacks, to_dev)

pytestmark = pytest.mark.gpu


def _mixed_case(seed, n=300, neg=0.1):
    rng = np.random.default_rng(seed)
    G = ms.random_gaussians(n, 200 + seed, box=(-22, 22), sigma=(0.6, 3.0), aniso=3.0, alpha=(0.1, 1.0),
                            negative_frac=neg)
    stacks = [ms.make_stack(ms.AXIAL, 9, 37, 50, 1.0, 1.1, 3.0, 3.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 7, 48, 40, 0.9, 0.9, 2.0, 2.5, rng=rng,
                            max_rot_deg=5.0, max_trans_mm=1.0),
              ms.make_stack(ms.SAGITTAL, 5, 33, 17, 1.3, 1.2, 0.0, 4.0)]
    return G, stacks


def _check_bins(G, stacks, R, K=3.0):
    rec = orc.records(G, stacks, K)
    st, (gid, sl, rect, inset, toff, ent) = gpu_bins(R, G.n)
    assert st["status"] == 0
    assert st["tiles"] == R.dev.n_tiles == sum(
        s.n_slices * -(-s.W // orc.TILE) * -(-s.H // orc.TILE) for s in stacks)
    assert st["records"] == rec.n
    assert np.array_equal(gid.numpy(), rec.gid) and np.array_equal(sl.numpy(), rec.slice)
    assert np.array_equal(rect.numpy(), rec.rect)
    assert np.array_equal(inset.numpy().view(np.uint64), rec.inset)
    counts, offs, ids = orc.tile_bins(rec, stacks)
    assert st["entries"] == ids.size
    assert np.array_equal(toff.numpy(), offs)
    ent = ent.numpy()
    for t in np.nonzero(counts)[0]:
        assert np.array_equal(np.sort(ent[offs[t]:offs[t + 1]]), ids[offs[t]:offs[t + 1]]), t
    return rec


def test_tiny_workload_fwd_bwd():
    """The 48^3 plain-method case: 3 orthogonal stacks of 16 slices, 48x48, 3 mm
    profile, 2048 devoxelised Gaussians; one FP32 forward + backward."""
    wl = ms.tiny_workload(0)
    vol = wl.phantom.volume()
    data = [ms.simulate_stack(vol, 1.0, s, seed=i, noise_sigma=wl.noise_sigma).numpy() for i, s in
            enumerate(wl.stacks)]
    G = ms.devoxelised_gaussians(wl.stacks, data, wl.n_gaussians, seed=0)
    R, out, dev = render_gpu(G, wl.stacks)
    rec = _check_bins(G, wl.stacks, R)
    want = orc.render(G, wl.stacks, rec)
    assert_render_close(out.cpu().numpy(), want, "tiny fwd")
    rng = np.random.default_rng(1)
    gout = rng.normal(size=want.size).astype(np.float32)
    g = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, wl.stacks, rec, gout.astype(np.float64))
    assert_grads_close(g, ref, G, "tiny")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mixed_stacks_fwd_bwd(seed):
    """Ragged sizes, an oblique stack with per-slice motion, a zero-thickness
    stack, negative intensities."""
    G, stacks = _mixed_case(seed)
    R, out, dev = render_gpu(G, stacks)
    rec = _check_bins(G, stacks, R)
    want = orc.render(G, stacks, rec)
    assert_render_close(out.cpu().numpy(), want, "mixed fwd")
    gout = np.random.default_rng(seed).normal(size=want.size).astype(np.float32)
    g = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, stacks, rec, gout.astype(np.float64))
    assert_grads_close(g, ref, G, "mixed")


@pytest.mark.parametrize("K", [2.0, 4.5])
def test_other_cutoffs(K):
    G, stacks = _mixed_case(7, n=150, neg=0.0)
    R, out, dev = render_gpu(G, stacks, K=K)
    rec = _check_bins(G, stacks, R, K=K)
    assert_render_close(out.cpu().numpy(), orc.render(G, stacks, rec), f"K={K}")


def test_deterministic_and_repeatable():
    G, stacks = _mixed_case(3)
    R, out1, dev = render_gpu(G, stacks)
    _, b1 = gpu_bins(R, G.n)
    out2 = R.forward(*dev)
    _, b2 = gpu_bins(R, G.n)
    assert torch.equal(out1, out2)
    for x, y in zip(b1, b2):
        assert torch.equal(x, y)


def test_large_records_listed_apart():
    """Records listing more than 16 tiles are binned apart from their chunks
    (at most 64 per chunk of 512 records; the rest stay in the chunk): a mix of
    large and small Gaussians on 96x112 slices, so that some chunks list fewer
    than 64 large records and others overflow. Bins, slices and gradients
    against the oracle; the tile lists repeat bit for bit."""
    rng = np.random.default_rng(11)
    big = ms.random_gaussians(700, 31, box=(-30, 30), sigma=(5.0, 12.0), aniso=2.0, alpha=(0.05, 0.3))
    small = ms.random_gaussians(1300, 32, box=(-40, 40), sigma=(0.6, 2.0), aniso=2.0, alpha=(0.1, 1.0),
                                negative_frac=0.1)
    order = rng.permutation(2000)
    G = ms.Gaussians(*(np.concatenate([getattr(big, f), getattr(small, f)])[order]
                       for f in ("mean", "quat", "scale", "alpha")))
    stacks = [ms.make_stack(ms.AXIAL, 6, 96, 112, 1.0, 1.0, 2.0, 6.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 5, 90, 96, 1.1, 1.0, 3.0, 7.0, rng=rng,
                            max_rot_deg=4.0, max_trans_mm=1.0)]
    R, out, dev = render_gpu(G, stacks)
    rec = _check_bins(G, stacks, R)
    area = np.array([len(rec.row_tiles(r)) for r in range(rec.n)])
    per_chunk = [np.count_nonzero(a[c:c + 512] > 16) for a in (area[rec.slice == k] for k in np.unique(rec.slice))
                 for c in range(0, a.size, 512)]
    assert 0 < min(per_chunk) < 64 < max(per_chunk), per_chunk  # both sides of the per-chunk list limit
    want = orc.render(G, stacks, rec)
    assert_render_close(out.cpu().numpy(), want, "large records fwd")
    gout = np.random.default_rng(12).normal(size=want.size).astype(np.float32)
    g = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, stacks, rec, gout.astype(np.float64))
    assert_grads_close(g, ref, G, "large records")
    _, b1 = gpu_bins(R, G.n)
    R.forward(*dev)
    _, b2 = gpu_bins(R, G.n)
    for x, y in zip(b1, b2):
        assert torch.equal(x, y)


def test_sparse_tiles_packed_backward():
    """Tiles holding a handful of records (a fitted model's background): the
    backward takes the tiles of at most 16 records eight at a time and packs
    their records into batches of up to 32 lanes, each lane over all rows of
    its own tile. 16k busy tiles, all sparse; bins, slices and gradients
    against the oracle."""
    G = ms.random_gaussians(6000, 41, box=(-60, 60), sigma=(0.5, 1.6), aniso=2.0, alpha=(0.1, 1.0),
                            negative_frac=0.1)
    rng = np.random.default_rng(42)
    stacks = [ms.make_stack(ms.AXIAL, 24, 128, 128, 1.0, 1.0, 2.0, 5.0),
              ms.make_stack(ms.CORONAL, 24, 120, 128, 1.0, 1.0, 2.0, 5.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 24, 128, 120, 1.0, 1.0, 2.0, 5.0, rng=rng,
                            max_rot_deg=3.0, max_trans_mm=1.0)]
    R, out, dev = render_gpu(G, stacks)
    rec = _check_bins(G, stacks, R)
    counts = orc.tile_bins(rec, stacks)[0]
    assert np.count_nonzero(counts) > 12000 and counts.max() <= 16
    want = orc.render(G, stacks, rec)
    assert_render_close(out.cpu().numpy(), want, "sparse tiles fwd")
    gout = np.random.default_rng(43).normal(size=want.size).astype(np.float32)
    g = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, stacks, rec, gout.astype(np.float64))
    assert_grads_close(g, ref, G, "sparse tiles")


def test_backward_into_caller_buffers():
    """backward(out=...) writes the gradients into given tensors (here views of
    one flat buffer, as a host round trip would use) and matches the default
    call (up to the FP32 order of the moment atomics); a tensor of the wrong
    shape is refused."""
    G, stacks = _mixed_case(4)
    R, out, dev = render_gpu(G, stacks)
    gout = torch.from_numpy(np.random.default_rng(4).normal(size=out.numel()).astype(np.float32)).cuda()
    g = R.backward(*dev, gout)
    n = G.n
    flat = torch.full((11 * n,), float("nan"), dtype=torch.float32, device="cuda")
    views = [flat[0:3 * n].view(n, 3), flat[3 * n:7 * n].view(n, 4), flat[7 * n:10 * n].view(n, 3), flat[10 * n:]]
    g2 = R.backward(*dev, gout, out=views)
    for a, b in zip(g, g2):
        assert torch.isfinite(b).all()
        assert (a - b).abs().max() <= 1e-5 * a.abs().max()
    assert g2[0].data_ptr() == flat.data_ptr()
    with pytest.raises(ValueError):
        R.backward(*dev, gout, out=[views[1], views[0], views[2], views[3]])


def test_capacity_overflow_then_growth():
    from paper_2603_00145_b300 import SliceRenderer
    from paper_2603_00145_b300.ops import mg_render_fwd, mg_render_stats_get

    G, stacks = _mixed_case(4)
    R = SliceRenderer(stacks, check=False)
    R.set_capacity(7, 20, G.n)
    m, q, s, a = to_dev(G)
    out = torch.empty(R.dev.n_vox, device="cuda")
    mg_render_fwd(m, q, s, a, R.dev, R.opts(), out, R.ws)
    st = mg_render_stats_get(R.ws)
    assert st["status"] == 3 and st["records"] > 7  # MG_ERR_CAPACITY with the need reported
    R2 = SliceRenderer(stacks)
    R2.set_capacity(7, 20, G.n)
    out2 = R2.forward(m, q, s, a)  # grows and retries
    assert_render_close(out2.cpu().numpy(), orc.render(G, stacks), "after growth")


def test_empty_and_outside():
    from paper_2603_00145_b300 import SliceRenderer

    stacks = [ms.make_stack(ms.AXIAL, 3, 20, 21, 1.0, 1.0, 3.0, 3.0)]
    R = SliceRenderer(stacks)
    e = torch.empty(0, 3, device="cuda")
    out = R.forward(e, torch.empty(0, 4, device="cuda"), e.clone(), torch.empty(0, device="cuda"))
    assert out.numel() == 3 * 20 * 21 and float(out.abs().max()) == 0.0
    G = ms.random_gaussians(50, 5, box=(200, 300))  # far outside the field of view
    _, out, _ = render_gpu(G, stacks)
    assert float(out.abs().max()) == 0.0


def test_not_finite_reported():
    from paper_2603_00145_b300 import SliceRenderer
    from paper_2603_00145_b300.ops import mg_render_fwd, mg_render_stats_get

    G, stacks = _mixed_case(5, n=40)
    G.mean[3, 1] = np.nan
    G.scale[7, 0] = 0.0
    R = SliceRenderer(stacks, check=False)
    R._ensure(G.n)
    m, q, s, a = to_dev(G)
    out = torch.empty(R.dev.n_vox, device="cuda")
    mg_render_fwd(m, q, s, a, R.dev, R.opts(), out, R.ws)
    assert mg_render_stats_get(R.ws)["status"] == 5  # MG_ERR_NOT_FINITE
    # the remaining Gaussians still render exactly as without the bad ones
    keep = np.setdiff1d(np.arange(G.n), [3, 7])
    assert np.isfinite(out.cpu().numpy()).all()
    want = orc.render(G.subset(keep), stacks)
    assert_render_close(out.cpu().numpy(), want, "bad inputs skipped")


def test_backward_requires_matching_forward():
    from paper_2603_00145_b300 import SliceRenderer
    from paper_2603_00145_b300 import _lib as L
    from paper_2603_00145_b300.ops import mg_render_bwd

    G, stacks = _mixed_case(6, n=30)
    R = SliceRenderer(stacks)
    R._ensure(G.n)
    m, q, s, a = to_dev(G)
    g = [torch.empty(G.n, 3, device="cuda"), torch.empty(G.n, 4, device="cuda"), torch.empty(G.n, 3, device="cuda"),
         torch.empty(G.n, device="cuda")]
    go = torch.zeros(R.dev.n_vox, device="cuda")
    st = mg_render_bwd(m, q, s, a, R.dev, R.opts(), go, *g, R.ws, raise_on_error=False)
    assert st == L.MG_ERR_STALE_WORKSPACE


def test_degenerate_gaussians_fp64_geometry():
    """Needle/pancake Gaussians (scale ratio up to 400) take the FP64 record
    geometry; bins stay bit-exact and values stay within tolerance."""
    rng = np.random.default_rng(9)
    G = ms.random_gaussians(120, 77, box=(-15, 15), sigma=(0.5, 2.0), aniso=1.5)
    sc = G.scale.copy()
    for i in range(0, G.n, 2):
        ax = rng.integers(3)
        sc[i, ax] *= rng.uniform(20, 60)
        sc[i, (ax + 1) % 3] /= rng.uniform(3, 8)
    G = ms.Gaussians(G.mean, G.quat, sc, G.alpha)
    stacks = [ms.make_stack(ms.AXIAL, 8, 40, 40, 0.8, 0.8, 2.0, 2.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 6, 36, 44, 0.9, 0.9, 2.0, 3.0)]
    R, out, dev = render_gpu(G, stacks)
    rec = _check_bins(G, stacks, R)
    assert_render_close(out.cpu().numpy(), orc.render(G, stacks, rec), "degenerate fwd")


def _needles(G, every, factor, seed):
    """Every ``every``-th Gaussian stretched by ``factor`` along one axis: a
    scale ratio above the FP64 threshold (near-degenerate covariance)."""
    rng = np.random.default_rng(seed)
    sc = G.scale.copy()
    idx = np.arange(0, G.n, every)
    sc[idx, rng.integers(3, size=idx.size)] *= factor
    return ms.Gaussians(G.mean, G.quat, sc, G.alpha)


def _anisotropic(G, seed):
    """The workload's isotropic initial Gaussians given random orientations and
    per-axis scale factors in [0.6, 1.6] (a fitted model's shapes): the
    quaternion gradient of an isotropic Gaussian is identically zero, so it
    would check nothing."""
    rng = np.random.default_rng(seed)
    q = ms.random_unit_quats(G.n, rng).astype(np.float32)
    sc = (G.scale * rng.uniform(0.6, 1.6, size=G.scale.shape)).astype(np.float32)
    return ms.Gaussians(G.mean, q, sc, G.alpha)


@pytest.mark.parametrize("lo,hi", [(4.0, 15.0), (20.0, 90.0)])
def test_elongated_gaussians_fp32_path(lo, hi):
    """Gaussians with scale ratios in [lo, hi] kept on the FP32 path (the FP64
    threshold raised from its default 16 to 100): the backward's single sweep
    of the rows (ratios up to 16) and its centre-out sums (above 16, where the
    chain amplifies moment errors) both hold the gradient bounds, element-wise,
    against the FP64 oracle; oblique moving, PSF and profile stacks."""
    rng = np.random.default_rng(int(lo))
    n = 400
    G0 = ms.random_gaussians(n, 60 + int(lo), box=(-18, 18), sigma=(0.5, 1.2), aniso=1.0, alpha=(0.1, 1.0),
                             negative_frac=0.1)
    sc = G0.scale.copy()
    sc[np.arange(n), rng.integers(3, size=n)] *= rng.uniform(lo, hi, size=n).astype(np.float32)
    G = ms.Gaussians(G0.mean, G0.quat, sc, G0.alpha)
    ratio = sc.max(1) / sc.min(1)
    assert ratio.max() < 100.0 and ratio.min() > lo * 0.5
    stacks = [ms.make_stack(ms.AXIAL, 8, 40, 44, 1.0, 1.0, 2.5, 3.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 7, 44, 40, 1.0, 1.0, 2.0, 3.5, rng=rng, max_rot_deg=5.0,
                            max_trans_mm=1.0),
              ms.make_stack(ms.CORONAL, 6, 36, 40, 1.0, 1.0, 3.0, 4.0, psf_u=0.8, psf_v=0.6)]
    R, out, dev = render_gpu(G, stacks, f64_ratio=100.0)
    rec = _check_bins(G, stacks, R)
    want = orc.render(G, stacks, rec)
    assert_render_close(out.cpu().numpy(), want, f"ratio {lo}-{hi} fwd")
    gout = np.random.default_rng(int(hi)).normal(size=want.size).astype(np.float32)
    g = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, stacks, rec, gout.astype(np.float64))
    assert_grads_close(g, ref, G, f"ratio {lo}-{hi}")


@pytest.mark.parametrize("name", ["feta", "motion", "stress"])
def test_bench_config_sampled_slices(name):
    """The workloads at full size, in the bench's launch configuration:
    FeTA-shaped (200k Gaussians; 3 x 64 slices of 256^2), motion (500k
    Gaussians; 4 stacks of 64 x 256^2, one oblique, per-slice motion <= 3 deg)
    and stress (2M Gaussians; 5 stacks of 96 x 384^2 at random orientations,
    motion <= 5 deg, one Gaussian in 500 stretched 150x onto the FP64
    geometry path), each Gaussian given a random orientation and per-axis
    scales. The GPU renders everything; the oracle checks one slice per stack,
    and the adjoint with dL/dI non-zero on those slices only."""
    maker = {"feta": ms.feta_workload, "motion": ms.motion_workload, "stress": ms.stress_workload}[name]
    wl = maker(0)
    G = _anisotropic(ms.phantom_init_gaussians(wl, seed=0), 3)
    if name == "stress":
        G = _needles(G, 500, 150.0, 5)
    R, out, dev = render_gpu(G, wl.stacks)
    picks = [(i, (17 + 13 * i) % s.n_slices) for i, s in enumerate(wl.stacks)]
    sub, ranges = sub_stacks(wl.stacks, picks)
    rec = orc.records(G, sub)
    want = orc.render(G, sub, rec)
    got = np.concatenate([out[a:b].cpu().numpy() for a, b in ranges])
    r, m = assert_render_close(got, want, f"{name} slices")
    gout_sub = np.random.default_rng(2).normal(size=want.size).astype(np.float32)
    gout = torch.zeros(R.dev.n_vox, device="cuda")
    o = 0
    for a, b in ranges:
        gout[a:b] = torch.from_numpy(gout_sub[o:o + b - a]).cuda()
        o += b - a
    g = R.backward(*dev, gout)
    ref = orc.grad(G, sub, rec, gout_sub.astype(np.float64))
    ge = assert_grads_close(g, ref, G, f"{name} slices")
    print(f"{name}: slices rel-L2 {r:.2e} max-abs {m:.2e}; grads " +
          " ".join(f"{k} {v:.2e}" for k, v in ge.items()))


def test_fitted_model_sampled_slices():
    """The FeTA-shaped workload at full size on the Gaussians a reconstruction
    iterates on: the 200k grid-initialised Gaussians after 2000 L1+L2 Adam
    iterations of the fit (a few grown over whole slices, most tiles holding a
    handful of records, so the sparse-tile and large-record paths carry the
    step). The GPU renders everything; the oracle checks one slice per stack
    and the adjoint with dL/dI non-zero on those slices only."""
    from paper_2603_00145_b300 import recon

    wl = ms.feta_workload(0)
    vol = wl.phantom.volume_torch(device="cuda")
    data = [ms.simulate_stack(vol, wl.phantom.spacing, s, seed=i, noise_sigma=wl.noise_sigma, device="cuda")
            for i, s in enumerate(wl.stacks)]
    del vol
    target = torch.cat([d_.reshape(-1) for d_ in data]).contiguous()
    G0 = ms.phantom_init_gaussians(wl, seed=0)
    model, _, _ = recon.fit(wl.stacks, target, G0, (0.0, 0.0, 0.0), wl.phantom.fov_mm / 2,
                            recon.FitConfig(iterations=2000, log_every=0), device="cuda")
    with torch.no_grad():
        G = ms.Gaussians(*(x.detach().float().contiguous().cpu().numpy() for x in model.gaussians()))
    del model, target, data
    R, out, dev = render_gpu(G, wl.stacks)
    assert R.stats()["records"] > 0
    picks = [(i, (17 + 13 * i) % s.n_slices) for i, s in enumerate(wl.stacks)]
    sub, ranges = sub_stacks(wl.stacks, picks)
    rec = orc.records(G, sub)
    want = orc.render(G, sub, rec)
    got = np.concatenate([out[a:b].cpu().numpy() for a, b in ranges])
    r, m = assert_render_close(got, want, "fitted slices")
    gout_sub = np.random.default_rng(2).normal(size=want.size).astype(np.float32)
    gout = torch.zeros(R.dev.n_vox, device="cuda")
    o = 0
    for a, b in ranges:
        gout[a:b] = torch.from_numpy(gout_sub[o:o + b - a]).cuda()
        o += b - a
    g = R.backward(*dev, gout)
    ref = orc.grad(G, sub, rec, gout_sub.astype(np.float64))
    ge = assert_grads_close(g, ref, G, "fitted slices")
    print(f"fitted: slices rel-L2 {r:.2e} max-abs {m:.2e}; grads " +
          " ".join(f"{k} {v:.2e}" for k, v in ge.items()))


def test_k6_slices_equal_untruncated_sum():
    """At K = 6 every omitted term is below exp(-18) ~ 1.5e-8 of its
    Gaussian's peak, so the slices must equal the untruncated profile-integrated
    sum over every Gaussian at every pixel (the oracle's ``exact`` render:
    no records, tiles or culling rule involved), within the render tolerance.
    Thick-profile, in-plane PSF, zero-thickness and an oblique stack with
    per-slice motion; a quarter of the Gaussians take the FP64 geometry."""
    rng = np.random.default_rng(61)
    G = ms.random_gaussians(320, 610, box=(-20, 20), sigma=(0.5, 2.5), aniso=3.0, negative_frac=0.1)
    G = _needles(G, 4, 130.0, 62)
    stacks = [ms.make_stack(ms.AXIAL, 7, 37, 45, 1.0, 1.1, 3.0, 3.0, psf_u=1.2, psf_v=0.8),
              ms.make_stack(ms.random_rotations(1, rng)[0], 6, 40, 34, 0.9, 0.9, 2.0, 2.5, rng=rng,
                            max_rot_deg=3.0, max_trans_mm=1.0),
              ms.make_stack(ms.axis_angle_matrix([1, 0, 0], np.deg2rad(30.0)) @ ms.CORONAL, 5, 29, 41, 1.0, 1.0,
                            2.0, 2.0, rng=rng, max_rot_deg=3.0, max_trans_mm=1.0, psf_u=0.0, psf_v=1.5),
              ms.make_stack(ms.SAGITTAL, 4, 30, 18, 1.3, 1.2, 0.0, 4.0)]
    R, out, dev = render_gpu(G, stacks, K=6.0)
    want = orc.render(G, stacks, exact=True)
    r, m = assert_render_close(out.cpu().numpy(), want, "K=6 vs untruncated")
    print(f"K=6 vs untruncated: rel-L2 {r:.2e} max-abs {m:.2e}")


def test_pair_counts_vs_oracle():
    """Evaluated pairs are an exact integer function of the bins; pairs inside
    the K-sigma ellipsoid agree up to FP32-vs-FP64 boundary decisions."""
    G, stacks = _mixed_case(8)
    R, out, dev = render_gpu(G, stacks)
    inside, evald = R.pair_count(*dev)
    rec = orc.records(G, stacks)
    o_in, o_ev = orc.pair_counts(G, stacks, rec)
    assert evald == o_ev
    assert abs(inside - o_in) <= max(2, 1e-4 * o_in), (inside, o_in)
    assert 0 < inside < evald


@pytest.mark.parametrize("seed", [0, 1])
def test_in_plane_psf_stacks_fwd_bwd(seed):
    """Full 3-D PSF (slice profile + in-plane Gaussian PSF): bins bit-exact,
    slices and gradients within tolerance, near-degenerate Gaussians included."""
    rng = np.random.default_rng(40 + seed)
    G = ms.random_gaussians(300, 500 + seed, box=(-20, 20), sigma=(0.5, 3.0), aniso=3.0, negative_frac=0.1)
    sc = G.scale.copy()
    for i in range(0, G.n, 7):
        sc[i, rng.integers(3)] *= 150.0   # FP64 record geometry
    G = ms.Gaussians(G.mean, G.quat, sc, G.alpha)
    stacks = [ms.make_stack(ms.AXIAL, 6, 37, 45, 1.0, 1.1, 3.0, 3.0, psf_u=1.2, psf_v=0.9),
              ms.make_stack(ms.random_rotations(1, rng)[0], 5, 40, 36, 0.9, 0.9, 2.0, 2.5, rng=rng,
                            max_rot_deg=5.0, max_trans_mm=1.0, psf_u=0.0, psf_v=1.5),
              ms.make_stack(ms.SAGITTAL, 4, 30, 18, 1.3, 1.2, 0.0, 4.0, psf_u=2.0, psf_v=2.0)]
    R, out, dev = render_gpu(G, stacks)
    rec = _check_bins(G, stacks, R)
    want = orc.render(G, stacks, rec)
    assert_render_close(out.cpu().numpy(), want, "psf fwd")
    gout = rng.normal(size=want.size).astype(np.float32)
    g = R.backward(*dev, torch.from_numpy(gout).cuda())
    ref = orc.grad(G, stacks, rec, gout.astype(np.float64))
    assert_grads_close(g, ref, G, "psf")
