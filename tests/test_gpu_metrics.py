"""Image-quality metrics (Section 3, Eqs. 10-12) on the GPU vs the oracle.

Both sides read the same FP32 images (the GPU's own envelope output, copied
to the host for the oracle), so pixel counts, peak positions and histogram
bins must agree exactly, and the FP64 statistics to rounding.
"""

import math

import numpy as np
import pytest

import synth
from gpu_util import run_gpu
from oracle import metrics as om

pytestmark = pytest.mark.gpu

EXACT = ("n_in", "n_out", "peak_j", "peak_l", "peak")
CLOSE = ("mu_in", "mu_out", "sigma_out", "snr_db", "cr_db", "gcnr", "fwhm_m")


def _random_rois(grid, n, seed):
    rng = np.random.default_rng(seed)
    w = grid["x1_m"] - grid["x0_m"]
    h = grid["z1_m"] - grid["z0_m"]
    rois = []
    for i in range(n):
        xc = grid["x0_m"] + rng.uniform(-0.1, 1.1) * w  # some centres off the image
        zc = grid["z0_m"] + rng.uniform(-0.1, 1.1) * h
        r = rng.uniform(0.01, 0.12) * min(w, h)
        kind = i % 3
        if kind == 0:
            t = dict(shape="disc", xc_m=xc, zc_m=zc, a_m=r)
            b = dict(shape="annulus", xc_m=xc, zc_m=zc, a_m=1.5 * r, b_m=2.5 * r)
        elif kind == 1:
            t = dict(shape="rect", xc_m=xc, zc_m=zc, a_m=r, b_m=0.5 * r)
            b = dict(shape="rect", xc_m=xc + 3 * r, zc_m=zc, a_m=r, b_m=2 * r)
        else:
            t = dict(shape="disc", xc_m=xc, zc_m=zc, a_m=r)
            b = dict(shape="rect", xc_m=grid["x0_m"] + 0.5 * w, zc_m=grid["z0_m"] + 0.5 * h,
                     a_m=0.5 * w, b_m=0.5 * h)  # the whole image
        rois.append((t, b))
    # an empty target (far outside) and an empty background
    rois.append((dict(shape="disc", xc_m=grid["x0_m"] - w, zc_m=zc, a_m=r), rois[0][1]))
    rois.append((rois[0][0], dict(shape="annulus", xc_m=xc, zc_m=zc, a_m=r, b_m=r)))
    return rois


def _gpu_metrics(images, grid, rois):
    import torch

    import paper_2203_14906_gb300 as pa

    t = torch.from_numpy(np.ascontiguousarray(images, dtype=np.float32)).cuda()
    return pa.image_metrics(t, grid, rois)


def _assert_same(gpu, ref, what=""):
    for f in EXACT:
        g, r = gpu[f], ref[f]
        both_nan = np.isnan(g.astype(float)) & np.isnan(r.astype(float))
        assert np.array_equal(g[~both_nan], r[~both_nan]), (what, f)
    for f in CLOSE:
        g, r = gpu[f], ref[f]
        assert np.array_equal(np.isnan(g), np.isnan(r)), (what, f)
        assert np.array_equal(np.isinf(g), np.isinf(r)), (what, f)
        ok = np.isfinite(r)
        assert np.allclose(g[ok], r[ok], rtol=1e-12, atol=1e-12), (what, f)


def test_envelope_images_match_oracle_exactly():
    """cfg1 envelope images (2 frames x 3 outputs), 32 ROI pairs of every
    shape, including regions off the image, a whole-image background and
    empty regions."""
    wl = synth.workload("cfg1")
    rf = np.stack([synth.make_frame(wl, s) for s in (1, 2)])
    out, _, _ = run_gpu(wl, rf, 3, stages=2)  # ENV only: [2][1][3][nx][nz]
    images = out[:, 0]
    rois = _random_rois(wl, 30, seed=5)
    gpu = _gpu_metrics(images, wl, rois)
    ref = om.metrics_batch(wl, images, rois)
    _assert_same(gpu, ref, "cfg1 env")
    assert np.all(gpu["n_in"][:, -2] == 0) and np.isnan(gpu["mu_in"][0, -2])
    assert np.all(gpu["n_out"][:, -1] == 0) and np.isnan(gpu["sigma_out"][0, -1])
    assert np.isfinite(gpu["gcnr"][:, :30]).sum() > 20


def test_constructed_images_closed_forms():
    grid = dict(nx=32, nz=32, x0_m=0.0, x1_m=3.2e-3, z0_m=0.0, z1_m=3.2e-3)
    dx = 1e-4
    rect = lambda j0, j1, l0, l1: dict(shape="rect", xc_m=(j0 + j1) / 2 * dx,  # noqa: E731
                                       zc_m=(l0 + l1) / 2 * dx, a_m=(j1 - j0) / 2 * dx,
                                       b_m=(l1 - l0) / 2 * dx)
    img = np.zeros((2, 32, 32), dtype=np.float32)
    img[0, 2:6, 2:6] = 4.0
    img[0, 10:20, 5:15] = np.where(np.arange(10, 20) % 2 == 0, 1.0, 3.0)[:, None]
    img[1, :, 7] = np.maximum(0.0, 1.0 - np.abs(np.arange(32) - 15) / 8.0)
    rois = [(rect(2, 6, 2, 6), rect(10, 20, 5, 15)), (rect(12, 18, 5, 10), rect(0, 4, 20, 30))]
    g = _gpu_metrics(img, grid, rois)
    assert g["n_in"][0, 0] == 16 and g["n_out"][0, 0] == 100
    assert g["mu_out"][0, 0] == 2.0 and g["sigma_out"][0, 0] == 1.0
    assert g["snr_db"][0, 0] == pytest.approx(40 * math.log10(2.0), abs=1e-12)
    assert g["cr_db"][0, 0] == pytest.approx(20 * math.log10(2.0), abs=1e-12)
    assert g["fwhm_m"][1, 1] == pytest.approx(8 * dx, rel=1e-12)
    assert g["gcnr"][0, 0] == 1.0


def test_many_images_and_pairs_across_launch_chunks():
    """8 images x 2100 ROI pairs (more pairs than one launch sequence takes):
    sampled pairs against the oracle, and two calls give identical bits."""
    import torch

    import paper_2203_14906_gb300 as pa

    grid = dict(nx=200, nz=300, x0_m=-10e-3, x1_m=10e-3, z0_m=1e-3, z1_m=31e-3)
    rng = np.random.default_rng(11)
    images = rng.gamma(2.0, 1.0, (8, 200, 300)).astype(np.float32)
    rois = _random_rois(grid, 2100, seed=12)
    t = torch.from_numpy(images).cuda()
    a = pa.image_metrics(t, grid, rois)
    b = pa.image_metrics(t, grid, rois)
    for f in a:
        assert np.array_equal(a[f], b[f], equal_nan=True), f
    pick = rng.choice(len(rois), 60, replace=False)
    sub = [rois[i] for i in pick]
    ref = om.metrics_batch(grid, images, sub)
    _assert_same({f: a[f][:, pick] for f in a}, ref, "chunked")


def test_fwhm_falls_with_order_through_the_gpu_path():
    """Section 3's claim on GPU-beamformed images of a point absorber (odd
    orders in the fundamental band, even orders in the harmonic band)."""
    wl = synth.workload("cfg1", nx=257, nz=256, noise_frac=0.0, x0_m=-6.425e-3, x1_m=6.425e-3)
    l0 = 160
    zs = wl["z0_m"] + (l0 + 0.5) * (wl["z1_m"] - wl["z0_m"]) / wl["nz"]
    rf = synth.render_rf(wl, synth.point_scene([0.0], [zs]))[None]
    roi = [(dict(shape="disc", xc_m=0.0, zc_m=zs, a_m=1.0e-3),
            dict(shape="annulus", xc_m=0.0, zc_m=zs, a_m=2.5e-3, b_m=4.0e-3))]
    w = {}
    for k in (3, 4, 5):
        out, _, _ = run_gpu(wl, rf, k, stages=2)
        m = _gpu_metrics(out[0, 0], wl, roi)  # DAS, DMAS, DMAS-k
        if k == 3:
            w[1], w[2] = m["fwhm_m"][0, 0], m["fwhm_m"][1, 0]
        w[k] = m["fwhm_m"][2, 0]
        assert m["peak_j"][2, 0] == 128 and m["peak_l"][2, 0] == l0
    assert w[1] > w[3] > w[5] > 0 and w[2] > w[4] > 0


def test_region_membership_on_exact_boundaries():
    """Centres on pixel centres and radii of whole pixel steps (pixel centres
    lying exactly on region boundaries), on grids with ragged sizes: the GPU's
    per-column row intervals give exactly the oracle's pixel sets."""
    rng = np.random.default_rng(21)
    for trial in range(12):
        nx, nz = int(rng.integers(3, 90)), int(rng.integers(3, 90))
        grid = dict(nx=nx, nz=nz, x0_m=-1e-3, x1_m=-1e-3 + nx * 1e-4, z0_m=2e-3,
                    z1_m=2e-3 + nz * 1e-4)
        rois = []
        for _ in range(40):
            xc = grid["x0_m"] + (int(rng.integers(-3, nx + 3)) + 0.5) * 1e-4
            zc = grid["z0_m"] + (int(rng.integers(-3, nz + 3)) + 0.5) * 1e-4
            a = int(rng.integers(0, 8)) * 1e-4
            b = a + int(rng.integers(0, 8)) * 1e-4
            shp = ("rect", "disc", "annulus")[int(rng.integers(0, 3))]
            rois.append((dict(shape=shp, xc_m=xc, zc_m=zc, a_m=a, b_m=b),
                         dict(shape="annulus", xc_m=xc, zc_m=zc, a_m=a, b_m=b + 2e-4)))
        img = rng.uniform(0.1, 1.0, (1, nx, nz)).astype(np.float32)
        gpu = _gpu_metrics(img, grid, rois)
        want_in = [int(om.region_mask(grid, t).sum()) for t, _ in rois]
        want_out = [int(om.region_mask(grid, b).sum()) for _, b in rois]
        assert list(gpu["n_in"][0]) == want_in, trial
        assert list(gpu["n_out"][0]) == want_out, trial
        _assert_same(gpu, om.metrics_batch(grid, img, rois), f"boundaries {trial}")
