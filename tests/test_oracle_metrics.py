"""Pins for the oracle's image-quality metrics (Section 3, Eqs. 10-12).

* SNR and CR closed forms on a constructed image: a constant target and a
  background of two interleaved levels (mean 2, population deviation 1).
* Region pixel counts equal the number of lattice points in a disc of
  radius^2 10 (Gauss's circle count, 37) and in the annulus around it.
* gCNR: identical samples give 0, separated ones 1, hand-counted partial
  overlaps, and two Gaussian samples reach 1 - OVL of the normal densities.
* FWHM: a triangular lobe (linear between pixels, so the interpolated
  crossing is exact), a Gaussian lobe (2 sqrt(2 ln 2) sigma), NaN at the edge.
* Section 3's qualitative claim on a point absorber: the lateral FWHM falls
  as the order grows (DAS > DMAS-3 > DMAS-5 and DMAS > DMAS-4).
"""

import math

import numpy as np
import pytest

import oracle
import synth
from oracle import metrics as om

GRID = dict(nx=32, nz=32, x0_m=0.0, x1_m=3.2e-3, z0_m=0.0, z1_m=3.2e-3)
DX = 1e-4


def _rect(j0, j1, l0, l1):
    """Rectangle whose pixel centres are exactly columns j0..j1-1, rows l0..l1-1."""
    return dict(shape="rect", xc_m=(j0 + j1) / 2 * DX, zc_m=(l0 + l1) / 2 * DX,
                a_m=(j1 - j0) / 2 * DX, b_m=(l1 - l0) / 2 * DX)


def test_snr_cr_closed_form():
    img = np.zeros((32, 32), dtype=np.float32)
    img[2:6, 2:6] = 4.0
    cols = np.arange(10, 20)
    img[10:20, 5:15] = np.where(cols % 2 == 0, 1.0, 3.0)[:, None]
    r = om.metrics(GRID, img, _rect(2, 6, 2, 6), _rect(10, 20, 5, 15))
    assert r["n_in"] == 16 and r["n_out"] == 100
    assert r["mu_in"] == 4.0 and r["mu_out"] == 2.0 and r["sigma_out"] == 1.0
    assert r["snr_db"] == pytest.approx(40 * math.log10(2.0), abs=1e-12)
    assert r["cr_db"] == pytest.approx(20 * math.log10(2.0), abs=1e-12)
    assert r["peak"] == 4.0 and (r["peak_j"], r["peak_l"]) == (2, 2)  # first in x-major order


def test_region_counts_gauss_circle():
    xc, zc = (16 + 0.5) * DX, (12 + 0.5) * DX  # a pixel centre
    disc = dict(shape="disc", xc_m=xc, zc_m=zc, a_m=math.sqrt(10.24) * DX)
    inner = dict(shape="disc", xc_m=xc, zc_m=zc, a_m=1.5 * DX)
    ring = dict(shape="annulus", xc_m=xc, zc_m=zc, a_m=1.5 * DX, b_m=math.sqrt(10.24) * DX)
    n = lambda r: int(om.region_mask(GRID, r).sum())  # noqa: E731
    assert n(disc) == 37  # lattice points with i^2 + j^2 <= 10
    assert n(inner) == 9  # i^2 + j^2 <= 2
    assert n(ring) == 28
    assert not np.any(om.region_mask(GRID, inner) & om.region_mask(GRID, ring))


def test_gcnr_exact_cases():
    a = np.array([0.2, 0.4, 0.6, 0.8], dtype=np.float32)
    assert om.gcnr(a, a) == 0.0
    assert om.gcnr(np.full(10, 1.0), np.full(30, 0.3)) == 1.0
    # target all at the maximum (bin 255); background half there, half at 0.1
    assert om.gcnr(np.ones(8), np.r_[np.ones(5), np.full(5, 0.1)]) == pytest.approx(0.5, abs=1e-15)
    # hand count: vmax = 1; bins of 0.25, 0.5, 0.75, 1.0 are 64, 128, 192, 255.
    # h_in = (1/4 each of 64, 128, 192, 255); h_out = (1/2 at 64, 1/2 at 0)
    # overlap = min(1/4, 1/2) = 1/4
    assert om.gcnr([0.25, 0.5, 0.75, 1.0], [0.25, 0.0]) == pytest.approx(0.75, abs=1e-15)
    assert list(om.amplitude_bins([0.0, -1.0, 0.25, 0.999, 1.0], 1.0)) == [0, 0, 64, 255, 255]


def test_gcnr_of_two_gaussians_is_one_minus_overlap():
    """Large samples of N(5, 1) and N(7, 1): gCNR -> 1 - OVL, OVL = 2 Phi(-1)."""
    rng = np.random.default_rng(0)
    a = rng.normal(7.0, 1.0, 400_000)
    b = rng.normal(5.0, 1.0, 400_000)
    ovl = 2 * 0.5 * math.erfc(1.0 / math.sqrt(2.0))
    assert om.gcnr(a, b) == pytest.approx(1.0 - ovl, abs=0.01)


def test_fwhm_triangle_exact():
    img = np.zeros((32, 32), dtype=np.float32)
    j = np.arange(32)
    img[:, 7] = np.maximum(0.0, 1.0 - np.abs(j - 15) / 8.0)
    r = om.metrics(GRID, img, _rect(12, 18, 5, 10), _rect(0, 4, 20, 30))
    assert (r["peak_j"], r["peak_l"]) == (15, 7)
    assert r["fwhm_m"] == pytest.approx(8 * DX, rel=1e-12)


def test_fwhm_gaussian_and_edge():
    img = np.zeros((128, 8), dtype=np.float32)
    j = np.arange(128)
    s = 6.0
    img[:, 3] = np.exp(-((j - 60.3) ** 2) / (2 * s * s))
    g = dict(nx=128, nz=8, x0_m=0.0, x1_m=128 * DX, z0_m=0.0, z1_m=8 * DX)
    want = 2 * math.sqrt(2 * math.log(2)) * s * DX
    assert om.fwhm(g, img, 60, 3) == pytest.approx(want, rel=0.01)
    img[:, 3] = np.exp(-((j - 2.0) ** 2) / (2 * s * s))  # left half cut by the edge
    assert math.isnan(om.fwhm(g, img, 2, 3))


def test_fwhm_falls_with_order_on_a_point_absorber():
    """Section 3: more correlated terms give a narrower main lobe.  Odd orders
    keep the fundamental band and even orders the second-harmonic band after
    the post filter, so widths are compared within each family (and every
    higher order against DAS)."""
    wl = synth.workload("cfg1", nx=257, nz=256, noise_frac=0.0, x0_m=-6.425e-3, x1_m=6.425e-3)
    l0 = 160
    zs = wl["z0_m"] + (l0 + 0.5) * (wl["z1_m"] - wl["z0_m"]) / wl["nz"]
    rf = synth.render_rf(wl, synth.point_scene([0.0], [zs]))
    tgt = dict(shape="disc", xc_m=0.0, zc_m=zs, a_m=1.0e-3)
    bg = dict(shape="annulus", xc_m=0.0, zc_m=zs, a_m=2.5e-3, b_m=4.0e-3)
    w = {}
    for k in (1, 2, 3, 4, 5):
        env = oracle.frame(wl, rf, order_k=k, stages=("raw", "env"))["env"]
        img = env["das" if k == 1 else ("dmas" if k == 2 else "ho")].astype(np.float32)
        m = om.metrics(wl, img, tgt, bg)
        assert (m["peak_j"], m["peak_l"]) == (128, l0)
        w[k] = m["fwhm_m"]
    assert w[1] > w[3] > w[5] > 0
    assert w[2] > w[4] > 0
    assert max(w[2], w[3], w[4], w[5]) < w[1]
