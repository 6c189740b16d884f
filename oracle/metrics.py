"""Image-quality metrics of Section 3, written out plainly in numpy FP64.

TEST INFRASTRUCTURE ONLY (the same rule as the rest of ``oracle/``): only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the CUDA library never does.

* SNR (Eq. 10) = 20 log10(mu_in / sigma_out), CR (Eq. 11) =
  20 log10(mu_in / mu_out): means over the target ("in") and background
  ("out") pixels; sigma_out is the background's population standard
  deviation (the paper does not say which; dividing by the pixel count is the
  reading taken).
* gCNR (Eq. 12) = 1 - sum_x min(h_in(x), h_out(x)) with h the probability
  mass of the normalised amplitude x in [0, 1] over 256 equal bins (the paper
  gives no bin count).  Normalisation by the largest value of the two regions
  (reading).  The bin of a value is an integer decided in floating point, so
  it is taken in FP32 exactly as the GPU takes it: floor((v * 256) / vmax),
  clamped to [0, 255], values <= 0 in bin 0.
* FWHM (lateral, the main-lobe width of Section 3): on the image row of the
  target maximum, walk out from the maximum while values stay >= half of it;
  each crossing is linearly interpolated between the last pixel >= half and
  the first pixel below; NaN if a side reaches the image edge.
* Regions hold the pixels whose centres lie inside a rectangle (|dx| <= a,
  |dz| <= b), a disc (d^2 <= a^2) or an annulus (a^2 < d^2 <= b^2).

Parity status: pinned by tests/test_oracle_metrics.py (closed forms on
constructed images, exact histogram cases, a triangular lobe whose FWHM the
linear crossing reproduces exactly, Gaussian lobes, region pixel counts).
"""

from __future__ import annotations

import numpy as np

BINS = 256
FIELDS = ("mu_in", "mu_out", "sigma_out", "snr_db", "cr_db", "gcnr", "fwhm_m", "peak",
          "n_in", "n_out", "peak_j", "peak_l")


def pixel_centres(grid):
    """x (length nx) and z (length nz) pixel-centre coordinates."""
    nx, nz = int(grid["nx"]), int(grid["nz"])
    dx = (grid["x1_m"] - grid["x0_m"]) / nx
    dz = (grid["z1_m"] - grid["z0_m"]) / nz
    x = grid["x0_m"] + (np.arange(nx, dtype=np.float64) + 0.5) * dx
    z = grid["z0_m"] + (np.arange(nz, dtype=np.float64) + 0.5) * dz
    return x, z, dx


def region_mask(grid, region):
    """Boolean [nx][nz] mask of the pixels inside ``region``."""
    x, z, _ = pixel_centres(grid)
    ex = x[:, None] - region["xc_m"]
    ez = z[None, :] - region["zc_m"]
    a = float(region["a_m"])
    b = float(region.get("b_m", 0.0))
    shape = region["shape"]
    if shape == "rect":
        return (np.abs(ex) <= a) & (np.abs(ez) <= b)
    d2 = ex * ex + ez * ez
    if shape == "disc":
        return d2 <= a * a
    if shape == "annulus":
        return (d2 > a * a) & (d2 <= b * b)
    raise ValueError(shape)


def amplitude_bins(v, vmax):
    """Bin index of each value for Eq. 12's histogram (FP32 decision)."""
    v = np.asarray(v, dtype=np.float32)
    vmax = np.float32(vmax)
    out = np.zeros(v.shape, dtype=np.int64)
    if not vmax > 0:
        return out
    pos = v > 0
    x = (v[pos] * np.float32(256.0)) / vmax
    out[pos] = np.minimum(255, np.floor(x).astype(np.int64))
    return out


def gcnr(v_in, v_out):
    """Eq. 12 on two samples of amplitudes."""
    v_in = np.asarray(v_in, dtype=np.float32)
    v_out = np.asarray(v_out, dtype=np.float32)
    vmax = max(v_in.max(), v_out.max())
    h_in = np.bincount(amplitude_bins(v_in, vmax), minlength=BINS) / v_in.size
    h_out = np.bincount(amplitude_bins(v_out, vmax), minlength=BINS) / v_out.size
    return 1.0 - np.minimum(h_in, h_out).sum()


def fwhm(grid, img, j0, l0):
    """Lateral FWHM on row l0 around the maximum at column j0."""
    x, _, dx = pixel_centres(grid)
    row = np.asarray(img, dtype=np.float32)[:, l0].astype(np.float64)
    half = 0.5 * row[j0]
    nx = row.size
    jl = j0
    while jl > 0 and row[jl - 1] >= half:
        jl -= 1
    jr = j0
    while jr < nx - 1 and row[jr + 1] >= half:
        jr += 1
    if jl == 0 or jr == nx - 1:
        return float("nan")
    xl = x[jl - 1] + ((half - row[jl - 1]) / (row[jl] - row[jl - 1])) * dx
    xr = x[jr + 1] - ((half - row[jr + 1]) / (row[jr] - row[jr + 1])) * dx
    return float(xr - xl)


def metrics(grid, img, target, background):
    """All fields of one (target, background) pair on one [nx][nz] image."""
    img = np.asarray(img, dtype=np.float32)
    mi = region_mask(grid, target)
    mo = region_mask(grid, background)
    vi = img[mi].astype(np.float64)
    vo = img[mo].astype(np.float64)
    nan = float("nan")
    r = dict(n_in=int(vi.size), n_out=int(vo.size))
    r["mu_in"] = float(vi.mean()) if vi.size else nan
    r["mu_out"] = float(vo.mean()) if vo.size else nan
    r["sigma_out"] = float(np.sqrt(np.mean((vo - vo.mean()) ** 2))) if vo.size else nan
    with np.errstate(divide="ignore", invalid="ignore"):
        r["snr_db"] = float(20.0 * np.log10(np.float64(r["mu_in"]) / np.float64(r["sigma_out"])))
        r["cr_db"] = float(20.0 * np.log10(np.float64(r["mu_in"]) / np.float64(r["mu_out"])))
    r["gcnr"] = float(gcnr(img[mi], img[mo])) if vi.size and vo.size else nan
    if vi.size:
        # first maximum in x-major order
        masked = np.where(mi, img, -np.inf)
        q = int(np.argmax(masked))
        j0, l0 = divmod(q, img.shape[1])
        r["peak"] = float(img[j0, l0])
        r["peak_j"], r["peak_l"] = j0, l0
        r["fwhm_m"] = fwhm(grid, img, j0, l0)
    else:
        r["peak"] = nan
        r["peak_j"] = r["peak_l"] = -1
        r["fwhm_m"] = nan
    return r


def metrics_batch(grid, images, rois):
    """images [n][nx][nz]; rois list of (target, background) -> dict of [n][n_roi]."""
    images = np.asarray(images)
    images = images.reshape(-1, images.shape[-2], images.shape[-1])
    out = {f: np.empty((images.shape[0], len(rois)),
                       dtype=np.int64 if f in ("n_in", "n_out", "peak_j", "peak_l") else np.float64)
           for f in FIELDS}
    for i, img in enumerate(images):
        for k, (t, b) in enumerate(rois):
            r = metrics(grid, img, t, b)
            for f in FIELDS:
                out[f][i, k] = r[f]
    return out
