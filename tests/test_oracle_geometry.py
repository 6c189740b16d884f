"""Pins for the oracle's delay, interpolation, apodisation and beamformer.

* Hand-computed delays on a 3-4-5 triangle geometry (Section 2.1, Eq. 1).
* The DAS image of a delta-pulse RF frame equals the analytic sum of
  triangle functions tri(tau_i(p) - n_i) (linear interpolation of a unit
  impulse), a sum of hyperbolic ridges; with integer delays (Eq. 1 as
  written) it counts the channels whose rounded delay hits the impulse.
* Hand-computed nearest-sample values; nearest and linear sampling agree
  wherever every delay is an exact number of samples.
* A single on-axis point absorber images to its true pixel, and higher
  orders lower the lateral sidelobes (Section 3's qualitative claim).
* The full-image beamformer equals the k-subset definition on tiny arrays.
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold():
    return json.load(open(os.path.join(GOLD, "geometry_worked.json")))


def test_worked_delays():
    g = _gold()
    wl = dict(g["geometry"])
    for c in g["delays"]:
        assert oracle.delay(wl, c["i"], c["j"], c["l"]) == pytest.approx(c["tau"], abs=1e-9)
    s = g["t0_shift"]
    wl2 = dict(wl, t0_s=s["t0_s"])
    assert oracle.delay(wl2, s["i"], s["j"], s["l"]) == pytest.approx(s["tau"], abs=1e-9)


def test_worked_lerp():
    g = _gold()["lerp"]
    for c in g["cases"]:
        assert oracle.lerp(g["row"], c["tau"]) == pytest.approx(c["expected"], abs=1e-12)


def test_worked_nearest():
    g = _gold()["nearest"]
    for c in g["cases"]:
        assert oracle.nearest(g["row"], c["tau"]) == c["expected"], c


def test_nearest_is_linear_at_the_rounded_index():
    """Away from the record's last sample, the nearest sample equals linear
    interpolation evaluated at round(tau) (fraction 0)."""
    rng = np.random.default_rng(3)
    row = rng.standard_normal(50)
    for tau in rng.uniform(-3.0, 52.0, 400):
        n = np.floor(tau + 0.5)
        want = oracle.lerp(row, n) if 0 <= n < 49 else (row[49] if n == 49 else 0.0)
        assert oracle.nearest(row, tau) == want


def test_delta_pulse_nearest_counts_hits():
    """Integer delays (Eq. 1): the DAS image of a delta-pulse frame counts, at
    each pixel, the channels whose rounded delay lands on the impulse."""
    wl = synth.workload("cfg1", nx=64, nz=48, interp="nearest")
    rf, ni = _delta_frame(wl, -0.9e-3, 9.5e-3)
    das = oracle.beamform(wl, rf)["das"]
    n = wl["n_elem"]
    xe = (np.arange(n) - (n - 1) / 2.0) * wl["pitch_m"]
    xp = wl["x0_m"] + (np.arange(wl["nx"]) + 0.5) * (wl["x1_m"] - wl["x0_m"]) / wl["nx"]
    zp = wl["z0_m"] + (np.arange(wl["nz"]) + 0.5) * (wl["z1_m"] - wl["z0_m"]) / wl["nz"]
    tau = wl["fs_hz"] / wl["c_m_s"] * np.sqrt(
        (xp[:, None, None] - xe[None, None, :]) ** 2 + zp[None, :, None] ** 2
    )
    frac = tau - np.floor(tau)
    assert np.min(np.abs(frac - 0.5)) > 1e-9  # no rounding ties on this grid
    want = (np.floor(tau + 0.5) == ni[None, None, :]).sum(axis=2)
    assert np.array_equal(das, want.astype(float))
    assert want.max() >= 8


def test_worked_apodisation():
    g = _gold()
    wl = dict(g["geometry"])
    wl.update(g["apod"]["geometry_change"])
    for c in g["apod"]["cases"]:
        assert oracle.apod(wl, c["i"], c["j"], c["l"]) == pytest.approx(c["expected"], abs=1e-12)
    # outside the active aperture the weight is zero
    wl_far = dict(wl, f_number=4.0)  # half-aperture 0.25 mm
    assert oracle.apod(wl_far, 3, 0, 0) == 0.0


def _delta_frame(wl, xs, zs):
    """Unit impulse per channel at round(fs r_i / c)."""
    n, ns = wl["n_elem"], wl["n_samples"]
    xe = (np.arange(n) - (n - 1) / 2.0) * wl["pitch_m"]
    r = np.sqrt((xs - xe) ** 2 + zs ** 2)
    ni = np.rint(wl["fs_hz"] * r / wl["c_m_s"]).astype(int)
    rf = np.zeros((n, ns))
    rf[np.arange(n), ni] = 1.0
    return rf, ni


def test_delta_pulse_hyperbola():
    """DAS of a delta-pulse frame = sum_i tri(tau_i(p) - n_i), closed form."""
    wl = synth.workload("cfg1", nx=64, nz=48)
    rf, ni = _delta_frame(wl, 1.2e-3, 11.0e-3)
    das = oracle.beamform(wl, rf)["das"]
    n = wl["n_elem"]
    xe = (np.arange(n) - (n - 1) / 2.0) * wl["pitch_m"]
    xp = wl["x0_m"] + (np.arange(wl["nx"]) + 0.5) * (wl["x1_m"] - wl["x0_m"]) / wl["nx"]
    zp = wl["z0_m"] + (np.arange(wl["nz"]) + 0.5) * (wl["z1_m"] - wl["z0_m"]) / wl["nz"]
    tau = wl["fs_hz"] / wl["c_m_s"] * np.sqrt(
        (xp[:, None, None] - xe[None, None, :]) ** 2 + zp[None, :, None] ** 2
    )
    tri = np.maximum(0.0, 1.0 - np.abs(tau - ni[None, None, :]))
    want = tri.sum(axis=2)
    assert np.max(np.abs(das - want)) < 1e-12
    assert want.max() > 10  # the ridge is actually hit


def test_point_absorber_peak_and_sidelobes():
    """Single on-axis absorber: envelope peaks at its true pixel (exact in x,
    +-1 in z), the image is mirror-symmetric about x = 0, and the lateral
    sidelobe level away from the main lobe falls as the order grows
    (Section 3: higher orders suppress sidelobes)."""
    wl = synth.workload("cfg1", nx=129, nz=256, noise_frac=0.0, x0_m=-6.45e-3, x1_m=6.45e-3)
    l0 = 160
    zs = wl["z0_m"] + (l0 + 0.5) * (wl["z1_m"] - wl["z0_m"]) / wl["nz"]
    rf = synth.render_rf(wl, synth.point_scene([0.0], [zs]))
    xp = wl["x0_m"] + (np.arange(wl["nx"]) + 0.5) * (wl["x1_m"] - wl["x0_m"]) / wl["nx"]
    assert abs(xp[64]) < 1e-15
    side_db = {}
    for k in (1, 2, 3, 4, 5):
        img = oracle.frame(wl, rf, order_k=k, stages=("raw", "env"))
        env = img["env"]["das" if k == 1 else ("dmas" if k == 2 else "ho")]
        j, l = np.unravel_index(np.argmax(env), env.shape)
        assert j == 64
        assert abs(l - l0) <= 1
        assert np.allclose(env, env[::-1, :], rtol=1e-9, atol=1e-12 * env.max())
        prof = env.max(axis=1) / env.max()
        side_db[k] = 20 * np.log10(prof[np.abs(xp) > 1.0e-3].max())
    for k in (2, 3, 4, 5):
        assert side_db[k] < side_db[k - 1] - 5.0


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_beamformer_equals_definition_tiny(k):
    wl = synth.workload("cfg1", n_elem=7, nx=7, nz=6, n_samples=512, noise_frac=0.05)
    wl["x0_m"], wl["x1_m"] = -1.05e-3, 1.05e-3
    rf = synth.make_frame(wl, 3)
    fast = oracle.beamform(wl, rf, order_k=k)["ho"]
    brute = oracle.beamform_bruteforce(wl, rf, order_k=k)
    scale = np.abs(brute).max()
    assert scale > 0
    assert np.max(np.abs(fast - brute)) <= 1e-11 * scale


def test_beamform_pixels_matches_full():
    wl = synth.workload("cfg1", nx=32, nz=32)
    rf = synth.make_frame(wl, 1)
    full = oracle.beamform(wl, rf)
    rng = np.random.default_rng(0)
    j = rng.integers(0, 32, 50)
    l = rng.integers(0, 32, 50)
    some = oracle.beamform_pixels(wl, rf, j, l)
    for o in ("das", "dmas", "ho"):
        assert np.array_equal(some[o], full[o][j, l])


def test_apodised_pixel_without_active_elements_is_zero():
    wl = synth.workload("cfg1", nx=16, nz=16, f_number=50.0)
    rf = synth.make_frame(wl, 1)
    out = oracle.beamform(wl, rf, order_k=4)
    # first depth row: half-aperture = z/(2F) is far below the pitch
    assert np.all(out["ho"][:, 0] == 0.0) and np.all(out["das"][:, 0] == 0.0)
