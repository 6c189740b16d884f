"""Pins for the oracle's post-processing (Section 3): FFT, Hilbert envelope,
band-pass mask and log compression.

The band-pass *parameters* are parity unpinned (the paper names no band);
what is pinned is the FFT (against its O(M^2) DFT and numpy.fft), the
analytic-signal mask, the envelope of an in-band cosine (constant, equal
to its amplitude), removal of DC, the closed form of the log stage, and the
mapping of depth bins to temporal frequency under one-way propagation
(hand-worked bins and Nyquist clip; an RF tone of known frequency carried
through the beamformer keeps or loses its envelope as its frequency says).
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("m", [1, 2, 8, 64, 512])
def test_fft_matches_dft_and_numpy(m):
    rng = np.random.default_rng(m)
    x = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    f = oracle.fft(x)
    assert np.allclose(f, oracle.dft(x), rtol=0, atol=1e-10 * max(1, m))
    assert np.allclose(f, np.fft.fft(x), rtol=0, atol=1e-11 * max(1, m))
    assert np.allclose(oracle.fft(f, inverse=True), x, atol=1e-12 * max(1, m))
    assert np.allclose(oracle.dft(f, inverse=True), x, atol=1e-10 * max(1, m))


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12))


def _wl(nz=512, depth=20e-3):
    return synth.workload("cfg2", nx=4, nz=nz, z0_m=0.0, z1_m=depth)


def test_mask_structure_and_band_edges():
    wl = _wl()
    m = oracle.fft_size(wl["nz"])
    h_odd, dc_odd = oracle.post_mask(wl, False)
    h_even, dc_even = oracle.post_mask(wl, True)
    assert not dc_odd and not dc_even
    assert np.all(h_odd[m // 2 + 1:] == 0) and np.all(h_even[m // 2 + 1:] == 0)
    f = np.array([oracle.bin_hz(wl, m, b) for b in range(m // 2 + 1)])
    f0 = wl["f0_hz"]
    # pass band gets the analytic weight 2, outside band + roll-off gets 0
    inside = (f >= 0.5 * f0) & (f <= 1.5 * f0)
    assert np.all(h_odd[: m // 2 + 1][inside] == 2.0)
    far = (f < 0.25 * f0 - 1) | (f > 1.75 * f0 + 1)
    assert np.all(h_odd[: m // 2 + 1][far] == 0.0)
    inside_e = (f >= 1.5 * f0) & (f <= 2.5 * f0)
    assert np.all(h_even[: m // 2 + 1][inside_e] == 2.0)
    assert h_odd[0] == 0.0 and h_even[0] == 0.0  # DC removed
    # roll-off is monotone between 0 and 2
    roll = (f > 0.25 * f0) & (f < 0.5 * f0)
    vals = h_odd[: m // 2 + 1][roll]
    assert np.all(np.diff(vals) >= 0) and np.all((vals > 0) & (vals < 2))


def test_mask_nyquist_clip_and_filter_off():
    # cfg1: 128 pixels over 20 mm -> axial Nyquist 4.93 MHz < 7.5 MHz
    wl = synth.workload("cfg1")
    h, dc_only = oracle.post_mask(wl, True)
    m = h.size
    assert dc_only
    assert h[0] == 0.0 and np.all(h[1 : m // 2] == 2.0) and h[m // 2] == 1.0
    h_off, _ = oracle.post_mask(dict(wl, band_hi_hz=-1.0), False)
    want = np.zeros(m)
    want[0] = want[m // 2] = 1.0
    want[1 : m // 2] = 2.0
    assert np.array_equal(h_off, want)


@pytest.mark.parametrize("even", [False, True])
def test_envelope_of_inband_cosine_is_its_amplitude(even):
    wl = _wl()
    nz = wl["nz"]
    m = oracle.fft_size(nz)
    h, _ = oracle.post_mask(wl, even)
    f = np.array([oracle.bin_hz(wl, m, b) for b in range(m // 2)])
    target = (2.0 if even else 1.0) * wl["f0_hz"]
    b0 = int(np.argmin(np.abs(f - target)))
    assert h[b0] == 2.0
    amp = 3.25
    col = amp * np.cos(2 * np.pi * b0 * np.arange(nz) / m + 0.3)
    env = oracle.envelope(col, h)
    assert np.allclose(env, amp, rtol=0, atol=1e-10)


def test_dc_is_removed():
    wl = _wl()  # nz = M = 512, no padding
    h, _ = oracle.post_mask(wl, False)
    assert np.max(oracle.envelope(np.full(512, 7.0), h)) < 1e-9
    assert oracle.envelope(np.zeros(512), h).max() == 0.0


def test_zero_padded_envelope_matches_numpy():
    """Envelope assembly (pad to M, mask, inverse, first nz, modulus)
    against numpy.fft with an explicit length-M transform."""
    wl = _wl(nz=200, depth=8e-3)
    m = oracle.fft_size(200)
    assert m == 256
    h, _ = oracle.post_mask(wl, False)
    col = np.random.default_rng(3).standard_normal(200)
    want = np.abs(np.fft.ifft(h * np.fft.fft(col, m)))[:200]
    assert np.allclose(oracle.envelope(col, h), want, rtol=0, atol=1e-12)


def test_log_closed_form():
    g = json.load(open(os.path.join(GOLD, "geometry_worked.json")))["log"]
    out = oracle.log_image(np.array(g["env"]), g["dyn_range_db"])
    assert np.allclose(out, g["expected"], atol=1e-12)
    assert np.all(oracle.log_image(np.zeros(5), 60.0) == -60.0)


# ---- depth-to-frequency mapping (reading of the Section 3 band-pass) ------
# Pinned from outside the oracle: hand-worked bin frequencies and masks, and
# an RF tone of known temporal frequency carried through the beamformer to
# its depth bin.  A mapping off by a factor of two (two-way c / 2, or 2 c)
# fails both the literal values and the tone outcomes.

def _post_gold():
    return json.load(open(os.path.join(GOLD, "post_worked.json")))


def test_bin_hz_hand_worked():
    for case in _post_gold()["bin_hz"]:
        wl = synth.workload("cfg1", nz=case["nz"], z0_m=case["z0_m"], z1_m=case["z1_m"],
                            c_m_s=case["c_m_s"])
        got = oracle.bin_hz(wl, case["m"], case["b"])
        assert got == pytest.approx(case["hz"], rel=1e-12), case["workload"]


def test_nyquist_clip_odd_order_cfg1():
    """cfg1's axial Nyquist rate (4.93 MHz) lies inside the odd band
    [2.5, 7.5] MHz: the band is clipped, not reduced to DC removal."""
    g = _post_gold()["cfg1_odd_mask"]
    wl = synth.workload("cfg1")
    h, dc_only = oracle.post_mask(wl, False)
    assert h.size == 128
    assert dc_only == g["dc_only"]
    assert np.all(h[: g["zero_bins_upto"] + 1] == 0.0)
    r0, r1 = g["rolloff_bins"]
    assert np.all((h[r0 : r1 + 1] > 0.0) & (h[r0 : r1 + 1] < 2.0))
    b0, b1 = g["band_bins"]
    assert np.all(h[b0 : b1 + 1] == 2.0)
    assert h[64] == g["nyquist_bin_weight"]
    assert np.all(h[65:] == 0.0)
    assert h[g["b20"]["b"]] == pytest.approx(g["b20"]["h"], abs=1e-12)


def tone_case(b):
    """(workload, RF frame) of the one-element tone pin at depth bin b."""
    g = _post_gold()["tone"]
    wl = dict(g["geometry"], name="tone", interp="linear")
    n = np.arange(wl["n_samples"])
    f = b * wl["fs_hz"] / wl["nz"]
    rf = np.cos(2 * np.pi * f * n / wl["fs_hz"] + g["phase"])[None, :]
    return wl, rf


@pytest.mark.parametrize("case", _post_gold()["tone"]["cases"], ids=lambda c: f"bin{c['b']}")
def test_tone_passes_or_is_blocked_by_its_temporal_frequency(case):
    wl, rf = tone_case(case["b"])
    out = oracle.frame(wl, rf, order_k=1)
    raw = out["raw"]["das"][0]
    # the DAS column is the tone sampled at tau = l + 1 (exact delays)
    want_raw = rf[0, 1 : wl["nz"] + 1]
    assert np.allclose(raw, want_raw, rtol=0, atol=1e-9)
    env = out["env"]["das"][0]
    assert np.allclose(env, case["odd_env"], rtol=0, atol=1e-9)
    h_even, _ = oracle.post_mask(wl, True)
    assert np.allclose(oracle.envelope(raw, h_even), case["even_env"], rtol=0, atol=1e-9)
