"""Parity in the launch configurations bench.py times.

* The FP32 step: cfg2 geometry, 32 frames (seed 11, frames 0..31) in one
  launch, log images only (raw and envelope computed in place), k = 3 - every
  frame against the FP64 oracle's full log image.
* The throughput batch: cfg5, 64 BF16 frames in one launch, k = 4, F# 1.5
  apodisation, Kahan sums - sampled raw pixels of every frame against the
  oracle evaluated pixel by pixel on the same (dequantised) RF, normalised
  by the oracle's largest sampled value, and the log images' properties
  (peak at 0 dB, values in [-60, 0]).
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import run_gpu

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


def test_fp32_step_32_frames_log_only():
    wl = synth.workload("cfg2")
    rf = synth.make_frames(wl, 11, 32)
    out, info, deq = run_gpu(wl, rf, 3, stages=4, max_batch=32)  # [32][1][3][512][512]
    assert info["device_error_flags"] == 0
    worst = 0.0
    for f in range(32):
        ref = oracle.frame(wl, deq[f], order_k=3, stages=("raw", "env", "log"))["log"]
        for oi, o in enumerate(oracle.OUTPUT_ORDER):
            g, r = out[f, 0, oi], ref[o]
            sel = r >= -6.0
            worst = max(worst, float(np.max(np.abs(g[sel] - r[sel]))))
            assert -1e-4 <= g.max() <= 0.0 and g.min() >= -60.0
    assert worst <= 0.05, worst


def test_throughput_batch_64_frames_sampled():
    wl = synth.workload("cfg5")
    rf = synth.make_frames(wl, 41, 64)
    out, info, deq = run_gpu(wl, rf, 4, rf_dtype="bf16", compensated=1, stages=5, max_batch=64)
    assert info["device_error_flags"] == 0
    rng = np.random.default_rng(7)
    for f in range(64):
        raw = out[f, 0]  # [3][1024][1024]: DAS, DMAS, DMAS-4
        # uniform samples, plus each output's maximum and pixels around it
        j = [rng.integers(0, wl["nx"], 192)]
        l = [rng.integers(0, wl["nz"], 192)]
        for oi in range(3):
            pk = np.unravel_index(np.argmax(np.abs(raw[oi])), raw[oi].shape)
            j.append(np.r_[pk[0], np.clip(pk[0] + rng.integers(-8, 9, 32), 0, wl["nx"] - 1)])
            l.append(np.r_[pk[1], np.clip(pk[1] + rng.integers(-8, 9, 32), 0, wl["nz"] - 1)])
        j, l = np.concatenate(j), np.concatenate(l)
        ref = oracle.beamform_pixels(wl, deq[f], j, l, order_k=4)
        for oi, o in enumerate(oracle.OUTPUT_ORDER):
            # the oracle's largest value over the samples (which hold the
            # pixel where each output peaks): at most the oracle image's
            # peak, so this normalisation is the stricter one
            peak = float(np.max(np.abs(ref[o])))
            err = np.max(np.abs(raw[oi][j, l] - ref[o]))
            assert err <= TOL32 * peak, (f, o, err / peak)
        lg = out[f, 1]
        mx = lg.max(axis=(1, 2))
        assert np.all((mx <= 0.0) & (mx >= -1e-4)) and lg.min() >= -60.0
