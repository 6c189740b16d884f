"""The five synthetic workloads (shapes of the paper's studies, seeded).

Each entry is a plain dictionary with the array geometry, acquisition
parameters, image grid and scene recipe.  Keys that name beamformer
parameters (``order_k``, ``f_number``, ``rf_dtype``...) are *requests*: the
generator itself only reads the geometry and scene keys.

cfg1  plain method, FP32/FP64: 64 elements, 0.3 mm pitch, c = 1540 m/s,
      fs = 40 MHz, 1024 samples, 128x128 grid over 19.2 x 20 mm, 5 point
      absorbers, Gaussian noise 5 % of peak; DAS, DMAS, DMAS-3.
cfg2  single frame FP32: 128 elements, 2048 samples at 40 MHz, 512x512 grid
      over 38.4 x 40 mm, 20 points + 4 vessel-like lines, noise 3 %;
      DAS and k = 2..5.
cfg3  precision: 256 elements, 4096 samples at 50 MHz, 1024x1024 grid over
      76.8 x 60 mm, 20 points with log-uniform amplitudes over 40 dB, RF
      scaled to unit RMS, stored BF16/FP16; k = 3, 5, compensated sums.
cfg4  serving mix: N in {64,128,256}, Ns in {1024,2048,4096} at 40 MHz,
      grid side in {256,512,1024}, k in {2..5}, Poisson arrivals 2000/s.
cfg5  throughput batch: 64 frames of 128 el x 2048 samples BF16, 1024x1024
      grid over 38.4 x 40 mm, k = 4, F-number 1.5 with Hann apodisation.

Pulse centre frequency is 5 MHz throughout (unstated for cfg3..5).
The lateral span equals the aperture, ``x in [-N p/2, +N p/2]``.
"""

from __future__ import annotations

import copy

import numpy as np

_BASE = dict(
    pitch_m=0.3e-3,
    c_m_s=1540.0,
    t0_s=0.0,
    f0_hz=5e6,
    band_lo_hz=0.0,
    band_hi_hz=0.0,
    dyn_range_db=60.0,
    f_number=0.0,
    rf_dtype="f32",
    compensated=0,
    n_lines=0,
    noise_frac=0.0,
)


def _mk(**kw):
    d = dict(_BASE)
    d.update(kw)
    half = d["n_elem"] * d["pitch_m"] / 2.0
    d.setdefault("x0_m", -half)
    d.setdefault("x1_m", +half)
    return d


CONFIGS = {
    "cfg1": _mk(
        name="cfg1",
        n_elem=64,
        fs_hz=40e6,
        n_samples=1024,
        nx=128,
        nz=128,
        z0_m=0.0,
        z1_m=20e-3,
        n_points=5,
        noise_frac=0.05,
        order_k=3,
        seeds=[1, 2, 3, 4, 5],
    ),
    "cfg2": _mk(
        name="cfg2",
        n_elem=128,
        fs_hz=40e6,
        n_samples=2048,
        nx=512,
        nz=512,
        z0_m=0.0,
        z1_m=40e-3,
        n_points=20,
        n_lines=4,
        noise_frac=0.03,
        order_k=3,
        orders=[2, 3, 4, 5],
        seeds=[11],
    ),
    "cfg3": _mk(
        name="cfg3",
        n_elem=256,
        fs_hz=50e6,
        n_samples=4096,
        nx=1024,
        nz=1024,
        z0_m=0.0,
        z1_m=60e-3,
        n_points=20,
        log_amp_db=40.0,
        unit_rms=True,
        order_k=3,
        orders=[3, 5],
        rf_dtype="bf16",
        compensated=1,
        seeds=[21],
    ),
    "cfg5": _mk(
        name="cfg5",
        n_elem=128,
        fs_hz=40e6,
        n_samples=2048,
        nx=1024,
        nz=1024,
        z0_m=0.0,
        z1_m=40e-3,
        n_points=20,
        n_lines=4,
        noise_frac=0.03,
        order_k=4,
        f_number=1.5,
        rf_dtype="bf16",
        compensated=1,
        n_frames=64,
        seeds=[41],
    ),
}


def workload(name: str, **overrides) -> dict:
    """A copy of workload ``name`` with keys overridden."""
    wl = copy.deepcopy(CONFIGS[name])
    wl.update(overrides)
    return wl


def serving_mix(n_requests: int, seed: int = 31, rate_hz: float = 2000.0):
    """cfg4: seeded request stream with Poisson arrivals.

    Returns a list of ``(arrival_s, workload_dict)``.  Channel count, sample
    count, grid side and order are uniform over their discrete sets; depth
    is ``min(40 mm, 0.5 Ns c / fs)`` and the lateral span is the aperture.
    """
    rng = np.random.default_rng([seed, 0])
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    out = []
    for i in range(n_requests):
        n = int(rng.choice([64, 128, 256]))
        ns = int(rng.choice([1024, 2048, 4096]))
        side = int(rng.choice([256, 512, 1024]))
        k = int(rng.integers(2, 6))
        depth = min(40e-3, 0.5 * ns * 1540.0 / 40e6)
        wl = _mk(
            name="cfg4",
            n_elem=n,
            fs_hz=40e6,
            n_samples=ns,
            nx=side,
            nz=side,
            z0_m=0.0,
            z1_m=depth,
            n_points=10,
            noise_frac=0.03,
            order_k=k,
            rf_dtype="bf16",
            compensated=1,
        )
        out.append((float(t[i]), wl))
    return out
