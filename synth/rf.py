"""Forward model for synthetic linear-array PA RF data (input generator only).

Geometry convention (shared with the beamformer only through the numbers in
the workload dictionaries): element ``i`` of an ``N``-element array with
pitch ``p`` sits at ``x_i = (i - (N-1)/2) * p``, ``z = 0``.  Light fires at
``t = 0`` and a source at ``(xs, zs)`` is heard by element ``i`` after the
one-way time of flight ``r_i / c`` (Section 2.1 writes only "the time delay
of that element"; photoacoustic reception is one-way).

Pulse: the first derivative of a Gaussian, ``g(t) = -(t/sigma) e^{1/2}
exp(-t^2 / 2 sigma^2)``, normalised to unit peak, with ``sigma = 1/(2 pi f0)``
so that its spectrum peaks at ``f0``.  Amplitude falls as ``1/r`` (r in mm).
No element directivity and no transducer band limit are modelled.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Scene:
    """Absorber positions (metres) and amplitudes for one frame."""

    xs: np.ndarray
    zs: np.ndarray
    amp: np.ndarray


def point_scene(xs, zs, amp=None) -> Scene:
    xs = np.atleast_1d(np.asarray(xs, dtype=np.float64))
    zs = np.atleast_1d(np.asarray(zs, dtype=np.float64))
    if amp is None:
        amp = np.ones_like(xs)
    return Scene(xs, zs, np.atleast_1d(np.asarray(amp, dtype=np.float64)))


def _line_points(rng, x_lo, x_hi, z_lo, z_hi, c, f0):
    """Points spaced lambda/4 along a random segment of length U(2, 10) mm."""
    length = rng.uniform(2e-3, 10e-3)
    theta = rng.uniform(0.0, np.pi)
    xc = rng.uniform(x_lo, x_hi)
    zc = rng.uniform(z_lo, z_hi)
    spacing = c / f0 / 4.0
    n = max(2, int(round(length / spacing)) + 1)
    t = (np.arange(n) - (n - 1) / 2.0) * spacing
    x = xc + t * np.cos(theta)
    z = zc + t * np.sin(theta)
    keep = (x >= x_lo) & (x <= x_hi) & (z >= z_lo) & (z <= z_hi)
    w = np.full(int(keep.sum()), spacing / 1e-3)  # weight = spacing in mm
    return x[keep], z[keep], w


def make_scene(rng, wl, n_points, n_lines=0, log_amp_db=None) -> Scene:
    """Random point (and line) absorbers inside the image box.

    Sources are kept away from the array face and the box edges (lateral
    90 % of the span, depth 10 %..95 % of the range) so that the 1/r
    amplitude law never blows up at r -> 0.
    """
    x0, x1, z0, z1 = wl["x0_m"], wl["x1_m"], wl["z0_m"], wl["z1_m"]
    xm, xh = 0.5 * (x0 + x1), 0.45 * (x1 - x0)
    x_lo, x_hi = xm - xh, xm + xh
    z_lo = z0 + 0.10 * (z1 - z0)
    z_hi = z0 + 0.95 * (z1 - z0)
    xs = rng.uniform(x_lo, x_hi, n_points)
    zs = rng.uniform(z_lo, z_hi, n_points)
    if log_amp_db is not None:
        amp = 10.0 ** (-rng.uniform(0.0, log_amp_db, n_points) / 20.0)
    else:
        amp = np.ones(n_points)
    xl, zl, al = [xs], [zs], [amp]
    for _ in range(n_lines):
        x, z, w = _line_points(rng, x_lo, x_hi, z_lo, z_hi, wl["c_m_s"], wl["f0_hz"])
        xl.append(x)
        zl.append(z)
        al.append(w)
    return Scene(np.concatenate(xl), np.concatenate(zl), np.concatenate(al))


def render_rf(wl, scene: Scene, dtype=np.float64) -> np.ndarray:
    """Noise-free RF ``[N][Ns]`` for the given scene (sum of 1/r pulses)."""
    n_elem, n_s = int(wl["n_elem"]), int(wl["n_samples"])
    pitch, c, fs = wl["pitch_m"], wl["c_m_s"], wl["fs_hz"]
    t0 = wl.get("t0_s", 0.0)
    f0 = wl["f0_hz"]
    sigma = 1.0 / (2.0 * np.pi * f0)
    half = int(np.ceil(6.0 * sigma * fs)) + 1
    xe = (np.arange(n_elem) - (n_elem - 1) / 2.0) * pitch
    rf = np.zeros((n_elem, n_s), dtype=np.float64)
    taps = np.arange(-half, half + 1)
    rows = np.arange(n_elem)[:, None]
    for xs, zs, a in zip(scene.xs, scene.zs, scene.amp):
        r = np.sqrt((xs - xe) ** 2 + zs ** 2)  # [N]
        t_arr = r / c - t0
        n_c = np.floor(t_arr * fs).astype(np.int64)  # [N]
        idx = n_c[:, None] + taps[None, :]  # [N, T]
        t = idx / fs - t_arr[:, None]
        g = -(t / sigma) * np.exp(0.5 - 0.5 * (t / sigma) ** 2)
        g *= (a / (r / 1e-3))[:, None]
        ok = (idx >= 0) & (idx < n_s)
        np.add.at(rf, (np.broadcast_to(rows, idx.shape)[ok], idx[ok]), g[ok])
    return rf.astype(dtype, copy=False)


def make_frame(wl, seed, frame=0) -> np.ndarray:
    """One seeded frame ``[N][Ns]`` (float64) of the workload ``wl``."""
    rng = np.random.default_rng([int(seed), int(frame)])
    scene = make_scene(
        rng,
        wl,
        int(wl["n_points"]),
        int(wl.get("n_lines", 0)),
        wl.get("log_amp_db"),
    )
    rf = render_rf(wl, scene)
    if wl.get("unit_rms", False):
        rms = float(np.sqrt(np.mean(rf * rf)))
        if rms > 0:
            rf = rf / rms
    noise = float(wl.get("noise_frac", 0.0))
    if noise > 0:
        peak = float(np.max(np.abs(rf))) if rf.size else 0.0
        rf = rf + rng.standard_normal(rf.shape) * (noise * peak)
    return rf


def make_frames(wl, seed, n_frames, first_frame=0) -> np.ndarray:
    """``[F][N][Ns]`` float64 stack of seeded frames."""
    return np.stack([make_frame(wl, seed, first_frame + f) for f in range(n_frames)])


def quantize(rf: np.ndarray, kind: str):
    """Round float64 RF to the storage type ``kind`` ('f32', 'bf16', 'f16').

    Returns ``(storage, dequantised_float64)``.  ``storage`` is a numpy array
    of float32 (f32), uint16 bit patterns (bf16) or float16 (f16).
    BF16 uses round-to-nearest-even on the float32 bit pattern.
    """
    if kind == "f32":
        s = rf.astype(np.float32)
        return s, s.astype(np.float64)
    if kind == "f16":
        s = rf.astype(np.float16)
        return s, s.astype(np.float64)
    if kind == "bf16":
        f = np.ascontiguousarray(rf, dtype=np.float32)
        u = f.view(np.uint32).astype(np.uint64)
        lsb = (u >> 16) & 1
        u = (u + 0x7FFF + lsb) >> 16
        b = u.astype(np.uint16)
        deq = (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return b, deq
    raise ValueError(f"unknown storage kind {kind!r}")
