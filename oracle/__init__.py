"""FP64 CPU oracle for HO-DMAS photoacoustic beamforming.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_2203_14906_gb300``) never imports it and shares no code with
it: the C library here (``pa_oracle.c``) is a plain double-precision
statement of the paper's definitions, compiled with gcc.

Parity status per function (see the pins in ``tests/test_oracle_*.py``):

* delay / interpolation / DAS          pinned (analytic delta-pulse hyperbola)
* signed roots                         pinned (libm cbrt/pow, sign rules)
* DMAS, DMAS-k combine (Eqs. 2-9)      pinned (exact integer brute force,
                                        k-subset definition, closed forms)
* point-absorber peak                  pinned (true pixel, symmetry)
* FFT                                  pinned (O(M^2) DFT, analytic cosine)
* Hilbert envelope                     pinned (constant envelope of a cosine)
* depth-to-frequency mapping           pinned (hand-worked bin frequencies and
                                        Nyquist clip, an RF tone of known
                                        temporal frequency through the whole path)
* band-pass parameters                 parity unpinned (the paper gives no band)
* log compression                      pinned (closed form)
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "libpa_oracle.so")
_SRC = os.path.join(_HERE, "pa_oracle.c")
_lock = threading.Lock()
_lib = None


class Desc(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int32),
        ("pitch_m", ctypes.c_double),
        ("c_m_s", ctypes.c_double),
        ("fs_hz", ctypes.c_double),
        ("t0_s", ctypes.c_double),
        ("n_samples", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("x0_m", ctypes.c_double),
        ("x1_m", ctypes.c_double),
        ("z0_m", ctypes.c_double),
        ("z1_m", ctypes.c_double),
        ("order_k", ctypes.c_int32),
        ("f_number", ctypes.c_double),
        ("f0_hz", ctypes.c_double),
        ("band_lo_hz", ctypes.c_double),
        ("band_hi_hz", ctypes.c_double),
        ("dyn_range_db", ctypes.c_double),
        ("nearest", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile ``pa_oracle.c`` into ``oracle/_lib/libpa_oracle.so``."""
    with _lock:
        if (
            not force
            and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC)
        ):
            return _LIBPATH
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off", "-fno-fast-math",
            "-o", tmp, _SRC, "-lm",
        ]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIBPATH)
        return _LIBPATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        D = ctypes.POINTER(Desc)
        pd = ctypes.POINTER(ctypes.c_double)
        pi32 = ctypes.POINTER(ctypes.c_int32)
        i, d = ctypes.c_int, ctypes.c_double
        sig = {
            "or_elem_x": (d, [D, i]),
            "or_pix_x": (d, [D, i]),
            "or_pix_z": (d, [D, i]),
            "or_delay": (d, [D, i, i, i]),
            "or_lerp": (d, [pd, i, d]),
            "or_nearest": (d, [pd, i, d]),
            "or_apod": (d, [D, i, i, i]),
            "or_root": (d, [d, i]),
            "or_power_sums": (None, [pd, i, i, pd]),
            "or_newton": (None, [pd, i, pd]),
            "or_paper_form": (d, [pd, i, i]),
            "or_bruteforce": (d, [pd, i, i]),
            "or_dmas_k": (d, [pd, i, i]),
            "or_beamform": (None, [D, pd, pd, pd, pd]),
            "or_beamform_pixels": (None, [D, pd, i, pi32, pi32, pd, pd, pd]),
            "or_beamform_bruteforce": (None, [D, pd, pd]),
            "or_fft_size": (i, [i]),
            "or_fft": (i, [pd, pd, i, i]),
            "or_dft": (None, [pd, pd, i, i, pd, pd]),
            "or_bin_hz": (d, [D, i, i]),
            "or_post_mask": (i, [D, i, i, pd]),
            "or_envelope": (None, [pd, i, i, pd, pd]),
            "or_envelope_image": (None, [D, i, pd, pd]),
            "or_log_image": (None, [pd, ctypes.c_int64, d, pd]),
            "or_set_threads": (None, [i]),
            "or_get_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------- helpers

def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def desc(wl: dict, order_k=None) -> Desc:
    """Oracle descriptor from a workload dictionary."""
    return Desc(
        n_elem=int(wl["n_elem"]),
        pitch_m=float(wl["pitch_m"]),
        c_m_s=float(wl["c_m_s"]),
        fs_hz=float(wl["fs_hz"]),
        t0_s=float(wl.get("t0_s", 0.0)),
        n_samples=int(wl["n_samples"]),
        nx=int(wl["nx"]),
        nz=int(wl["nz"]),
        x0_m=float(wl["x0_m"]),
        x1_m=float(wl["x1_m"]),
        z0_m=float(wl["z0_m"]),
        z1_m=float(wl["z1_m"]),
        order_k=int(wl["order_k"] if order_k is None else order_k),
        f_number=float(wl.get("f_number", 0.0)),
        f0_hz=float(wl.get("f0_hz", 5e6)),
        band_lo_hz=float(wl.get("band_lo_hz", 0.0)),
        band_hi_hz=float(wl.get("band_hi_hz", 0.0)),
        dyn_range_db=float(wl.get("dyn_range_db", 60.0)),
        nearest=int(wl.get("interp", "linear") == "nearest"),
    )


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def root(s: float, k: int) -> float:
    return float(lib().or_root(float(s), int(k)))


def power_sums(x, k):
    x = _f64(x)
    p = np.zeros(k + 1)
    lib().or_power_sums(_pd(x), x.size, k, _pd(p))
    return p


def newton(p, k):
    p = _f64(p)
    e = np.zeros(k + 1)
    lib().or_newton(_pd(p), k, _pd(e))
    return e


def paper_form(s, k):
    s = _f64(s)
    return float(lib().or_paper_form(_pd(s), s.size, k))


def bruteforce(s, k):
    s = _f64(s)
    return float(lib().or_bruteforce(_pd(s), s.size, k))


def dmas_k(s, k):
    s = _f64(s)
    return float(lib().or_dmas_k(_pd(s), s.size, k))


def delay(wl, i, j, l):
    d = desc(wl)
    return float(lib().or_delay(ctypes.byref(d), i, j, l))


def lerp(row, tau):
    row = _f64(row)
    return float(lib().or_lerp(_pd(row), row.size, float(tau)))


def nearest(row, tau):
    row = _f64(row)
    return float(lib().or_nearest(_pd(row), row.size, float(tau)))


def apod(wl, i, j, l):
    d = desc(wl)
    return float(lib().or_apod(ctypes.byref(d), i, j, l))


def beamform(wl, rf, order_k=None):
    """One frame rf[N][Ns] -> dict of [nx][nz] float64 images."""
    d = desc(wl, order_k)
    rf = _f64(rf)
    assert rf.shape == (d.n_elem, d.n_samples)
    shape = (d.nx, d.nz)
    das, dmas, ho = np.empty(shape), np.empty(shape), np.empty(shape)
    lib().or_beamform(ctypes.byref(d), _pd(rf), _pd(das), _pd(dmas), _pd(ho))
    return {"das": das, "dmas": dmas, "ho": ho}


def beamform_pixels(wl, rf, j, l, order_k=None):
    d = desc(wl, order_k)
    rf = _f64(rf)
    j = np.ascontiguousarray(j, dtype=np.int32)
    l = np.ascontiguousarray(l, dtype=np.int32)
    n = j.size
    das, dmas, ho = np.empty(n), np.empty(n), np.empty(n)
    pi32 = ctypes.POINTER(ctypes.c_int32)
    lib().or_beamform_pixels(
        ctypes.byref(d), _pd(rf), n, j.ctypes.data_as(pi32),
        l.ctypes.data_as(pi32), _pd(das), _pd(dmas), _pd(ho),
    )
    return {"das": das, "dmas": dmas, "ho": ho}


def beamform_bruteforce(wl, rf, order_k=None):
    d = desc(wl, order_k)
    rf = _f64(rf)
    ho = np.empty((d.nx, d.nz))
    lib().or_beamform_bruteforce(ctypes.byref(d), _pd(rf), _pd(ho))
    return ho


def fft_size(nz):
    return int(lib().or_fft_size(int(nz)))


def fft(x, inverse=False):
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real).copy(), _f64(x.imag).copy()
    rc = lib().or_fft(_pd(re), _pd(im), re.size, int(inverse))
    if rc != 0:
        raise ValueError("length is not a power of two")
    return re + 1j * im


def dft(x, inverse=False):
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real), _f64(x.imag)
    ore, oim = np.empty(re.size), np.empty(re.size)
    lib().or_dft(_pd(re), _pd(im), re.size, int(inverse), _pd(ore), _pd(oim))
    return ore + 1j * oim


def bin_hz(wl, m, b):
    d = desc(wl)
    return float(lib().or_bin_hz(ctypes.byref(d), m, b))


def post_mask(wl, even_order, m=None):
    d = desc(wl)
    if m is None:
        m = fft_size(d.nz)
    h = np.empty(m)
    dc_only = lib().or_post_mask(ctypes.byref(d), int(bool(even_order)), m, _pd(h))
    return h, bool(dc_only)


def envelope(col, h):
    col = _f64(col)
    h = _f64(h)
    env = np.empty(col.size)
    lib().or_envelope(_pd(col), col.size, h.size, _pd(h), _pd(env))
    return env


def envelope_image(wl, raw, even_order):
    d = desc(wl)
    raw = _f64(raw)
    env = np.empty_like(raw)
    lib().or_envelope_image(ctypes.byref(d), int(bool(even_order)), _pd(raw), _pd(env))
    return env


def log_image(env, dr_db):
    env = _f64(env)
    out = np.empty_like(env)
    lib().or_log_image(_pd(env), env.size, float(dr_db), _pd(out))
    return out


OUTPUT_ORDER = ("das", "dmas", "ho")


def output_is_even(name: str, order_k: int) -> bool:
    """Band selection: DAS is order 1, DMAS order 2, HO order k."""
    return {"das": False, "dmas": True}.get(name, order_k % 2 == 0)


def frame(wl, rf, order_k=None, stages=("raw", "env", "log")):
    """Full hot path on one frame: {stage: {output: image}}."""
    k = int(wl["order_k"] if order_k is None else order_k)
    raw = beamform(wl, rf, k)
    out = {"raw": raw}
    if "env" in stages or "log" in stages:
        env = {o: envelope_image(wl, raw[o], output_is_even(o, k)) for o in OUTPUT_ORDER}
        out["env"] = env
        if "log" in stages:
            dr = float(wl.get("dyn_range_db", 60.0))
            out["log"] = {o: log_image(env[o], dr) for o in OUTPUT_ORDER}
    return out
