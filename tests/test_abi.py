"""Host-side checks of the C ABI that need no GPU.

* The library builds for sm_103a, loads, and exports every function that
  ``include/*.h`` declares.
* Descriptor validation rejects bad requests before any device call.
* The oracle and the CUDA library share no code (no cross includes).
"""

import ctypes
import glob
import os
import re

import pytest

import synth
from paper_2203_14906_gb300 import _build, _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(pa_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_function():
    L = _native.load()
    declared = _declared_functions()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, f"missing exports: {missing}"
    assert set(_native.EXPORTS) <= declared


def test_version_and_status_strings():
    L = _native.load()
    assert L.pa_version() >= 105
    assert L.pa_status_str(0) == b"ok"
    assert L.pa_status_str(1) == b"invalid argument"


def _status(desc, n_frames=1):
    L = _native.load()
    b = ctypes.c_size_t()
    return L.pa_plan_footprint(ctypes.byref(desc), n_frames, ctypes.byref(b)), b.value


def test_validation_rejects_bad_descriptors():
    wl = synth.workload("cfg1")
    ok, nbytes = _status(_native.make_desc(wl))
    assert ok == _native.PA_OK and nbytes > 0
    bad = [
        dict(order_k=0),
        dict(order_k=9),
        dict(n_elem=2, order_k=3),  # N < k
        dict(nx=0),
        dict(nz=0),
        dict(n_samples=1),
        dict(z0_m=-1e-3),
        dict(x1_m=-9.6e-3),  # empty lateral extent
        dict(nx=100, delay_table="lattice"),  # pitch / dx not an integer
        dict(nx=32, delay_table="lattice"),  # pitch / dx = 1/2
        dict(nx=64 * 64, delay_table="lattice"),  # pitch / dx = 64 > 32
    ]
    for over in bad:
        w = dict(wl)
        w.update(over)
        if "n_elem" in over:
            w["x0_m"], w["x1_m"] = -over["n_elem"] * 1.5e-4, over["n_elem"] * 1.5e-4
            w["nx"] = over["n_elem"] * 2
        st, _ = _status(_native.make_desc(w, order_k=w["order_k"]))
        assert st == _native.PA_EINVAL, (over, st)
    d = _native.make_desc(wl)
    d.outputs = 0
    assert _status(d)[0] == _native.PA_EINVAL
    d = _native.make_desc(wl)
    d.rf_dtype = 7
    assert _status(d)[0] == _native.PA_EINVAL
    d = _native.make_desc(wl)
    d.interp = 2
    assert _status(d)[0] == _native.PA_EINVAL
    assert _status(_native.make_desc(dict(wl, interp="nearest")))[0] == _native.PA_OK
    d = _native.make_desc(wl)
    d.delay_table = 3
    assert _status(d)[0] == _native.PA_EINVAL


def test_grids_off_the_lattice_take_the_full_table():
    """Any lateral pitch is accepted; off the lattice the footprint counts
    the full table (4 bytes per padded pixel and channel step, N + 3 or more
    steps, plus 4 with apodisation), and a table above the stated maximum is
    refused."""
    wl = synth.workload("cfg1")
    base = _status(_native.make_desc(wl))[1]
    for nx, span in ((100, 19.2e-3), (32, 19.2e-3), (64 * 64, 19.2e-3), (7, 3e-3)):
        w = dict(wl, nx=nx, x0_m=-span / 2, x1_m=span / 2)
        st, nbytes = _status(_native.make_desc(w))
        assert st == _native.PA_OK, nx
        # nv >= N + 6 virtual channels, nz_pad = 128 rows
        assert nbytes - base >= nx * 64 * 128 * 4 - 3 * 1024 * 1024, nx
    # lattice grids keep the small table unless the full one is asked for
    st, nbytes_full = _status(_native.make_desc(dict(wl, delay_table="full")))
    assert st == _native.PA_OK and nbytes_full - base > 0.9 * 128 * 64 * 128 * 4
    w = dict(wl, nx=32768, nz=2048)  # 32768 x 2048 x 68 steps x 4 B > 16 GiB
    assert _status(_native.make_desc(w))[0] == _native.PA_EUNSUPPORTED


def test_plan_validation_happens_before_device_work():
    L = _native.load()
    h = ctypes.c_void_p()
    d = _native.make_desc(synth.workload("cfg1"), order_k=0)
    assert L.pa_plan(ctypes.byref(d), None, ctypes.byref(h)) == _native.PA_EINVAL
    assert b"order_k" in L.pa_last_error()
    assert L.pa_destroy(None) == _native.PA_OK


def test_footprint_grows_with_frames():
    wl = synth.workload("cfg2")
    d = _native.make_desc(wl)
    a = _native.footprint(d, 1)
    b = _native.footprint(d, 8)
    assert b > a
    per = (b - a) / 7
    want = 128 * 2048 * 4 + 3 * 3 * 512 * 512 * 4
    assert abs(per - want) < 1e-6 * want + 1


def test_oracle_and_cuda_sources_share_nothing():
    cu = glob.glob(os.path.join(ROOT, "paper_2203_14906_gb300", "csrc", "*"))
    for f in cu:
        txt = open(f).read()
        assert "pa_oracle" not in txt and "oracle/" not in txt, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        txt = open(f).read()
        assert "pa_hodmas" not in txt and "pa_internal" not in txt, f
    pkg = glob.glob(os.path.join(ROOT, "paper_2203_14906_gb300", "*.py"))
    for f in pkg:
        txt = open(f).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def test_build_is_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.build())


def test_server_config_validation_without_gpu():
    from paper_2203_14906_gb300 import serving

    L = _native.load()
    serving._bind(L)
    h = ctypes.c_void_p()
    bad = serving.ServerConfig(0, 1, 1, 1, 4)  # zero budget
    assert L.pa_server_create(ctypes.byref(bad), ctypes.byref(h)) == _native.PA_EINVAL
    bad = serving.ServerConfig(1 << 30, 0, 1, 1, 4)  # no slots
    assert L.pa_server_create(ctypes.byref(bad), ctypes.byref(h)) == _native.PA_EINVAL
    bad = serving.ServerConfig(1 << 30, 1, 1, 1, 8)  # bad stage mask
    assert L.pa_server_create(ctypes.byref(bad), ctypes.byref(h)) == _native.PA_EINVAL
    t = ctypes.c_uint64()
    d = _native.make_desc(synth.workload("cfg1"))
    assert L.pa_server_submit(None, ctypes.byref(d), None, None, 0.0, ctypes.byref(t)) == _native.PA_EINVAL
    assert L.pa_server_destroy(None) == _native.PA_OK


def test_metrics_validation_without_gpu():
    """pa_image_metrics checks its arguments before touching the device."""
    L = _native.load()
    g = _native.make_grid(dict(nx=16, nz=16, x0_m=0.0, x1_m=1e-3, z0_m=0.0, z1_m=1e-3))
    reg = _native.make_region
    roi = (_native.Roi * 1)(_native.Roi(reg(dict(shape="disc", xc_m=0, zc_m=0, a_m=1e-4)),
                                        reg(dict(shape="annulus", xc_m=0, zc_m=0, a_m=1e-4,
                                                 b_m=3e-4))))
    call = lambda grid, n_img, rois, n_roi: L.pa_image_metrics(  # noqa: E731
        ctypes.byref(grid), None, n_img, rois, n_roi, None, None)
    assert call(g, 0, roi, 1) == _native.PA_OK  # nothing to do
    assert call(g, 1, roi, 0) == _native.PA_EINVAL
    assert call(g, 1, roi, _native.PA_METRICS_MAX_ROIS + 1) == _native.PA_EINVAL
    assert call(g, 1, roi, 1) == _native.PA_EINVAL  # null image / output buffers
    assert b"null buffer" in L.pa_last_error()
    bad = (_native.Roi * 1)(_native.Roi(_native.Region(7, 0, 0, 1e-4, 0), roi[0].background))
    assert call(g, 1, bad, 1) == _native.PA_EINVAL
    neg = (_native.Roi * 1)(_native.Roi(reg(dict(shape="disc", xc_m=0, zc_m=0, a_m=-1.0)),
                                        roi[0].background))
    assert call(g, 1, neg, 1) == _native.PA_EINVAL
    g.x1_m = g.x0_m
    assert call(g, 1, roi, 1) == _native.PA_EINVAL
    assert L.pa_image_metrics(None, None, 1, roi, 1, None, None) == _native.PA_EINVAL
    assert ctypes.sizeof(_native.Metrics) == 88
