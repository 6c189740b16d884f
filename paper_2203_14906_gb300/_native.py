"""ctypes binding of the C ABI declared in ``include/pa_hodmas.h``.

Argument marshalling only: every step of the beamformer runs in the CUDA
library.  There is no CPU fallback; if the library cannot be built or
loaded, every entry point raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_lock = threading.Lock()
_libs: dict = {}

PA_OK, PA_EINVAL, PA_ENOMEM, PA_ECUDA, PA_ETIMEOUT, PA_EUNSUPPORTED, PA_EBUSY = range(7)
PA_RF_F32, PA_RF_BF16, PA_RF_F16 = 0, 1, 2
PA_OUT_DAS, PA_OUT_DMAS, PA_OUT_HODMAS = 1, 2, 4
PA_STAGE_RAW, PA_STAGE_ENV, PA_STAGE_LOG = 1, 2, 4
PA_INTERP_LINEAR, PA_INTERP_NEAREST = 0, 1
INTERPS = {"linear": PA_INTERP_LINEAR, "nearest": PA_INTERP_NEAREST}
PA_TABLE_AUTO, PA_TABLE_LATTICE, PA_TABLE_FULL = 0, 1, 2
DELAY_TABLES = {"auto": PA_TABLE_AUTO, "lattice": PA_TABLE_LATTICE, "full": PA_TABLE_FULL}

RF_DTYPES = {"f32": PA_RF_F32, "bf16": PA_RF_BF16, "f16": PA_RF_F16}

# Every symbol the header declares (checked by the load test).
EXPORTS = (
    "pa_plan",
    "pa_plan_footprint",
    "pa_plan_get_info",
    "pa_beamform",
    "pa_beamform_host",
    "pa_plan_use_graph",
    "pa_plan_profile",
    "pa_plan_profile_read",
    "pa_plan_set_host_schedule",
    "pa_plan_host_schedule",
    "pa_pipe_time",
    "pa_pipe_schedule",
    "pa_image_metrics",
    "pa_destroy",
    "pa_status_str",
    "pa_last_error",
    "pa_version",
    "pa_lanes_raw",
)


class PlanDesc(ctypes.Structure):
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
        ("outputs", ctypes.c_uint32),
        ("rf_dtype", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("f_number", ctypes.c_double),
        ("f0_hz", ctypes.c_double),
        ("band_lo_hz", ctypes.c_double),
        ("band_hi_hz", ctypes.c_double),
        ("dyn_range_db", ctypes.c_double),
        ("compensated", ctypes.c_int32),
        ("interp", ctypes.c_int32),
        ("delay_table", ctypes.c_int32),
    ]


class PipeModel(ctypes.Structure):
    """Pipeline model of the host-buffer path (see pa_pipe_model)."""

    _fields_ = [
        ("items_per_frame", ctypes.c_int32),
        ("resident", ctypes.c_int32),
        ("n_sets", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("upload_us", ctypes.c_double),
        ("kernel_us", ctypes.c_double),
        ("download_us", ctypes.c_double),
        ("launch_us", ctypes.c_double),
        ("wave_share", ctypes.c_double),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("lattice_m", ctypes.c_int32),
        ("tile_x", ctypes.c_int32),
        ("tile_z", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("n_tiles", ctypes.c_int32),
        ("threads", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("fft_size", ctypes.c_int32),
        ("n_outputs", ctypes.c_int32),
        ("warnings", ctypes.c_uint32),
        ("nominal_pairs", ctypes.c_int64),
        ("active_pairs", ctypes.c_int64),
        ("executed_pairs", ctypes.c_int64),
        ("device_bytes", ctypes.c_size_t),
        ("tma_staging", ctypes.c_int32),
        ("device_error_flags", ctypes.c_uint32),
        ("chunk_steps", ctypes.c_int32),
        ("lane_rows", ctypes.c_int32),
        ("tmem_columns", ctypes.c_int32),
        ("delay_table", ctypes.c_int32),
        ("table_bytes", ctypes.c_size_t),
        ("tmem_dense", ctypes.c_int32),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class PAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


PA_REGION_RECT, PA_REGION_DISC, PA_REGION_ANNULUS = 0, 1, 2
REGION_SHAPES = {"rect": PA_REGION_RECT, "disc": PA_REGION_DISC, "annulus": PA_REGION_ANNULUS}
PA_METRICS_MAX_ROIS = 4096


class Region(ctypes.Structure):
    _fields_ = [
        ("shape", ctypes.c_int32),
        ("xc_m", ctypes.c_double),
        ("zc_m", ctypes.c_double),
        ("a_m", ctypes.c_double),
        ("b_m", ctypes.c_double),
    ]


class Roi(ctypes.Structure):
    _fields_ = [("target", Region), ("background", Region)]


class Grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("x0_m", ctypes.c_double),
        ("x1_m", ctypes.c_double),
        ("z0_m", ctypes.c_double),
        ("z1_m", ctypes.c_double),
    ]


class Metrics(ctypes.Structure):
    _fields_ = [
        ("mu_in", ctypes.c_double),
        ("mu_out", ctypes.c_double),
        ("sigma_out", ctypes.c_double),
        ("snr_db", ctypes.c_double),
        ("cr_db", ctypes.c_double),
        ("gcnr", ctypes.c_double),
        ("fwhm_m", ctypes.c_double),
        ("peak", ctypes.c_double),
        ("n_in", ctypes.c_int64),
        ("n_out", ctypes.c_int64),
        ("peak_j", ctypes.c_int32),
        ("peak_l", ctypes.c_int32),
    ]


def make_region(r) -> Region:
    """``r``: a Region, or a dict {shape: rect|disc|annulus, xc_m, zc_m, a_m, b_m}."""
    if isinstance(r, Region):
        return r
    return Region(REGION_SHAPES[r["shape"]] if isinstance(r["shape"], str) else int(r["shape"]),
                  float(r["xc_m"]), float(r["zc_m"]), float(r["a_m"]), float(r.get("b_m", 0.0)))


def make_grid(wl) -> Grid:
    """Image grid of a workload dict or a PlanDesc."""
    g = (lambda k: getattr(wl, k)) if isinstance(wl, PlanDesc) else (lambda k: wl[k])
    return Grid(int(g("nx")), int(g("nz")), float(g("x0_m")), float(g("x1_m")),
                float(g("z0_m")), float(g("z1_m")))


def load(checked: bool = False, build: bool = True):
    """Load (building if stale) the CUDA library; raises if unavailable."""
    key = bool(checked)
    with _lock:
        if key in _libs:
            return _libs[key]
        override = os.environ.get("PA_LIB_PATH")  # a library built elsewhere (comparisons)
        if override:
            path = override
        else:
            path = _build.build(checked=checked) if build else _build.lib_path(checked)
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA beamformer library missing: {path}")
        L = ctypes.CDLL(path)
        vp, i32, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32
        D = ctypes.POINTER(PlanDesc)
        L.pa_plan.argtypes = [D, vp, ctypes.POINTER(vp)]
        L.pa_plan.restype = ctypes.c_int
        L.pa_plan_footprint.argtypes = [D, i32, ctypes.POINTER(ctypes.c_size_t)]
        L.pa_plan_footprint.restype = ctypes.c_int
        L.pa_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        L.pa_plan_get_info.restype = ctypes.c_int
        L.pa_beamform.argtypes = [vp, vp, i32, vp, u32, vp]
        L.pa_beamform.restype = ctypes.c_int
        L.pa_beamform_host.argtypes = [vp, vp, i32, vp, u32, vp]
        L.pa_beamform_host.restype = ctypes.c_int
        L.pa_lanes_raw.argtypes = [vp, vp, i32, vp, i32, vp]
        L.pa_lanes_raw.restype = ctypes.c_int
        L.pa_plan_use_graph.argtypes = [vp, i32]
        L.pa_plan_use_graph.restype = ctypes.c_int
        L.pa_plan_profile.argtypes = [vp, i32]
        L.pa_plan_profile.restype = ctypes.c_int
        L.pa_plan_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64)]
        L.pa_plan_profile_read.restype = ctypes.c_int
        I32P = ctypes.POINTER(ctypes.c_int32)
        L.pa_plan_set_host_schedule.argtypes = [vp, i32, u32, I32P, i32]
        L.pa_plan_set_host_schedule.restype = ctypes.c_int
        L.pa_plan_host_schedule.argtypes = [vp, i32, u32, I32P, i32, I32P, I32P]
        L.pa_plan_host_schedule.restype = ctypes.c_int
        L.pa_pipe_time.argtypes = [ctypes.POINTER(PipeModel), I32P, i32,
                                   ctypes.POINTER(ctypes.c_double)]
        L.pa_pipe_time.restype = ctypes.c_int
        L.pa_pipe_schedule.argtypes = [ctypes.POINTER(PipeModel), i32, i32, I32P, i32, I32P]
        L.pa_pipe_schedule.restype = ctypes.c_int
        L.pa_log_compress_noalloc.argtypes = [vp, i32, ctypes.c_int64, ctypes.c_float, vp, vp]
        L.pa_log_compress_noalloc.restype = ctypes.c_int
        L.pa_image_metrics.argtypes = [ctypes.POINTER(Grid), vp, i32, ctypes.POINTER(Roi), i32,
                                       vp, vp]
        L.pa_image_metrics.restype = ctypes.c_int
        L.pa_destroy.argtypes = [vp]
        L.pa_destroy.restype = ctypes.c_int
        L.pa_status_str.argtypes = [ctypes.c_int]
        L.pa_status_str.restype = ctypes.c_char_p
        L.pa_last_error.argtypes = []
        L.pa_last_error.restype = ctypes.c_char_p
        L.pa_version.argtypes = []
        L.pa_version.restype = i32
        _libs[key] = L
        return L


def check(L, status):
    if status != PA_OK:
        raise PAError(status, f"{L.pa_status_str(status).decode()}: {L.pa_last_error().decode()}")


def make_desc(wl: dict, order_k=None, outputs=7, rf_dtype=None, max_batch=1,
              compensated=None) -> PlanDesc:
    """C descriptor from a workload dictionary (keys as in ``synth.configs``)."""
    dt = rf_dtype if rf_dtype is not None else wl.get("rf_dtype", "f32")
    return PlanDesc(
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
        outputs=int(outputs),
        rf_dtype=RF_DTYPES[dt] if isinstance(dt, str) else int(dt),
        max_batch=int(max_batch),
        f_number=float(wl.get("f_number", 0.0)),
        f0_hz=float(wl.get("f0_hz", 5e6)),
        band_lo_hz=float(wl.get("band_lo_hz", 0.0)),
        band_hi_hz=float(wl.get("band_hi_hz", 0.0)),
        dyn_range_db=float(wl.get("dyn_range_db", 60.0)),
        compensated=int(wl.get("compensated", 0) if compensated is None else compensated),
        interp=INTERPS[wl.get("interp", "linear")],
        delay_table=DELAY_TABLES[wl.get("delay_table", "auto")],
    )


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Plan:
    """Resident plan: delay/apodisation table, RF windows, post masks."""

    def __init__(self, desc: PlanDesc, stream=None, checked: bool = False):
        self._L = load(checked)
        self.desc = desc
        h = ctypes.c_void_p()
        check(self._L, self._L.pa_plan(ctypes.byref(desc), _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = PlanInfo()
        check(self._L, self._L.pa_plan_get_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def out_shape(self, n_frames, stages):
        n_st = bin(int(stages) & 7).count("1")
        n_out = bin(int(self.desc.outputs) & 7).count("1")
        return (n_frames, n_st, n_out, self.desc.nx, self.desc.nz)

    def beamform(self, rf_dev_ptr: int, n_frames: int, out_dev_ptr: int, stages: int, stream=None):
        """Device-pointer call (pa_beamform); asynchronous on ``stream``."""
        check(self._L, self._L.pa_beamform(self._h, rf_dev_ptr, int(n_frames), out_dev_ptr,
                                           int(stages), _stream_handle(stream)))

    def beamform_host(self, rf_host_ptr: int, n_frames: int, out_host_ptr: int, stages: int,
                      stream=None):
        """Host-pointer call (pa_beamform_host); returns when output is written."""
        check(self._L, self._L.pa_beamform_host(self._h, rf_host_ptr, int(n_frames), out_host_ptr,
                                                int(stages), _stream_handle(stream)))

    def set_host_schedule(self, n_frames: int, stages: int, chunks):
        """Fix the chunk schedule of beamform_host for (n_frames, stages);
        an empty list returns that shape to tuning."""
        c = (ctypes.c_int32 * max(1, len(chunks)))(*[int(x) for x in chunks])
        check(self._L, self._L.pa_plan_set_host_schedule(self._h, int(n_frames), int(stages), c,
                                                         len(chunks)))

    def host_schedule(self, n_frames: int, stages: int):
        """(chunks, state) the next beamform_host call of this shape uses;
        state 1 tuning, 2 tuned, 3 set by the caller."""
        room = max(1, int(n_frames))
        c = (ctypes.c_int32 * room)()
        n, st = ctypes.c_int32(), ctypes.c_int32()
        check(self._L, self._L.pa_plan_host_schedule(self._h, int(n_frames), int(stages), c, room,
                                                     ctypes.byref(n), ctypes.byref(st)))
        return [c[i] for i in range(n.value)], st.value

    def use_graph(self, enable: bool = True):
        """Launch each sequence as a CUDA graph (default) or kernel by kernel."""
        check(self._L, self._L.pa_plan_use_graph(self._h, int(bool(enable))))

    def profile(self, enable: bool = True, fused_only: bool = False):
        """Record CUDA events around each of this plan's kernel launches (or,
        with fused_only, around the fused beamforming kernel's alone)."""
        mode = 0 if not enable else (2 if fused_only else 1)
        check(self._L, self._L.pa_plan_profile(self._h, mode))

    def profile_read(self):
        """{kernel: (total_ms, launches)} since the last read; synchronises."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        check(self._L, self._L.pa_plan_profile_read(self._h, ms, n))
        return {name: (ms[i], n[i]) for i, name in enumerate(("bf_fused", "post", "log"))}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.pa_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _pipe_model(items_per_frame, resident, upload_us, kernel_us, download_us, launch_us=8.0,
                wave_share=1.0, n_sets=3) -> PipeModel:
    return PipeModel(items_per_frame=int(items_per_frame), resident=int(resident),
                     n_sets=int(n_sets), reserved=0, upload_us=float(upload_us),
                     kernel_us=float(kernel_us), download_us=float(download_us),
                     launch_us=float(launch_us), wave_share=float(wave_share))


def pipe_time(chunks, checked: bool = False, **model) -> float:
    """Makespan (us) of a chunk schedule under the host-path pipeline model
    (keyword arguments as the fields of PipeModel; no GPU needed)."""
    L = load(checked)
    m = _pipe_model(**model)
    c = (ctypes.c_int32 * max(1, len(chunks)))(*[int(x) for x in chunks])
    us = ctypes.c_double()
    check(L, L.pa_pipe_time(ctypes.byref(m), c, len(chunks), ctypes.byref(us)))
    return us.value


def pipe_schedule(n_frames: int, max_chunk: int, checked: bool = False, **model) -> list:
    """Least-makespan schedule of the searched family (no GPU needed)."""
    L = load(checked)
    m = _pipe_model(**model)
    room = max(1, int(n_frames))
    c = (ctypes.c_int32 * room)()
    n = ctypes.c_int32()
    check(L, L.pa_pipe_schedule(ctypes.byref(m), int(n_frames), int(max_chunk), c, room,
                                ctypes.byref(n)))
    return [c[i] for i in range(n.value)]


def footprint(desc: PlanDesc, n_frames: int, checked: bool = False) -> int:
    L = load(checked)
    b = ctypes.c_size_t()
    check(L, L.pa_plan_footprint(ctypes.byref(desc), int(n_frames), ctypes.byref(b)))
    return int(b.value)
