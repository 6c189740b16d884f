"""GPU (CUDA, sm_103a) vs FP64 oracle, element by element, through the C ABI.

Tolerances: FP32 path 1e-4 of the image peak (RAW and ENV), 0.05 dB after
log compression on pixels within 6 dB of the peak; reduced-precision path
5e-3 of the peak against the oracle on the unquantised RF.
"""

import numpy as np
import pytest

import synth
from gpu_util import assert_parity, compare, oracle_frames, run_gpu

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL_LP = 5e-3


def _frames(wl, seeds):
    return np.stack([synth.make_frame(wl, s) for s in seeds])


def test_cfg1_all_seeds_batched_k3():
    """cfg1 (64 el, 1024 samples, 128x128): five seeded frames in one launch."""
    wl = synth.workload("cfg1")
    rf = _frames(wl, wl["seeds"])
    out, info, deq = run_gpu(wl, rf, 3)
    assert info["device_error_flags"] == 0
    assert info["tma_staging"] == 0  # FP32 RF: vectorised-load staging by default
    res = compare(out, oracle_frames(wl, deq, 3))
    assert_parity(res, TOL32, what="cfg1 k=3")


@pytest.mark.parametrize("k", [1, 2, 4, 5, 6, 7, 8])
def test_cfg1_every_order(k):
    wl = synth.workload("cfg1")
    rf = _frames(wl, [1])
    out, _, deq = run_gpu(wl, rf, k)
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"cfg1 k={k}")


@pytest.mark.parametrize("k", [6, 7, 8])
def test_high_orders_compensated_bf16(k):
    """Orders 6-8 on the compensated BF16 path (generic roots and powers,
    Newton's identities in FP64)."""
    wl = synth.workload("cfg1", rf_dtype="bf16")
    rf = _frames(wl, [2])
    out, info, deq = run_gpu(wl, rf, k, rf_dtype="bf16", compensated=1)
    assert info["device_error_flags"] == 0
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"bf16 k={k} compute")
    assert_parity(compare(out, oracle_frames(wl, rf, k)), TOL_LP, what=f"bf16 k={k} e2e")


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_cfg2_full_size(k):
    """cfg2 at full size: 128 el x 2048 samples, 512x512, orders 2..5."""
    wl = synth.workload("cfg2")
    rf = _frames(wl, wl["seeds"])
    out, _, deq = run_gpu(wl, rf, k)
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"cfg2 k={k}")


def test_ragged_grid_odd_aperture_unaligned_samples():
    """Grid not a multiple of the tile, odd N, Ns % 4 != 0 (scalar staging),
    lattice m = 2, several tiles and ragged tails in both directions."""
    wl = synth.workload("cfg1", n_elem=37, n_samples=1001, nx=74, nz=77, z1_m=18e-3)
    wl["x0_m"], wl["x1_m"] = -37 * 0.15e-3, 37 * 0.15e-3
    rf = _frames(wl, [7, 8])
    for k in (3, 4):
        out, info, deq = run_gpu(wl, rf, k, max_batch=1)
        assert info["lattice_m"] == 2
        assert info["tma_staging"] == 0  # Ns % 4 != 0: vectorised-load staging
        assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"ragged k={k}")


@pytest.mark.parametrize("k,dtype", [(3, "f32"), (2, "f32"), (5, "bf16")])
def test_small_grid_in_a_large_batch_takes_wide_tiles(k, dtype):
    """A 128 x 128 grid in a plan for 64 frames (1024 tiles of 32 x 32 per
    full launch) is tiled 32 columns wide; two frames through that plan
    (ragged rows: nz = 120) match the oracle, and a one-frame plan of the
    same grid keeps 16-column tiles with the same results."""
    wl = synth.workload("cfg1", nz=120, z1_m=18.75e-3)
    rf = _frames(wl, [21, 22])
    ref = None
    for mb, tile in ((64, 32), (1, 16)):
        out, info, deq = run_gpu(wl, rf, k, rf_dtype=dtype, compensated=int(dtype != "f32"),
                                 max_batch=mb)
        assert info["tile_x"] == tile, (mb, info["tile_x"])
        assert info["device_error_flags"] == 0
        # against the oracle on the dequantised RF: the FP32 bar for both forms
        assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"k={k} max_batch={mb}")
        if ref is None:
            ref = out
        else:
            assert np.max(np.abs(out[:, 0] - ref[:, 0])) <= 1e-5 * np.max(np.abs(ref[:, 0]))


def test_pixels_beyond_the_record_and_t0():
    """Short records (many delays fall off the end) and t0 > 0 (negative
    delays near the array): those channels must drop out exactly."""
    wl = synth.workload("cfg1", n_samples=300, t0_s=2.0e-6, nz=96)
    rf = _frames(wl, [3])
    out, _, deq = run_gpu(wl, rf, 3)
    assert_parity(compare(out, oracle_frames(wl, deq, 3)), TOL32, what="invalid delays")


@pytest.mark.parametrize("m", [1, 4, 8, 16])
def test_lattice_factors(m):
    """Pitch / lateral pixel pitch = m (serving mixes use 1..16)."""
    n = 32
    wl = synth.workload("cfg1", n_elem=n, nx=n * m, nz=64, z1_m=12e-3)
    wl["x0_m"], wl["x1_m"] = -n * 0.15e-3, n * 0.15e-3
    rf = _frames(wl, [5])
    out, info, deq = run_gpu(wl, rf, 3)
    assert info["lattice_m"] == m
    assert_parity(compare(out, oracle_frames(wl, deq, 3)), TOL32, what=f"m={m}")


def test_apodised_cfg5_frames_bf16():
    """cfg5 geometry (1024x1024, 128 el, F# 1.5 Hann, k=4), BF16 RF with
    compensated sums: two frames."""
    wl = synth.workload("cfg5")
    rf = np.stack([synth.make_frame(wl, 41, f) for f in range(2)])
    out, info, deq = run_gpu(wl, rf, 4, rf_dtype="bf16", compensated=1)
    assert info["tma_staging"] == 1  # 16-bit RF: TMA staging by default
    assert info["device_error_flags"] == 0
    assert info["active_pairs"] < info["nominal_pairs"]
    assert info["executed_pairs"] < info["nominal_pairs"]
    ref_deq = oracle_frames(wl, deq, 4)
    assert_parity(compare(out, ref_deq), TOL32, what="cfg5 vs dequantised")
    ref = oracle_frames(wl, rf, 4)
    assert_parity(compare(out, ref), TOL_LP, what="cfg5 vs unquantised")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("k", [3, 5])
def test_cfg3_precision(dtype, k):
    """cfg3 (256 el, 4096 samples at 50 MHz, 1024x1024): 16-bit RF, Kahan
    power sums, FP64 combine; error against the oracle on the unquantised
    RF (end to end) and on the dequantised RF (compute only)."""
    wl = synth.workload("cfg3")
    rf = _frames(wl, wl["seeds"])
    out, _, deq = run_gpu(wl, rf, k, rf_dtype=dtype, compensated=1)
    assert_parity(compare(out, oracle_frames(wl, rf, k)), TOL_LP, what=f"cfg3 {dtype} e2e")
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"cfg3 {dtype} compute")


def test_all_zero_frame_and_empty_call():
    import torch

    import paper_2203_14906_gb300 as pa

    wl = synth.workload("cfg1", nx=64, nz=64)
    out, _, _ = run_gpu(wl, np.zeros((1, 64, 1024)), 3)
    assert np.all(out[0, :2] == 0.0)
    assert np.all(out[0, 2] == -60.0)
    with pa.Plan(pa.make_desc(wl)) as plan:
        rf = torch.zeros((0, 64, 1024), device="cuda")
        o = pa.beamform(plan, rf, 7)
        assert o.shape[0] == 0


def test_minimum_aperture_n_equals_k():
    wl = synth.workload("cfg1", n_elem=5, nx=10, nz=40, z1_m=10e-3)
    wl["x0_m"], wl["x1_m"] = -5 * 0.15e-3, 5 * 0.15e-3
    rf = _frames(wl, [2])
    out, _, deq = run_gpu(wl, rf, 5)
    assert_parity(compare(out, oracle_frames(wl, deq, 5)), TOL32, what="N=k")


def test_stage_and_output_subsets_match_full():
    """Any subset of stages/outputs gives the same planes as the full call."""
    wl = synth.workload("cfg1", nx=64, nz=96, z1_m=15e-3)
    rf = _frames(wl, [4])
    full, _, _ = run_gpu(wl, rf, 3)
    for outputs, stages in ((4, 4), (1, 2), (6, 5), (2, 1)):
        sub, _, _ = run_gpu(wl, rf, 3, outputs=outputs, stages=stages)
        s_idx = [i for i, b in enumerate((1, 2, 4)) if stages & b]
        o_idx = [i for i, b in enumerate((1, 2, 4)) if outputs & b]
        want = full[:, s_idx][:, :, o_idx]
        assert np.array_equal(sub, want), (outputs, stages)


def test_frame_result_independent_of_batch():
    """A frame alone and inside a batch gives bitwise identical images."""
    wl = synth.workload("cfg1")
    rf = _frames(wl, [1, 2, 3])
    batch, _, _ = run_gpu(wl, rf, 4)
    for f in range(3):
        alone, _, _ = run_gpu(wl, rf[f:f + 1], 4)
        assert np.array_equal(alone[0], batch[f])
    split, _, _ = run_gpu(wl, rf, 4, max_batch=2)
    assert np.array_equal(split, batch)


def test_host_buffer_path_matches_device_path():
    wl = synth.workload("cfg1")
    rf = _frames(wl, [1, 2, 3, 4, 5])
    dev, _, _ = run_gpu(wl, rf, 3)
    host, _, _ = run_gpu(wl, rf, 3, host=True, max_batch=2)
    assert np.array_equal(dev, host)


def test_host_schedule_tuning_keeps_bits():
    """pa_beamform_host times candidate chunk schedules on its first calls of
    a shape: every call gives the device path's bits, tuning ends with a
    valid schedule, and caller-set ragged schedules give the same bits."""
    import torch

    import paper_2203_14906_gb300 as pa

    wl = synth.workload("cfg1")
    rf = _frames(wl, range(1, 8))  # 7 frames
    store, _ = synth.quantize(rf, "f32")
    st = pa.PA_STAGE_ENV | pa.PA_STAGE_LOG
    with pa.Plan(pa.make_desc(wl, order_k=3, max_batch=4)) as plan:
        dev = pa.beamform(plan, torch.from_numpy(store).cuda(), st)
        torch.cuda.synchronize()
        dev = dev.cpu().numpy()
        sched, state = plan.host_schedule(7, st)
        assert state == 1 and sum(sched) == 7
        calls = 0
        while state == 1 and calls < 200:
            assert np.array_equal(pa.beamform_host(plan, store, st), dev), sched
            calls += 1
            sched, state = plan.host_schedule(7, st)
        assert state == 2 and sum(sched) == 7 and max(sched) <= 4 and calls >= 2
        for fixed in ([3, 1, 2, 1], [1] * 7, [4, 3]):
            plan.set_host_schedule(7, st, fixed)
            assert plan.host_schedule(7, st) == (fixed, 3)
            assert np.array_equal(pa.beamform_host(plan, store, st), dev), fixed
        plan.set_host_schedule(7, st, [])
        assert plan.host_schedule(7, st) == (sched, 2)
        for bad in ([4, 4], [5, 2], [7, 0], [3, 3]):
            with pytest.raises(pa.PAError):
                plan.set_host_schedule(7, st, bad)
        # another shape of the same plan tunes on its own
        assert plan.host_schedule(5, st)[1] == 1
        assert np.array_equal(pa.beamform_host(plan, store[:5], st), dev[:5])


def test_host_call_graph_with_pinned_buffers():
    """Pinned host buffers run the whole host-path call as one graph (per
    frames, stages and schedule; rebuilt while the schedule is tuned, host
    addresses rewritten when the caller's buffers change); pageable buffers
    take the stream form.  Every call gives the device path's bits."""
    import torch

    import paper_2203_14906_gb300 as pa

    wl = synth.workload("cfg1")
    rf = _frames(wl, range(1, 10))  # 9 frames
    store, _ = synth.quantize(rf, "f32")
    st = pa.PA_STAGE_ENV | pa.PA_STAGE_LOG
    with pa.Plan(pa.make_desc(wl, order_k=4, max_batch=4)) as plan:
        dev = pa.beamform(plan, torch.from_numpy(store).cuda(), st)
        torch.cuda.synchronize()
        dev = dev.cpu().numpy()
        rf_p = torch.from_numpy(store).pin_memory()
        outs = [torch.empty(plan.out_shape(9, st), dtype=torch.float32).pin_memory()
                for _ in range(2)]
        for call in range(60):
            out = outs[call % 2] if call % 7 else None  # None: a pageable result array
            got = pa.beamform_host(plan, rf_p if call % 5 else store, st, out=out)
            got = got.numpy() if isinstance(got, torch.Tensor) else got
            assert np.array_equal(got, dev), call
        assert plan.host_schedule(9, st)[1] == 2
        assert plan.info()["device_error_flags"] == 0


def _random_workload(rng, case):
    m = int(rng.integers(1, 5))
    n_elem = int(rng.integers(8, 72))
    dx = 0.3e-3 / m
    nx = int(rng.integers(9, 110))
    nz = int(rng.integers(17, 160))
    dz = float(rng.uniform(40e-6, 110e-6))
    x0 = -nx * dx / 2 + float(rng.uniform(-1.0, 1.0)) * 2e-3
    z0 = float(rng.uniform(0.0, 4e-3))
    wl = synth.workload(
        "cfg1", n_elem=n_elem, nx=nx, nz=nz, x0_m=x0, x1_m=x0 + nx * dx, z0_m=z0,
        z1_m=z0 + nz * dz, n_samples=int(rng.integers(300, 1400)),
        t0_s=float(rng.choice([0.0, 0.5e-6])), n_points=3,
        f_number=1.5 if case % 4 == 3 else 0.0,
        interp="nearest" if case % 3 == 2 else "linear")
    wl["seeds"] = [int(rng.integers(1, 1000))]
    return wl


@pytest.mark.parametrize("case", range(24))
def test_random_geometries(case):
    """Seeded random geometries: lattice factor 1-4, 8-71 channels, ragged
    grids (9-109 x 17-159), record lengths not divisible by 4, off-centre
    windows, time offsets, F-number apodisation, nearest-sample delays, every
    RF type and orders 1-8; every stage against the oracle on the same
    (dequantised) RF at the FP32 tolerance."""
    rng = np.random.default_rng(1000 + case)
    wl = _random_workload(rng, case)
    k = int(rng.integers(1, 9))
    dtype = str(rng.choice(["f32", "bf16", "f16"]))
    rf = _frames(wl, [wl["seeds"][0], wl["seeds"][0] + 1])
    out, info, deq = run_gpu(wl, rf, k, rf_dtype=dtype, compensated=int(dtype != "f32"),
                             max_batch=int(rng.integers(1, 3)))
    assert info["device_error_flags"] == 0
    what = (f"case {case}: N={wl['n_elem']} m={info['lattice_m']} grid={wl['nx']}x{wl['nz']} "
            f"Ns={wl['n_samples']} k={k} {dtype} F#={wl['f_number']} {wl['interp']}")
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=what)


def test_checked_build_raises_no_bounds_flags():
    """Bounds-checked build of the same kernels over the edge-case geometries."""
    cases = [
        (synth.workload("cfg1"), 3, "f32", 0),
        (synth.workload("cfg1", n_samples=300, t0_s=2e-6, nz=96), 5, "f32", 0),
        (synth.workload("cfg5", nx=256, nz=256), 4, "bf16", 1),
        (synth.workload("cfg1", n_samples=300, t0_s=2e-6, nz=96, interp="nearest"), 3, "f32", 0),
    ]
    for wl, k, dt, comp in cases:
        rf = synth.make_frame(wl, 1)[None]
        _, info, _ = run_gpu(wl, rf, k, rf_dtype=dt, compensated=comp, checked=True)
        assert info["device_error_flags"] == 0, (wl["name"], k)


def test_graph_launch_matches_direct_launch():
    """CUDA-graph launches (default) and kernel-by-kernel launches give the
    same bits, including repeated graph launches on new buffers."""
    import torch

    import paper_2203_14906_gb300 as pa

    wl = synth.workload("cfg1")
    rf = torch.from_numpy(synth.quantize(_frames(wl, [1, 2, 3]), "f32")[0]).cuda()
    with pa.Plan(pa.make_desc(wl, order_k=3, max_batch=2)) as plan:
        plan.use_graph(False)
        direct = pa.beamform(plan, rf, 7)
        plan.use_graph(True)
        g1 = pa.beamform(plan, rf, 7)
        g2 = pa.beamform(plan, rf.clone(), 7)
        g3 = pa.beamform(plan, rf[1:].contiguous(), 7)
        torch.cuda.synchronize()
    assert torch.equal(direct, g1) and torch.equal(direct, g2)
    assert torch.equal(direct[1:], g3)


def test_kernel_timing_in_both_launch_modes():
    """Kernel timing works on the graph path (event-record nodes around each
    kernel) and kernel by kernel: one timed launch per kernel per call, the
    same bits as untimed launches, and timed graphs kept apart from the
    untimed ones."""
    import torch

    import paper_2203_14906_gb300 as pa

    wl = synth.workload("cfg1")
    rf = torch.from_numpy(synth.quantize(_frames(wl, [4, 5, 6]), "f32")[0]).cuda()
    with pa.Plan(pa.make_desc(wl, order_k=3, max_batch=3)) as plan:
        ref = pa.beamform(plan, rf, 7)
        for graph in (True, False):
            plan.use_graph(graph)
            plan.profile(True)
            outs = [pa.beamform(plan, rf, 7) for _ in range(3)]
            outs.append(pa.beamform(plan, rf, 3))  # no log stage
            prof = plan.profile_read()
            plan.profile(False)
            assert prof["bf_fused"][1] == 4 and prof["post"][1] == 4, (graph, prof)
            assert prof["log"][1] == 3, (graph, prof)
            assert all(v[0] > 0.0 for v in prof.values()), (graph, prof)
            for o in outs[:3]:
                assert torch.equal(o, ref)
            assert torch.equal(outs[3], ref[:, :2])  # stages raw + envelope
            # the fused kernel alone
            plan.profile(True, fused_only=True)
            o = pa.beamform(plan, rf, 7)
            prof = plan.profile_read()
            plan.profile(False)
            assert prof["bf_fused"][1] == 1 and prof["bf_fused"][0] > 0.0, (graph, prof)
            assert prof["post"][1] == 0 and prof["log"][1] == 0, (graph, prof)
            assert torch.equal(o, ref)
        plan.use_graph(True)
        again = pa.beamform(plan, rf, 7)
        assert plan.profile_read()["bf_fused"][1] == 0
        assert torch.equal(again, ref)
        # the host-buffer path, timed (pinned buffers: per-chunk graphs
        # instead of the whole-call graph) and untimed
        rf_h = rf.cpu().pin_memory()
        out_h = torch.empty(tuple(ref.shape), dtype=torch.float32).pin_memory()
        plan.profile(True, fused_only=True)
        pa.beamform_host(plan, rf_h, 7, out=out_h)
        prof = plan.profile_read()
        plan.profile(False)
        assert prof["bf_fused"][1] >= 1 and prof["post"][1] == 0, prof
        assert torch.equal(out_h, ref.cpu())
        out_h.zero_()
        pa.beamform_host(plan, rf_h, 7, out=out_h)
        assert torch.equal(out_h, ref.cpu())
        from paper_2203_14906_gb300._native import check

        with pytest.raises(pa.PAError):
            check(plan._L, plan._L.pa_plan_profile(plan._h, 3))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tma_and_load_staging_agree(dtype, monkeypatch):
    """Both RF staging paths (TMA boxes, vectorised loads) give the same bits."""
    wl = synth.workload("cfg2", nx=256, nz=256, z1_m=20e-3)
    rf = _frames(wl, [11, 12])
    outs = {}
    for st in ("tma", "loads"):
        monkeypatch.setenv("PA_STAGING", st)
        out, info, _ = run_gpu(wl, rf, 5, rf_dtype=dtype, compensated=int(dtype != "f32"))
        assert info["tma_staging"] == (st == "tma")
        assert info["device_error_flags"] == 0
        outs[st] = out
    assert np.array_equal(outs["tma"], outs["loads"])


def test_lane_groups_keep_bits(monkeypatch):
    """Lane groups of 32, 16 and 8 depth rows (one, two or four slots per
    warp) give the same bits: each pixel's channel order is unchanged."""
    for wl, k in ((synth.workload("cfg1"), 3), (synth.workload("cfg1", f_number=1.5), 4)):
        rf = _frames(wl, [2, 3])
        outs = []
        for rows in ("32", "16", "8"):
            monkeypatch.setenv("PA_LANE_ROWS", rows)
            out, info, _ = run_gpu(wl, rf, k)
            assert info["device_error_flags"] == 0
            outs.append(out)
        assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_lane_groups_with_tmem_sums(monkeypatch):
    """Compensated sums keep their Kahan totals in tensor memory, read and
    written warp-wide: without apodisation every lane grouping gives the same
    bits; with apodisation the plan keeps one slot per warp whatever
    PA_LANE_ROWS asks for, and the results match the oracle."""
    wl = synth.workload("cfg1")
    rf = _frames(wl, [4])
    outs = []
    for rows in ("32", "16", "8"):
        monkeypatch.setenv("PA_LANE_ROWS", rows)
        out, info, _ = run_gpu(wl, rf, 3, rf_dtype="bf16", compensated=1)
        assert info["device_error_flags"] == 0 and info["lane_rows"] == int(rows)
        outs.append(out)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    wl_a = synth.workload("cfg1", f_number=1.5)
    rf_a = _frames(wl_a, [5])
    monkeypatch.setenv("PA_LANE_ROWS", "8")
    out, info, deq = run_gpu(wl_a, rf_a, 4, rf_dtype="bf16", compensated=1)
    assert info["lane_rows"] == 32 and info["device_error_flags"] == 0
    assert_parity(compare(out, oracle_frames(wl_a, deq, 4)), TOL32, what="apodised, TMEM sums")


def test_tmem_residency_fits_the_sm():
    """Resident blocks per SM times the TMEM columns each block allocates
    stay within the SM's 512 columns (no block's allocation waits on another
    block of the same launch), for compensated plans of every order and the
    benchmark geometries; plain plans allocate none."""
    import paper_2203_14906_gb300 as pa

    for name, k in (("cfg1", 1), ("cfg1", 3), ("cfg2", 3), ("cfg2", 5), ("cfg2", 8), ("cfg3", 5),
                    ("cfg5", 4)):
        wl = synth.workload(name)
        for comp in (0, 1):
            with pa.Plan(pa.make_desc(wl, order_k=k, outputs=7, rf_dtype="bf16",
                                      compensated=comp)) as plan:
                info = plan.info()
            if comp:
                assert info["tmem_columns"] in (32, 64, 128, 256), (name, k)
                assert info["blocks_per_sm"] * info["tmem_columns"] <= 512, (name, k, info)
                assert info["blocks_per_sm"] >= 2 or k >= 6, (name, k, info)
            else:
                assert info["tmem_columns"] == 0


def test_long_columns_and_odd_width():
    """nz > 1024 (2048-point envelope transforms, the out-of-place FFT path),
    an odd number of columns (the last column pair has one column) and a
    lattice factor of 3."""
    wl = synth.workload("cfg1", n_elem=25, nx=75, nz=1500, n_samples=2048, z1_m=30e-3)
    wl["x0_m"], wl["x1_m"] = -25 * 0.15e-3, 25 * 0.15e-3
    rf = _frames(wl, [9])
    out, info, deq = run_gpu(wl, rf, 3)
    assert info["fft_size"] == 2048 and info["lattice_m"] == 3
    assert_parity(compare(out, oracle_frames(wl, deq, 3)), TOL32, what="nz=1500, nx=75")


def test_short_columns():
    """nz < 64: envelope transforms of 32 and 8 points (out-of-place path)."""
    for nz in (20, 7):
        wl = synth.workload("cfg1", nx=64, nz=nz, z1_m=nz * 0.4e-3)
        rf = _frames(wl, [6])
        out, info, deq = run_gpu(wl, rf, 4)
        assert_parity(compare(out, oracle_frames(wl, deq, 4)), TOL32, what=f"nz={nz}")


@pytest.mark.parametrize("k", [1, 3, 4])
def test_nearest_sample_delays(k):
    """Integer delays exactly as Eq. 1 writes them (no interpolation): cfg1
    batched, a ragged grid with short records and t0 > 0 (indices at both
    ends of the record), and cfg5-style apodisation with BF16 RF."""
    wl = synth.workload("cfg1", interp="nearest")
    rf = _frames(wl, [1, 2])
    out, info, deq = run_gpu(wl, rf, k)
    assert info["device_error_flags"] == 0
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"nearest cfg1 k={k}")
    wl = synth.workload("cfg1", interp="nearest", n_elem=37, n_samples=301, t0_s=1.5e-6,
                        nx=74, nz=77, z1_m=18e-3)
    wl["x0_m"], wl["x1_m"] = -37 * 0.15e-3, 37 * 0.15e-3
    rf = _frames(wl, [7])
    out, _, deq = run_gpu(wl, rf, k, max_batch=1)
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"nearest ragged k={k}")
    wl = synth.workload("cfg5", interp="nearest", nx=256, nz=256)
    rf = _frames(wl, [41])
    out, info, deq = run_gpu(wl, rf, k, rf_dtype="bf16", compensated=1)
    assert info["tma_staging"] == 1
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"nearest apod k={k}")


def test_nearest_full_size_cfg2():
    wl = synth.workload("cfg2", interp="nearest")
    rf = _frames(wl, wl["seeds"][:2])
    out, _, deq = run_gpu(wl, rf, 3)
    assert_parity(compare(out, oracle_frames(wl, deq, 3)), TOL32, what="nearest cfg2")


def test_chunk_length_does_not_change_bits(monkeypatch):
    """The channel steps staged per shared-memory chunk (plan policy, or the
    PA_CHUNK_STEPS override) change only the staging schedule: every pixel
    still sums its channels in the same order, so the images are identical.
    FP32 loads staging and BF16 TMA staging, with and without apodisation."""
    wl = synth.workload("cfg1", n_elem=128, nx=256, nz=96, z1_m=12e-3)
    wl["x0_m"], wl["x1_m"] = -128 * 0.15e-3, 128 * 0.15e-3
    rf = _frames(wl, [3, 4])
    wa = synth.workload("cfg5", nx=256, nz=128)
    ra = _frames(wa, [41])
    for w, r, k, dt, comp in ((wl, rf, 3, "f32", 0), (wl, rf, 5, "bf16", 1), (wa, ra, 4, "bf16", 1)):
        monkeypatch.delenv("PA_CHUNK_STEPS", raising=False)
        ref, info, _ = run_gpu(w, r, k, rf_dtype=dt, compensated=comp)
        assert info["chunk_steps"] % 4 == 0 and info["chunk_steps"] <= 64
        for steps in ("4", "32", "64"):
            monkeypatch.setenv("PA_CHUNK_STEPS", steps)
            out, info2, _ = run_gpu(w, r, k, rf_dtype=dt, compensated=comp)
            assert info2["chunk_steps"] <= int(steps)
            assert info2["device_error_flags"] == 0
            assert np.array_equal(out, ref), (w["name"], k, dt, steps)


def test_off_centre_window():
    """An image window narrower than the aperture, off its centre and
    starting below the surface (x in [-4.5, 7.5] mm, z in [6, 18] mm):
    lattice offsets of both signs at the window edges, k = 3 and 4."""
    wl = synth.workload("cfg1", nx=80, nz=96, x0_m=-4.5e-3, x1_m=7.5e-3, z0_m=6e-3, z1_m=18e-3)
    rf = _frames(wl, [3])
    for k in (3, 4):
        out, info, deq = run_gpu(wl, rf, k)
        assert info["lattice_m"] == 2 and info["device_error_flags"] == 0
        assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"window k={k}")


def test_graph_cache_beyond_its_bound():
    """Forty different batch sizes on one plan (the plan keeps at most 32
    launch graphs, dropping the oldest): every call still gives the bits of a
    direct launch."""
    import torch

    import paper_2203_14906_gb300 as pa

    wl = synth.workload("cfg1", nx=64, nz=32, z1_m=10e-3)
    rf = torch.from_numpy(synth.quantize(_frames(wl, list(range(40))), "f32")[0]).cuda()
    with pa.Plan(pa.make_desc(wl, order_k=3, max_batch=40)) as plan:
        plan.use_graph(False)
        ref = pa.beamform(plan, rf, 7)
        plan.use_graph(True)
        for n in list(range(1, 41)) + [3, 17, 40]:
            out = pa.beamform(plan, rf[:n].contiguous(), 7)
            assert torch.equal(out, ref[:n]), n


@pytest.mark.parametrize("b", [45, 77, 6])
def test_tone_through_the_gpu_post_filter(b):
    """The pinned one-element tone: an RF tone of known temporal frequency
    lands on its depth bin and the GPU band-pass keeps or removes it as the
    oracle does (in band: envelope 1; out of band: 0)."""
    from test_oracle_post import _post_gold, tone_case

    case = {c["b"]: c for c in _post_gold()["tone"]["cases"]}[b]
    wl, rf = tone_case(b)
    out, info, deq = run_gpu(wl, rf[None], 1, outputs=1, stages=3)
    assert info["device_error_flags"] == 0
    # the envelope is 1 or 0 (a blocked tone has no peak to normalise by,
    # so it is checked in absolute terms against the unit tone amplitude)
    env = out[0, 1, 0, 0]
    ref = oracle_frames(wl, deq, 1, stages=("raw", "env"))[0]
    assert np.allclose(env, case["odd_env"], rtol=0, atol=1e-4)
    assert np.max(np.abs(env - ref["env"]["das"][0])) <= TOL32
    assert_parity(compare(out[:, :1], [ref], outputs=1, stages=1), TOL32, what=f"tone bin {b}")


# ---- full per-pixel delay table (grids off the lattice) --------------------

def _random_off_lattice(rng):
    """A lateral pixel pitch drawn from a continuous range (0.05-0.8 mm, so
    pitch / dx between 0.375 and 6, almost never an integer): finer and
    coarser grids than the element pitch."""
    n_elem = int(rng.integers(8, 72))
    dx = float(rng.uniform(0.05e-3, 0.8e-3))
    nx = int(rng.integers(5, 110))
    nz = int(rng.integers(17, 160))
    dz = float(rng.uniform(40e-6, 110e-6))
    x0 = -nx * dx / 2 + float(rng.uniform(-1.0, 1.0)) * 2e-3
    z0 = float(rng.uniform(0.0, 4e-3))
    wl = synth.workload(
        "cfg1", n_elem=n_elem, nx=nx, nz=nz, x0_m=x0, x1_m=x0 + nx * dx, z0_m=z0,
        z1_m=z0 + nz * dz, n_samples=int(rng.integers(300, 1400)),
        t0_s=float(rng.choice([0.0, 0.5e-6])), n_points=3,
        f_number=float(rng.choice([0.0, 0.0, 1.5])),
        interp=str(rng.choice(["linear", "linear", "nearest"])))
    wl["seeds"] = [int(rng.integers(1, 1000))]
    return wl


@pytest.mark.parametrize("case", range(16))
def test_random_off_lattice_geometries(case):
    """Seeded random grids whose lateral pitch is not the element pitch over
    an integer: the plan takes the full table (one entry per pixel and
    element), every RF type, orders 1-8, apodisation and nearest-sample
    delays; every stage against the oracle at the FP32 tolerance."""
    rng = np.random.default_rng(5000 + case)
    wl = _random_off_lattice(rng)
    k = int(rng.integers(1, 9))
    k = min(k, wl["n_elem"])
    dtype = str(rng.choice(["f32", "bf16", "f16"]))
    rf = _frames(wl, [wl["seeds"][0], wl["seeds"][0] + 1])
    out, info, deq = run_gpu(wl, rf, k, rf_dtype=dtype, compensated=int(dtype != "f32"),
                             max_batch=int(rng.integers(1, 3)))
    assert info["device_error_flags"] == 0
    assert info["delay_table"] == 2 and info["lattice_m"] == 0
    what = (f"case {case}: N={wl['n_elem']} pitch/dx={0.3e-3 * wl['nx'] / (wl['x1_m'] - wl['x0_m']):.4f} "
            f"grid={wl['nx']}x{wl['nz']} Ns={wl['n_samples']} k={k} {dtype} "
            f"F#={wl['f_number']} {wl['interp']}")
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=what)


@pytest.mark.parametrize("k", [3, 5])
def test_off_lattice_full_size_cfg2_400_columns(k):
    """cfg2 (128 el x 2048 samples, 40 mm deep, 512 rows) on a 400-column
    grid over the same 38.4 mm: pitch / dx = 3.125, full table, 1e-4 gate."""
    wl = synth.workload("cfg2", nx=400)
    rf = _frames(wl, wl["seeds"])
    out, info, deq = run_gpu(wl, rf, k)
    assert info["delay_table"] == 2 and info["device_error_flags"] == 0
    assert_parity(compare(out, oracle_frames(wl, deq, k)), TOL32, what=f"cfg2 nx=400 k={k}")


@pytest.mark.parametrize("kind", ["fp32", "bf16_apod"])
def test_full_table_equals_lattice_table(kind):
    """On a lattice grid both table forms hold the same FP64 delays: the
    lattice entry keeps the fraction a rounded to FP32, the full entry
    truncated to 23 bits (within 1.2e-7 of each other), and compensated sums
    fold their FP32 partial sums at channels that depend on a column's place
    within its thread, which differs between the forms.  The images agree to
    1e-5 of their peaks, far inside the 1e-4 gate each meets against the
    oracle."""
    if kind == "fp32":
        wl, k, dt, comp = synth.workload("cfg1"), 3, "f32", 0
    else:
        wl, k, dt, comp = synth.workload("cfg5", nx=256, nz=256), 4, "bf16", 1
    rf = _frames(wl, [3, 4])
    outs = {}
    for form in ("lattice", "full"):
        out, info, deq = run_gpu(dict(wl, delay_table=form), rf, k, rf_dtype=dt, compensated=comp)
        assert info["delay_table"] == (1 if form == "lattice" else 2)
        assert info["device_error_flags"] == 0
        outs[form] = out
    a, b = outs["lattice"], outs["full"]
    peak = np.max(np.abs(a), axis=(-2, -1), keepdims=True)
    assert np.max(np.abs(a - b) / np.maximum(peak, 1e-30)) <= 1e-5
    assert_parity(compare(b, oracle_frames(wl, deq, k)), TOL32, what=f"full table {kind}")


def test_full_table_checked_build():
    """Bounds-checked build over full-table geometries (coarse, fine,
    apodised): no table row or shared address leaves its range."""
    cases = [
        (synth.workload("cfg1", nx=32, x0_m=-9.6e-3, x1_m=9.6e-3), 3, "f32", 0),  # dx = 2 pitch
        (synth.workload("cfg1", nx=100), 5, "f32", 0),  # pitch / dx = 1.5625
        (synth.workload("cfg5", nx=300, nz=256), 4, "bf16", 1),  # apodised, 3.906
    ]
    for wl, k, dt, comp in cases:
        rf = synth.make_frame(wl, 1)[None]
        _, info, _ = run_gpu(wl, rf, k, rf_dtype=dt, compensated=comp, checked=True)
        assert info["device_error_flags"] == 0 and info["delay_table"] == 2, (wl["nx"], k)


@pytest.mark.parametrize("lanes", [4, 8, 32])
def test_channel_lanes_mapping_matches_fused(lanes):
    """The channels-on-lanes mapping (kept for measurement) computes the
    same RAW images as the fused kernel, to FP32 rounding (its channel sums
    are added in another order)."""
    import ctypes

    import torch

    import paper_2203_14906_gb300 as pa
    from paper_2203_14906_gb300 import _native

    for name in ("cfg1", "cfg2"):
        wl = synth.workload(name)
        F = 2
        rf = torch.from_numpy(synth.quantize(_frames(wl, [3, 4]), "f32")[0]).cuda()
        with pa.Plan(pa.make_desc(wl, order_k=3, max_batch=F)) as plan:
            want = pa.beamform(plan, rf, 1)
            got = torch.full_like(want, 7.0)
            L = _native.load()
            st = L.pa_lanes_raw(plan._h, rf.data_ptr(), F, got.data_ptr(), lanes,
                                torch.cuda.current_stream().cuda_stream)
            assert st == 0, L.pa_last_error()
            torch.cuda.synchronize()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        peak = np.max(np.abs(w), axis=(-2, -1), keepdims=True)
        assert np.max(np.abs(w - g) / peak) <= 1e-5, (name, lanes)
