"""Host logic of bench.py (CPU): the precision report's per-image error
measures against the FP64 oracle, checked on oracle images with errors of
known size planted in them; and the roofline accounting - the committed
DRAM-traffic record is used only for the kernel source and launch shape it
was taken on, and the per-pair operation model."""

import numpy as np

import bench
import oracle
import synth


def _oracle_as_gpu_output(wl, k):
    rf = synth.make_frame(wl, 1)
    ref = oracle.frame(wl, rf, order_k=k)
    out = np.stack([np.stack([ref[st][o] for o in oracle.OUTPUT_ORDER])
                    for st in ("raw", "env", "log")])
    return out, ref


def test_errors_of_the_oracle_against_itself_are_zero():
    wl = synth.workload("cfg1", nx=32, nz=48, z1_m=10e-3)
    out, ref = _oracle_as_gpu_output(wl, 3)
    rep = bench._errors(out, ref)
    assert set(rep) == set(oracle.OUTPUT_ORDER)
    for d in rep.values():
        assert all(v == 0.0 for v in d.values()), d


def test_planted_errors_are_reported_at_their_size():
    """A raw pixel off by 1e-3 of the peak, an envelope pixel off by 2e-3 of
    the peak and a main-lobe log pixel off by 0.04 dB are each reported as
    that error; a -40 dB pixel off by 1 dB counts only in the image mean."""
    wl = synth.workload("cfg1", nx=32, nz=48, z1_m=10e-3)
    out, ref = _oracle_as_gpu_output(wl, 3)
    o = 2  # DMAS-3
    name = oracle.OUTPUT_ORDER[o]
    raw, env, lg = ref["raw"][name], ref["env"][name], ref["log"][name]
    out[0, o].flat[5] += 1e-3 * np.max(np.abs(raw))
    out[1, o].flat[7] += 2e-3 * np.max(np.abs(env))
    top = int(np.argmax(lg))
    out[2, o].flat[top] += 0.04
    low = np.flatnonzero(lg < -20.0)[0]
    out[2, o].flat[low] += 1.0
    rep = bench._errors(out, ref)[name]
    assert abs(rep["raw_max_err_of_peak"] - 1e-3) < 1e-9
    assert abs(rep["env_max_err_of_peak"] - 2e-3) < 1e-9
    assert abs(rep["log_max_abs_db_top6db"] - 0.04) < 1e-9
    assert abs(rep["log_mean_abs_db"] - (1.04 / lg.size)) < 1e-9
    others = [bench._errors(out, ref)[n] for n in oracle.OUTPUT_ORDER if n != name]
    assert all(v == 0.0 for d in others for v in d.values())


def test_headline_form_switch():
    class A:
        form = "fp32"

    assert bench.form_dtype(A) == ("f32", 0)
    A.form = "precision"
    assert bench.form_dtype(A) == ("bf16", 1)


# ---- roofline accounting: the DRAM-traffic record and the per-pair model


def _fake_sources(tmp_path, body):
    csrc = tmp_path / "csrc"
    csrc.mkdir(exist_ok=True)
    (csrc / "pa_bf_kernel.cuh").write_text(body)
    (csrc / "pa_internal.cuh").write_text("int x;\n")
    (csrc / "pa_post.cu").write_text("not hashed\n")
    return str(csrc)


def test_kernel_hash_ignores_comments_and_spacing_only(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "CSRC", _fake_sources(tmp_path, "int f() { return 1; } // one\n"))
    h0 = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "CSRC", _fake_sources(tmp_path, "/* a\nb */ int  f()\n{ return 1; }\n"))
    assert bench.kernel_source_hash() == h0
    monkeypatch.setattr(bench, "CSRC", _fake_sources(tmp_path, "int f() { return 2; }\n"))
    assert bench.kernel_source_hash() != h0
    (tmp_path / "csrc" / "pa_post.cu").write_text("changed, still not hashed\n")
    h1 = bench.kernel_source_hash()
    (tmp_path / "csrc" / "pa_post.cu").write_text("changed again\n")
    assert bench.kernel_source_hash() == h1


def test_traffic_record_is_used_only_for_the_kernel_and_launch_it_was_taken_on(tmp_path,
                                                                             monkeypatch):
    import json

    monkeypatch.setattr(bench, "CSRC", _fake_sources(tmp_path, "int f() { return 1; }\n"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    launch = {f: i + 1 for i, f in enumerate(bench.LAUNCH_FIELDS)}
    assert bench.measured_traffic("dram_bytes_per_launch", launch) is None  # no record
    (tmp_path / "profiles").mkdir()
    rec = {"kernel_hash": bench.kernel_source_hash(), "launch": dict(launch),
           "dram_bytes_per_launch": 1234}
    (tmp_path / "profiles" / "bf_fused_traffic.json").write_text(json.dumps(rec))
    assert bench.measured_traffic("dram_bytes_per_launch", launch) == 1234
    other = dict(launch, chunk_steps=launch["chunk_steps"] + 1)
    assert bench.measured_traffic("dram_bytes_per_launch", other) is None
    rec["kernel_hash"] = "0" * 16
    (tmp_path / "profiles" / "bf_fused_traffic.json").write_text(json.dumps(rec))
    assert bench.measured_traffic("dram_bytes_per_launch", launch) is None


def test_operations_per_pair_model():
    """2k + 7 for the combined DAS + DMAS + DMAS-k pass (13 at k = 3, 17 at
    k = 5, as Table 1's per-channel counts add up); k <= 2 reuse the DMAS
    sums."""
    assert [bench.ops_per_pair(k) for k in (1, 2, 3, 4, 5, 8)] == [7, 9, 13, 15, 17, 23]
