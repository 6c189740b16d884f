"""Host logic of bench.py's precision report (CPU): the per-image error
measures against the FP64 oracle, checked on oracle images with errors of
known size planted in them."""

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
