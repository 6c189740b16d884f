"""Failure detection on the GPU without faulting it.

The fused kernel's TMA staging waits are bounded (about a second of SM
clock).  In the checked build (the only one that reads it),
PA_INJECT_TMA_SHORTFALL makes every chunk expect 16 bytes more than its
copies deliver, so the barrier never completes: each block's wait runs out,
the block sets error flag 8, counts a timeout and returns.  In this injected
case every copy has landed (only the expected byte count is short), so none
is left in flight.  The host path reports PA_ETIMEOUT, the server completes
the request with PA_ETIMEOUT, and plans built afterwards work normally.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _small():
    wl = synth.workload("cfg1", nx=64, nz=64, z1_m=10e-3)
    store, _ = synth.quantize(synth.make_frame(wl, 1)[None], "bf16")
    return wl, store


def test_bounded_wait_reports_timeout_on_the_host_path(monkeypatch):
    import paper_2203_14906_gb300 as pa
    from paper_2203_14906_gb300._native import PA_ETIMEOUT, PAError

    wl, store = _small()
    monkeypatch.setenv("PA_INJECT_TMA_SHORTFALL", "1")
    with pa.Plan(pa.make_desc(wl, order_k=3, rf_dtype="bf16", compensated=1), checked=True) as plan:
        assert plan.info()["tma_staging"] == 1
        with pytest.raises(PAError) as e:
            pa.beamform_host(plan, store.view(np.uint16), pa.PA_STAGE_LOG)
        assert e.value.status == PA_ETIMEOUT
        assert plan.info()["device_error_flags"] & 8
    monkeypatch.delenv("PA_INJECT_TMA_SHORTFALL")
    with pa.Plan(pa.make_desc(wl, order_k=3, rf_dtype="bf16", compensated=1), checked=True) as plan:
        out = pa.beamform_host(plan, store.view(np.uint16), pa.PA_STAGE_LOG)
        assert plan.info()["device_error_flags"] == 0
    assert np.isfinite(out).all() and out.max() == 0.0


def test_server_completes_a_timed_out_batch_with_etimeout(monkeypatch):
    import torch

    import paper_2203_14906_gb300 as pa
    from paper_2203_14906_gb300._native import PA_ETIMEOUT
    from paper_2203_14906_gb300.serving import Server

    wl, store = _small()
    rf = torch.from_numpy(store[0].view(np.int16)).pin_memory()
    out = torch.zeros((1, 3, 64, 64), dtype=torch.float32).pin_memory()
    desc = pa.make_desc(wl, order_k=3, rf_dtype="bf16", compensated=1)
    monkeypatch.setenv("PA_INJECT_TMA_SHORTFALL", "1")
    with Server(budget_bytes=1 << 30, slots=2, max_batch=2, checked=True) as srv:
        r = srv.wait(srv.submit(desc, rf.data_ptr(), out.data_ptr()), timeout_ms=60000)
        st = srv.stats()
    assert r["status"] == PA_ETIMEOUT
    assert st["failed"] == 1 and st["completed"] == 0
    monkeypatch.delenv("PA_INJECT_TMA_SHORTFALL")
    with Server(budget_bytes=1 << 30, slots=2, max_batch=2, checked=True) as srv:
        r = srv.wait(srv.submit(desc, rf.data_ptr(), out.data_ptr()), timeout_ms=60000)
    assert r["status"] == 0 and out.max() == 0.0


def test_release_build_ignores_the_injection(monkeypatch):
    """The release library never reads PA_INJECT_TMA_SHORTFALL."""
    import paper_2203_14906_gb300 as pa

    wl, store = _small()
    monkeypatch.setenv("PA_INJECT_TMA_SHORTFALL", "1")
    with pa.Plan(pa.make_desc(wl, order_k=3, rf_dtype="bf16", compensated=1)) as plan:
        out = pa.beamform_host(plan, store.view(np.uint16), pa.PA_STAGE_LOG)
        assert plan.info()["device_error_flags"] == 0
    assert np.isfinite(out).all() and out.max() == 0.0
