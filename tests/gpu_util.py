"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and compare it with the FP64 oracle on the same seeded inputs."""

from __future__ import annotations

import numpy as np

import oracle
import synth

STAGES_ALL = 7
OUTPUTS_ALL = 7


def run_gpu(wl, rf64, order_k, rf_dtype="f32", compensated=0, outputs=OUTPUTS_ALL,
            stages=STAGES_ALL, max_batch=None, checked=False, host=False):
    """rf64: [F][N][Ns] float64.  Returns (out [F][S][O][nx][nz], info, deq64)."""
    import torch

    import paper_2203_14906_gb300 as pa

    rf64 = np.asarray(rf64)
    if rf64.ndim == 2:
        rf64 = rf64[None]
    store, deq = synth.quantize(rf64, rf_dtype)
    F = rf64.shape[0]
    desc = pa.make_desc(wl, order_k=order_k, outputs=outputs, rf_dtype=rf_dtype,
                        max_batch=max_batch or F, compensated=compensated)
    plan = pa.Plan(desc, checked=checked)
    try:
        if host:
            out = pa.beamform_host(plan, store, stages)
        else:
            if rf_dtype == "bf16":
                t = torch.from_numpy(store.view(np.int16)).cuda().view(torch.bfloat16)
            else:
                t = torch.from_numpy(store).cuda()
            o = pa.beamform(plan, t, stages)
            torch.cuda.synchronize()
            out = o.cpu().numpy()
        info = plan.info()
    finally:
        plan.close()
    return out, info, deq


def oracle_frames(wl, rf64, order_k, stages=("raw", "env", "log")):
    rf64 = np.asarray(rf64)
    if rf64.ndim == 2:
        rf64 = rf64[None]
    return [oracle.frame(wl, rf64[f], order_k=order_k, stages=stages) for f in range(rf64.shape[0])]


def compare(out, refs, outputs=OUTPUTS_ALL, stages=STAGES_ALL, outs_order=oracle.OUTPUT_ORDER):
    """Per (frame, stage, output): RAW/ENV max|d|/max|ref|; LOG max |dB|
    over pixels within 6 dB of the peak, plus the mean |dB| over the image."""
    st_names = [s for b, s in ((1, "raw"), (2, "env"), (4, "log")) if stages & b]
    o_names = [o for b, o in zip((1, 2, 4), outs_order) if outputs & b]
    res = {}
    for f, ref in enumerate(refs):
        for si, st in enumerate(st_names):
            for oi, o in enumerate(o_names):
                g = out[f, si, oi]
                r = ref[st][o]
                if st == "log":
                    sel = r >= -6.0
                    res[(f, st, o)] = (
                        float(np.max(np.abs(g[sel] - r[sel]))) if sel.any() else 0.0,
                        float(np.mean(np.abs(g - r))),
                    )
                else:
                    peak = float(np.max(np.abs(r)))
                    res[(f, st, o)] = float(np.max(np.abs(g - r)) / peak) if peak > 0 else float(np.max(np.abs(g)))
    return res


def assert_parity(res, tol_rel, tol_db=0.05, what=""):
    bad = []
    for key, v in res.items():
        if key[1] == "log":
            if v[0] > tol_db:
                bad.append((key, v))
        elif v > tol_rel:
            bad.append((key, v))
    assert not bad, f"{what} parity failures: {bad[:8]}"
