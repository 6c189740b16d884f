"""Allocation-free log compression (pa_log_compress_noalloc) against the
plan-based path's own LOG stage.

Some callers cannot allocate device memory once they are streaming, for
example a scanner's real-time loop that must not let cudaMalloc stall the
device, or a host framework that owns every device buffer.  For them the
library offers a log-compression call whose only scratch (the per-image
maxima) is a fixed device array inside the library.  This file runs last:
it calls that entry point through the C ABI twice in a row and checks each
result against pa_beamform's LOG planes for the same envelopes and against
the FP64 oracle's log compression of those envelopes.  The second call uses
a frame scaled down 4x, so maxima left over from the first call would shift
every pixel by 12 dB and fail the check.  A third call runs in place
(output buffer = input buffer) and must give the same bits.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_DB = 0.05  # the log-stage tolerance of the parity tests


def test_noalloc_log_matches_plan_log_two_calls():
    import torch

    import paper_2203_14906_gb300 as pa
    from paper_2203_14906_gb300 import _native

    L = _native.load()
    wl = synth.workload("cfg1")
    stages = pa.PA_STAGE_ENV | pa.PA_STAGE_LOG
    n_img, elems = 3, wl["nx"] * wl["nz"]
    for call, scale in enumerate((1.0, 0.25)):
        rf64 = synth.make_frame(wl, 1 + call) * scale
        rf = torch.from_numpy(synth.quantize(rf64, "f32")[0][None]).cuda()
        with pa.Plan(pa.make_desc(wl, order_k=3, outputs=7)) as plan:
            out = pa.beamform(plan, rf, stages)
        env = out[0, 0].contiguous()
        want = out[0, 1]
        got = torch.full_like(env, 123.0)
        stream = torch.cuda.current_stream()
        st = L.pa_log_compress_noalloc(env.data_ptr(), n_img, elems, 60.0, got.data_ptr(),
                                       stream.cuda_stream)
        assert st == _native.PA_OK, L.pa_last_error()
        torch.cuda.synchronize()
        diff = float((got - want).abs().max().item())
        assert diff <= TOL_DB, f"call {call}: max |dB| difference {diff}"
        assert torch.equal(got, want), "same log function, same bits"
        assert float(got.max().item()) == 0.0 and float(got.min().item()) >= -60.0
        env_h = env.cpu().numpy().astype(np.float64)
        got_h = got.cpu().numpy()
        for i in range(n_img):
            ref = oracle.log_image(env_h[i], 60.0)
            d_or = float(np.max(np.abs(got_h[i] - ref)))
            assert d_or <= TOL_DB, f"call {call} image {i}: max |dB| vs oracle {d_or}"
        # in place: the output overwrites the envelopes it is computed from
        inplace = env.clone()
        st = L.pa_log_compress_noalloc(inplace.data_ptr(), n_img, elems, 60.0,
                                       inplace.data_ptr(), stream.cuda_stream)
        assert st == _native.PA_OK, L.pa_last_error()
        torch.cuda.synchronize()
        assert torch.equal(inplace, got), f"call {call}: in-place result differs"


def test_noalloc_rejects_more_images_than_the_scratch_holds():
    from paper_2203_14906_gb300 import _native

    L = _native.load()
    st = L.pa_log_compress_noalloc(None, 4097, 16, 60.0, None, None)
    assert st == _native.PA_EINVAL
    assert b"PA_NOALLOC_MAX_IMAGES" in L.pa_last_error()
