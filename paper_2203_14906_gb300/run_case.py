"""Run one workload's launch sequence a few times and print its kernel times.

For profiling a single configuration (under ncu, or with CUDA-event timing
alone), e.g.

    python -m paper_2203_14906_gb300.run_case --workload cfg5 --frames 4

Inputs are seeded random RF of the workload's shape (the arithmetic does not
depend on the values); the timed launches are preceded by warm-up launches
and each is preceded by a 256 MiB write that flushes the L2.
"""

from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="cfg2", choices=["cfg1", "cfg2", "cfg3", "cfg5"])
    ap.add_argument("--frames", type=int, default=None, help="frames per launch (default: the workload's)")
    ap.add_argument("--order", type=int, default=None, help="order k (default: the workload's)")
    ap.add_argument("--rf", default=None, choices=["f32", "bf16", "f16"])
    ap.add_argument("--compensated", type=int, default=None, choices=[0, 1])
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--launches", type=int, default=3)
    args = ap.parse_args(argv)

    import torch

    import synth
    import paper_2203_14906_gb300 as pa

    wl = synth.workload(args.workload)
    F = args.frames or int(wl.get("n_frames", 1))
    k = args.order or int(wl.get("order_k", 3))
    rf_dtype = args.rf or wl.get("rf_dtype", "f32")
    comp = args.compensated if args.compensated is not None else int(wl.get("compensated", 0))
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    x = torch.randn(F, wl["n_elem"], wl["n_samples"], device=dev, generator=g)
    rf = x.to({"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[rf_dtype])
    desc = pa.make_desc(wl, order_k=k, outputs=7, rf_dtype=rf_dtype, max_batch=F, compensated=comp)
    with pa.Plan(desc, stream=stream) as plan, torch.cuda.stream(stream):
        out = torch.empty(plan.out_shape(F, pa.PA_STAGE_LOG), dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            flush.zero_()
            pa.beamform(plan, rf, pa.PA_STAGE_LOG, out=out, stream=stream)
        stream.synchronize()
        plan.profile_read()
        plan.profile(True)
        for _ in range(args.launches):
            flush.zero_()
            pa.beamform(plan, rf, pa.PA_STAGE_LOG, out=out, stream=stream)
        stream.synchronize()
        prof = plan.profile_read()
        plan.profile(False)
        info = plan.info()
    print(json.dumps({
        "workload": args.workload, "frames": F, "order_k": k, "rf": rf_dtype, "compensated": comp,
        "kernels_ms_per_launch": {kk: v[0] / max(v[1], 1) for kk, v in prof.items()},
        "blocks_per_sm": info["blocks_per_sm"], "chunk_steps": info["chunk_steps"],
        "lane_rows": info["lane_rows"], "tmem_columns": info["tmem_columns"],
        "nominal_pairs": info["nominal_pairs"] * F, "active_pairs": info["active_pairs"] * F,
        "device_error_flags": info["device_error_flags"],
    }))
    return 0


if __name__ == "__main__":
    sys.exit(main())
