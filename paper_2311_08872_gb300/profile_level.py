"""Time one level's batch of coupled samples on the GPU (CUDA events on the
launching stream) -- the small, repeatable command used for kernel profiles.

    python -m paper_2311_08872_gb300.profile_level --workload mlmc16_256 --level 4 --samples 19

Prints one JSON line: samples, device ms per launch, cell-steps/s.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="mlmc16_256")
    ap.add_argument("--level", type=int, default=4)
    ap.add_argument("--samples", type=int, default=19)
    ap.add_argument("--mc", action="store_true", help="plain MC stream (fine path only)")
    ap.add_argument("--repeat", type=int, default=2, help="timed launches after one warm-up launch")
    ap.add_argument("--T", type=float, default=None, help="override the final time (fewer steps per sample)")
    args = ap.parse_args()

    import torch

    from paper_2311_08872_gb300 import build, mlmc_dk, workloads

    build.build()
    wl = workloads.get(args.workload)
    if args.T is not None:
        wl = wl.with_(T=args.T)
    st = torch.cuda.current_stream()
    with mlmc_dk.Context.from_workload(wl, stream=st.cuda_stream) as ctx:
        info = ctx.level_info(args.level)
        tag = 1 if args.mc else 0
        cost = info.cost_mc if (args.mc or args.level == 0) else info.cost
        sums = torch.zeros(mlmc_dk.sums_len(ctx.n_quant), dtype=torch.float64, device="cuda")
        ctx.run_level_dev(args.level, tag, 0, args.samples, wl.seed, sums.data_ptr(), 0, st.cuda_stream)
        ms = []
        for r in range(args.repeat):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.run_level_dev(args.level, tag, 0, args.samples, wl.seed + 1 + r, sums.data_ptr(), 0, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    avg = sum(ms) / len(ms)
    print(json.dumps({"workload": wl.name, "level": args.level, "n": info.n, "fine_steps": info.M,
                      "streamed": bool(info.streamed), "coupled": tag == 0 and args.level > 0,
                      "theta_b0": info.theta_b0 if info.theta else 0.0, "cheb_steps": info.cheb_steps,
                      "samples": args.samples, "ms_per_launch": avg,
                      "cell_steps_per_s": args.samples * cost / (avg * 1e-3)}))


if __name__ == "__main__":
    main()
