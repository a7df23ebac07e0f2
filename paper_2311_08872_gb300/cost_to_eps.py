"""Pilot-based MLMC and plain-MC cost to an RMSE eps on the GPU path.

    python -m paper_2311_08872_gb300.cost_to_eps --workload lowdens32_512

For every level: a pilot batch of coupled samples (sized to about
--seconds of device time) gives V_l = Var[P_l - P_(l-1)], E_l and the device
time per sample t_l; a plain-MC pilot on the finest level gives Var[P_L] and
its time per sample.  With eps = eps_rel |sum_l E_l| (relative to the largest
diagonal quantity when there are several), the eps-optimal allocation of
Eq. (opt_M_ell), M_l = ceil(2 eps^-2 sqrt(V_l / t_l) sum_k sqrt(V_k t_k)),
taken as the maximum over quantities, costs sum_l M_l t_l; plain MC needs
ceil(2 Var[P_L] / eps^2) finest-level samples (the extrapolation the paper
uses for its MC times, Section 7.3).  With --surrogate the learned level
below 0 is trained (2^18 level-0 paths, 8 epochs) and level 0 is replaced by
the pair {level below 0, correction level}, each with its own pilot variance
and device time per sample.  All figures are extrapolated from measured
rates and pilot variances, and printed as one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _moments(s):
    n = s.n
    e = s.dp1 / n
    v = max(0.0, (s.dp2 - s.dp1 ** 2 / n) / (n - 1))
    vf = max(0.0, (s.pf2 - s.pf1 ** 2 / n) / (n - 1))
    return e, v, s.pf1 / n, vf


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lowdens32_512")
    ap.add_argument("--eps-rel", type=float, default=None, help="default: the workload's")
    ap.add_argument("--seconds", type=float, default=1.5, help="device time per pilot batch")
    ap.add_argument("--max-pilot", type=int, default=100000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--surrogate", action="store_true", help="also the cost with the learned level below 0")
    ap.add_argument("--L-max", type=int, default=None, help="finest level (default: the workload's)")
    ap.add_argument("--N", type=float, default=None, help="particle number (default: the workload's)")
    args = ap.parse_args()

    import torch

    from paper_2311_08872_gb300 import build, mlmc_dk, workloads

    build.build()
    wl = workloads.get(args.workload)
    if args.L_max is not None:
        wl = wl.with_(L_max=args.L_max)
    if args.N is not None:
        wl = wl.with_(N=args.N)
    eps_rel = args.eps_rel if args.eps_rel is not None else (wl.eps_rel or 1e-2)
    st = torch.cuda.current_stream()
    rows = []
    with mlmc_dk.Context.from_workload(wl, stream=st.cuda_stream) as ctx:
        ctx.tune(1)
        nq = ctx.n_quant
        rate = 2.4e11       # first guess of cell-steps/s to size the pilots
        for l in range(wl.L_max + 1):
            info = ctx.level_info(l)
            # a few samples to measure the rate, then a pilot of about --seconds
            probe = max(2, info.in_flight or 0)
            n = int(min(args.max_pilot, max(probe, args.seconds * rate / info.cost)))
            sums = ctx.run_level(l, n, args.seed)
            t = sums[0].kernel_s / n
            rate = info.cost / t
            q = [_moments(sums[k]) for k in range(nq)]
            rows.append({"level": l, "n": info.n, "fine_steps": info.M, "pilot": n, "s_per_sample": t,
                         "cell_steps_per_s": info.cost / t, "E": [x[0] for x in q], "V": [x[1] for x in q],
                         "EPf": [x[2] for x in q], "VPf": [x[3] for x in q]})
        sur = None
        if args.surrogate:
            ctx.surrogate_init(args.seed + 3)
            tr = ctx.surrogate_train(1 << 18, epochs=8, batch=1024, lr=1e-3, seed=args.seed + 4)
            sur = {"train_s": tr["seconds"], "val_mse": tr["val_mse"], "parts": []}
            for part in (-1, 0):
                n = 200000
                sm = ctx.run_surrogate(part, n, args.seed + 7 + part)
                t = sm[0].kernel_s / n
                q = [_moments(sm[k]) for k in range(nq)]
                sur["parts"].append({"part": part, "pilot": n, "s_per_sample": t, "E": [x[0] for x in q],
                                     "V": [x[1] for x in q]})
        L = wl.L_max
        info = ctx.level_info(L)
        n_mc = max(2, int(min(args.max_pilot, args.seconds * rows[-1]["cell_steps_per_s"] / info.cost_mc)))
        mc = ctx.run_level(L, n_mc, args.seed + 1, mc=True)
        t_mc = mc[0].kernel_s / n_mc
        var_pl = [_moments(mc[k])[3] for k in range(nq)]
    # relative eps against the largest diagonal quantity's estimate
    est = [sum(r["E"][k] for r in rows) for k in range(nq)]
    eps = eps_rel * max(abs(x) for x in est)
    M = [0] * len(rows)
    for k in range(nq):
        s = sum(math.sqrt(r["V"][k] * r["s_per_sample"]) for r in rows)
        for l, r in enumerate(rows):
            m = math.ceil(2.0 / eps ** 2 * math.sqrt(r["V"][k] / r["s_per_sample"]) * s) if r["V"][k] > 0 else 0
            M[l] = max(M[l], m)
    t_mlmc = sum(m * r["s_per_sample"] for m, r in zip(M, rows))
    m_mc = max(math.ceil(2.0 * v / eps ** 2) for v in var_pl)
    if sur is not None:
        # levels {below 0, correction, 1..L} in place of {0, 1..L}
        vl = sur["parts"] + rows[1:]
        Ms = [0] * len(vl)
        for k in range(nq):
            s = sum(math.sqrt(r["V"][k] * r["s_per_sample"]) for r in vl)
            for i, r in enumerate(vl):
                m = math.ceil(2.0 / eps ** 2 * math.sqrt(r["V"][k] / r["s_per_sample"]) * s) if r["V"][k] > 0 else 0
                Ms[i] = max(Ms[i], m)
        sur["M_opt"] = Ms
        sur["mlmc_s"] = sum(m * r["s_per_sample"] for m, r in zip(Ms, vl))
        sur["mlmc_s_incl_training"] = sur["mlmc_s"] + sur["train_s"]
    print(json.dumps({"workload": wl.name, "L_max": wl.L_max, "N": wl.N, "eps_rel": eps_rel, "eps_abs": eps, "estimate": est, "levels": rows,
                      "M_opt": M, "mlmc_s": t_mlmc, "mc_samples": m_mc, "mc_s_per_sample": t_mc,
                      "mc_s": m_mc * t_mc, "mlmc_speedup_vs_mc": m_mc * t_mc / t_mlmc if t_mlmc > 0 else None,
                      "surrogate": sur, "extrapolated": True}))


if __name__ == "__main__":
    main()
