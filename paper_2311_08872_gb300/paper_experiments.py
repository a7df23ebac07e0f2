"""The two kinds of experiment of Section 7 on the paper's own setting.

    python -m paper_2311_08872_gb300.paper_experiments --workload paper_reg --N 2e5 --type 1
    python -m paper_2311_08872_gb300.paper_experiments --workload paper_irreg --N 2e9 --type 2

Setting (Section 7.2): torus (0, 2 pi)^2, h_l = 2 pi 2^-(2+l), tau_l = 1e-3 4^(5-l),
T = 1.024, psi = x^2, phi = sin x + sin y, initial datum rho-bar_(0,reg) or
rho-bar_(0,irreg) (workloads `paper_reg`, `paper_irreg`), N particles.

Type 1: Algorithm 1 (mlmc_dk_estimate, absolute eps) for each accuracy of the
paper's lists (10^-1.4 ... 10^-2.6, and 10^-2.75 for the irregular datum),
with plain Monte Carlo on the finest level L reached: ceil(2 Var[P_L] / eps^2)
samples (the paper extrapolates its MC times the same way).  Costs use the
device time per sample of each level measured on large pilot batches, since
the small batches of a run on these tiny grids are bound by launch latency:
MLMC sum_l M_l t_l, MC M_MC t_MC(L).  Output per eps: L, samples per level,
estimate, both costs and their ratio.

Type 2: for each finest level L = 1..L_max, MLMC with the geometric
progression M_(l-1) = 4 M_l and a plain-MC estimator on level L of the same
cost; the ratio of their variances is the variance reduction factor of
Proposition PropVarFactor, printed beside h_min^-beta |log2 h_min|^-1 scaled to
agree at L = 1 (beta = 2 for the NN coupling, 4 for the Fourier coupling:
`paper_reg_fourier`, the regular setting on 6^2, 18^2, 54^2).

Each row is printed as it completes, then one JSON line with all rows.  Times
are device times of the level kernels (CUDA events) on the GPU this runs on.
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

EPS_REG = [10 ** -1.4, 10 ** -1.7, 10 ** -2.0, 10 ** -2.2, 10 ** -2.4, 10 ** -2.6]
EPS_IRREG = [10 ** -1.4, 10 ** -1.7, 10 ** -2.0, 10 ** -2.2, 10 ** -2.4, 10 ** -2.75]


def _var(s):
    return max(0.0, (s.dp2 - s.dp1 ** 2 / s.n) / (s.n - 1))


def _var_pf(s):
    return max(0.0, (s.pf2 - s.pf1 ** 2 / s.n) / (s.n - 1))


def per_sample_times(ctx, L_max, seed, seconds=0.3):
    """Device seconds per coupled sample (level 0: per sample) and per plain-MC
    sample of every level, and Var[P_l] of plain MC, from pilots large enough
    (about `seconds` each) that launch latency is amortised."""
    out = []
    for l in range(L_max + 1):
        info = ctx.level_info(l)
        n_c = int(max(256, min(2_000_000, seconds * 2.5e11 / info.cost)))
        n_m = int(max(256, min(2_000_000, seconds * 2.5e11 / info.cost_mc)))
        c = ctx.run_level(l, n_c, seed + 2 * l)[0]
        m = ctx.run_level(l, n_m, seed + 2 * l + 1, mc=True)[0]
        out.append({"level": l, "t_coupled": c.kernel_s / c.n, "t_mc": m.kernel_s / m.n, "var_P": _var_pf(m),
                    "pilot_coupled": n_c, "pilot_mc": n_m})
    return out


def type1(ctx, eps_list, seed, times):
    """Algorithm 1 per eps; costs from the amortised per-sample device times
    (MLMC: sum_l M_l t_l; MC: ceil(2 Var[P_L] / eps^2) t_MC(L)); the device
    time of the run itself (small batches, launch-latency bound) beside it."""
    rows = []
    for i, eps in enumerate(eps_list):
        r = ctx.estimate(eps, False, seed + 17 * i)
        L = r.L
        var_pl = r.var_pf[L] if r.var_pf[L] > 0 else times[L]["var_P"]
        m_mc = math.ceil(2.0 * var_pl / eps ** 2)
        mlmc_s = sum(r.M[l] * times[l]["t_coupled"] for l in range(L + 1))
        mc_s = m_mc * times[L]["t_mc"]
        rows.append({"eps": eps, "log10_eps": math.log10(eps), "L": L, "converged": bool(r.converged),
                     "M": [r.M[l] for l in range(L + 1)], "E": [r.E[l] for l in range(L + 1)],
                     "V": [r.V[l] for l in range(L + 1)], "estimate": r.estimate,
                     "mlmc_s": mlmc_s, "mlmc_run_device_s": sum(r.kernel_s[l] for l in range(L + 1)),
                     "mlmc_run_wall_s": r.wall_s, "mc_samples": m_mc, "mc_s": mc_s, "mc_extrapolated": True,
                     "speedup_mc_over_mlmc": mc_s / mlmc_s if mlmc_s > 0 else None,
                     "eps2_cost_mlmc": eps ** 2 * mlmc_s, "eps2_cost_mc": eps ** 2 * mc_s})
        print(json.dumps({"row": rows[-1]}), flush=True)
    return rows


def type2(ctx, L_max, M_finest, seed, length, times):
    """MLMC with M_(l-1) = 4 M_l against plain MC on level L at equal cost
    (amortised per-sample device times): variance reduction factor."""
    rows = []
    for L in range(1, L_max + 1):
        M = [M_finest * 4 ** (L - l) for l in range(L + 1)]
        var_mlmc, secs, V = 0.0, 0.0, []
        for l in range(L + 1):
            s = ctx.run_level(l, M[l], seed + 31 * L + l)[0]
            V.append(_var(s))
            var_mlmc += V[-1] / s.n
            secs += M[l] * times[l]["t_coupled"]
        m_mc = secs / times[L]["t_mc"]
        var_mc = times[L]["var_P"] / m_mc
        h_min = length / ctx.level_info(L).n
        beta = 4 if ctx.level_info(L).coupling == 1 else 2
        rows.append({"L": L, "h_min": h_min, "M": M, "V": V, "mlmc_s": secs, "var_mlmc": var_mlmc,
                     "mc_samples_same_cost": m_mc, "var_P_L": times[L]["var_P"], "var_mc": var_mc,
                     "variance_reduction": var_mc / var_mlmc if var_mlmc > 0 else None,
                     "predicted_shape": h_min ** -beta / abs(math.log2(h_min))})
        print(json.dumps({"row": rows[-1]}), flush=True)
    base = rows[0]["variance_reduction"] / rows[0]["predicted_shape"] if rows and rows[0]["variance_reduction"] else None
    for r in rows:
        r["predicted_scaled"] = base * r["predicted_shape"] if base else None
    return rows


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper_reg", choices=["paper_reg", "paper_irreg", "paper_reg_fourier"])
    ap.add_argument("--N", type=float, default=2e5)
    ap.add_argument("--type", type=int, default=1, choices=[1, 2])
    ap.add_argument("--eps", type=str, default=None, help="comma-separated absolute accuracies (default: the paper's)")
    ap.add_argument("--M-finest", type=int, default=1024, help="type 2: samples on the finest level")
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args()

    import torch

    from paper_2311_08872_gb300 import build, mlmc_dk, workloads

    build.build()
    wl = workloads.get(args.workload).with_(N=args.N)
    st = torch.cuda.current_stream()
    with mlmc_dk.Context.from_workload(wl, stream=st.cuda_stream) as ctx:
        ctx.tune(1)
        times = per_sample_times(ctx, wl.L_max, args.seed + 5000)
        if args.type == 1:
            eps = [float(x) for x in args.eps.split(",")] if args.eps else (
                EPS_IRREG if args.workload == "paper_irreg" else EPS_REG)
            rows = type1(ctx, eps, args.seed, times)
        else:
            rows = type2(ctx, wl.L_max, args.M_finest, args.seed, wl.length, times)
        levels = [{"level": l, "n": ctx.level_info(l).n, "h": ctx.level_info(l).h, "tau": ctx.level_info(l).tau,
                   "M": ctx.level_info(l).M} for l in range(wl.L_max + 1)]
    print(json.dumps({"workload": wl.name, "N": wl.N, "type": args.type, "levels": levels, "times": times,
                      "rows": rows}))


if __name__ == "__main__":
    main()
