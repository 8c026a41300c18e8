"""Partition study of the N-shaped method: the paper's time model (Sec. 4.3),
its optimum (Eq. optimal_nblocks for one iteration, Eq. optimal-P-multistage
for nested iterations), a least-squares fit of the model's constants to times
measured on the GPU, and the sweep that measures them (the shape of Fig. 2).

Model.  With n_bl(0) = n rows and n_bl(i+1) parallel blocks at level i, one
thread per block, a solve with n_it nested iterations costs

    t = alpha * sum_{i<n_it} n_bl(i) / n_bl(i+1)  +  beta * n_bl(n_it)  (+ c0 + c1 n_it)

(the first sum is the sequential RD/RU/SS work of one block per level, the
second the serial RS stage on the last reduced system).  The paper's model has
no c0, c1; on a GPU every level costs two kernel launches, so the fit carries a
constant per solve and one per level.  For fixed n_it the model is smallest
when every level divides by the same ratio r:

    r* = (n beta / alpha)^(1 / (n_it + 1)),  n_bl(1)* = n / r*,
    t* = alpha (n_it + 1) r*,

which for n_it = 1 is n_bl* = delta sqrt(n), delta = sqrt(alpha / beta)
(Eq. optimal_nblocks), and for alpha = beta the paper's equal split
n_bl(i)/n_bl(i+1) ~ n_bl(n_it) ~ n^(1/(n_it+1)) (Eq. optimal-P-multistage).

Run on a GPU:  python -m paper_2205_00856_b300.partition --n 300000
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np


# ----------------------------------------------------------------- model (host only)
def level_blocks(n: int, n_it: int, nbl1: int, min_block: int = 3) -> list[int]:
    """Block sizes [m_0 .. m_{n_it-1}] that put about nbl1 threads on level 0 and
    split the remaining levels by equal ratios r = nbl1^(1/n_it) (so the RS stage
    gets about r rows, the equal-work split of Eq. optimal-P-multistage)."""
    if n < 3 or n_it < 1 or nbl1 < 1:
        raise ValueError("need n >= 3, n_it >= 1, nbl1 >= 1")
    m0 = max(min_block, int(round((n - 1) / nbl1)))
    blocks = [m0]
    rows = (n - 1 + m0 - 1) // m0 + 1  # P_0 + 1
    for i in range(1, n_it):
        left = n_it - i + 1  # reductions still to make, counting the RS split
        r = max(min_block, int(round((rows - 1) ** (1.0 / left))))
        blocks.append(r)
        rows = (rows - 1 + r - 1) // r + 1
    return blocks


def level_counts(n: int, blocks) -> tuple[list[int], int]:
    """(blocks per level n_bl(1..n_it), rows of the RS system) for a block list."""
    rows, counts = n, []
    for m in blocks:
        P = (rows - 1 + m - 1) // m
        counts.append(P)
        rows = P + 1
    return counts, rows


def features(n: int, blocks) -> np.ndarray:
    """Model features [sum of block lengths, RS rows, 1, levels] of one configuration."""
    counts, base = level_counts(n, blocks)
    rows = [n] + [c + 1 for c in counts[:-1]]
    seq = sum(r / c for r, c in zip(rows, counts))  # n_bl(i) / n_bl(i+1)
    return np.array([seq, float(base), 1.0, float(len(blocks))])


def model_time(n: int, blocks, alpha: float, beta: float, c0: float = 0.0, c1: float = 0.0) -> float:
    return float(features(n, blocks) @ np.array([alpha, beta, c0, c1]))


def optimum(n: float, n_it: int, alpha: float, beta: float) -> dict:
    """Continuous optimum of the model for fixed depth: equal ratio r* per level."""
    r = (n * beta / alpha) ** (1.0 / (n_it + 1))
    return {"ratio": r, "nbl1": n / r, "rs_rows": n / r ** n_it, "time": alpha * (n_it + 1) * r}


def paper_optimum_nbl1(n: float, n_it: int) -> float:
    """Eq. optimal-P-multistage up to its constant: n_bl(1) ~ n^(n_it/(n_it+1))."""
    return n ** (n_it / (n_it + 1.0))


def fit(records, n_key: str = "n") -> dict:
    """Least-squares alpha, beta, c0, c1 from records {n, blocks, ms}; alpha and
    beta in ms per row, constants in ms.  Returns them with delta = sqrt(alpha/beta)
    and the coefficient of determination R^2."""
    X = np.array([features(r[n_key], r["blocks"]) for r in records])
    y = np.array([r["ms"] for r in records], dtype=float)
    # relative residuals: times span orders of magnitude across the sweep
    w = 1.0 / y
    coef, *_ = np.linalg.lstsq(X * w[:, None], y * w, rcond=None)
    alpha, beta, c0, c1 = (float(v) for v in coef)
    pred = X @ coef
    ss_res = float(np.sum(((y - pred) * w) ** 2))
    ss_tot = float(np.sum(((y - np.average(y, weights=w * w)) * w) ** 2))
    out = {"alpha_ms": alpha, "beta_ms": beta, "c0_ms": c0, "c1_ms": c1,
           "r2_relative": 1.0 - ss_res / ss_tot if ss_tot > 0 else float("nan")}
    out["delta"] = math.sqrt(alpha / beta) if alpha > 0 and beta > 0 else float("nan")
    return out


# ----------------------------------------------------------------- GPU sweep
def time_plan(torch, cnb, plan, n, cfg, steps: int, reps: int) -> float:
    """ms per CN step (in place, store mode), one cn_step call per step -- each
    step a complete N-shaped solve with its own level-0 kernels, as the paper's
    time model describes it (a multi-step call would fuse one step's substitution
    with the next step's reduction) -- the calls replayed from a CUDA graph so no
    host launch cost enters; best of reps after one warm-up replay."""
    import workloads as W
    psi = torch.from_numpy(W.gaussian(n, cfg["dx"], cfg["x_min"], 0.0, 1.0, 0.0)).to("cuda")
    E = torch.full((steps,), 0.01, dtype=torch.float64, device="cuda")
    plan.step(psi, 1, E_mid=E, psi_out=psi)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            for k in range(steps):
                plan.step(psi, 1, E_mid=E[k:k + 1], psi_out=psi)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / steps)
    plan.check()
    del g
    return best


def sweep(n: int, depths, nbl1_grid, arith: str = "f64", steps: int = 10, reps: int = 3) -> dict:
    """Time one CN step of the soft-Coulomb workload on n points for every depth
    and first-level thread count, fit the model, and compare optima."""
    import torch

    import paper_2205_00856_b300 as cnb
    import workloads as W

    cfg = W.soft_coulomb_config(n=n)
    ar = cnb.ARITH_DF64 if arith == "df64" else cnb.ARITH_F64
    recs = []
    for L in depths:
        for nbl1 in nbl1_grid:
            blocks = level_blocks(n, L, nbl1)
            counts, base = level_counts(n, blocks)
            if counts[0] < 1 or (L > 1 and min(counts) < 1):
                continue
            try:
                # one thread per block: the per-block serial elimination the paper's model times
                plan = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0,
                                arith=ar, levels=blocks, flags=cnb.FLAG_SERIAL_BLOCKS)
            except cnb.CNError:
                continue  # depth too deep for this first level
            ms = time_plan(torch, cnb, plan, n, cfg, steps, reps)
            plan.close()
            recs.append({"n": n, "n_it": L, "blocks": blocks, "nbl": counts, "rs_rows": base, "ms": ms})
    default = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=ar)
    default_ms = time_plan(torch, cnb, default, n, cfg, steps, reps)
    info = default.info()
    default.close()
    model = fit(recs)
    per_depth = []
    for L in depths:
        rs = [r for r in recs if r["n_it"] == L]
        if not rs:
            continue
        best = min(rs, key=lambda r: r["ms"])
        opt = optimum(n, L, model["alpha_ms"], model["beta_ms"]) if model["alpha_ms"] > 0 and model["beta_ms"] > 0 \
            else None
        per_depth.append({"n_it": L, "measured_best_nbl1": best["nbl"][0], "measured_best_ms": best["ms"],
                          "measured_best_blocks": best["blocks"],
                          "model_opt_nbl1": opt["nbl1"] if opt else None,
                          "model_opt_ms": (opt["time"] + model["c0_ms"] + model["c1_ms"] * L) if opt else None,
                          "paper_formula_nbl1_shape": paper_optimum_nbl1(n, L)})
    return {"n": n, "arith": arith, "workload": "soft_coulomb_laser_1d_cn", "steps": steps, "reps": reps,
            "records": recs, "fit": model, "per_depth": per_depth,
            "default_plan": {"ms": default_ms, "level_rows": info["level_rows"],
                             "level_block": info["level_block"]}}


def summarize(res: dict, command: str) -> str:
    """Markdown summary of a sweep: fit, per-depth optimum vs model vs the
    paper's formula, and the time of every configuration."""
    f = res["fit"]
    lines = [f"# Partition sweep: {res['workload']}, n = {res['n']}, {res['arith']}", "",
             f"Command: `{command}`", "",
             f"ms per CN step (in place, store mode, one cn_step call per step, replayed from a CUDA graph), best of {res['reps']} x {res['steps']} steps after one warm-up.",
             "Model t = alpha sum_i n_bl(i)/n_bl(i+1) + beta n_bl(n_it) + c0 + c1 n_it, fitted by least squares "
             "on relative residuals over all configurations.", "",
             f"Fit: alpha = {f['alpha_ms'] * 1e3:.4g} us/row, beta = {f['beta_ms'] * 1e3:.4g} us/row, "
             f"c0 = {f['c0_ms'] * 1e3:.4g} us, c1 = {f['c1_ms'] * 1e3:.4g} us/level, "
             f"delta = sqrt(alpha/beta) = {f['delta']:.4g}, relative R^2 = {f['r2_relative']:.4f}", "",
             "| n_it | measured best n_bl(1) | blocks | ms | model optimum n_bl(1) | model ms | "
             "paper n^(n_it/(n_it+1)) |", "|---|---|---|---|---|---|---|"]
    for p in res["per_depth"]:
        lines.append(f"| {p['n_it']} | {p['measured_best_nbl1']} | {p['measured_best_blocks']} | "
                     f"{p['measured_best_ms']:.4f} | {p['model_opt_nbl1']:.0f} | {p['model_opt_ms']:.4f} | "
                     f"{p['paper_formula_nbl1_shape']:.0f} |")
    d = res["default_plan"]
    lines += ["", f"Default plan (block {d['level_block'][0]}, reduced levels nested until <= 1024 rows, which "
              f"one CTA solves by cyclic reduction; levels {d['level_rows']}): {d['ms']:.4f} ms.", "",
              "## All configurations", "",
              "| n_it | n_bl(1) | blocks | RS rows | ms | model ms |", "|---|---|---|---|---|---|"]
    for r in res["records"]:
        mt = model_time(res["n"], r["blocks"], f["alpha_ms"], f["beta_ms"], f["c0_ms"], f["c1_ms"])
        lines.append(f"| {r['n_it']} | {r['nbl'][0]} | {r['blocks']} | {r['rs_rows']} | {r['ms']:.4f} | {mt:.4f} |")
    return "\n".join(lines) + "\n"


def _log_grid(lo: int, hi: int, per_octave: int) -> list[int]:
    k = np.arange(math.log2(lo) * per_octave, math.log2(hi) * per_octave + 1e-9) / per_octave
    return sorted({int(round(2 ** v)) for v in k})


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=300000)
    ap.add_argument("--depths", type=str, default="1,2,3,4")
    ap.add_argument("--nbl-min", type=int, default=16)
    ap.add_argument("--nbl-max", type=int, default=65536)
    ap.add_argument("--per-octave", type=int, default=2)
    ap.add_argument("--arith", choices=["f64", "df64"], default="f64")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--md", type=str, default=None, help="also write a markdown summary here")
    a = ap.parse_args(argv)
    res = sweep(a.n, [int(v) for v in a.depths.split(",")], _log_grid(a.nbl_min, a.nbl_max, a.per_octave),
                a.arith, a.steps, a.reps)
    print(json.dumps(res), flush=True)
    if a.md:
        cmd = "python -m paper_2205_00856_b300.partition " + " ".join(argv if argv is not None else sys.argv[1:])
        with open(a.md, "w") as fh:
            fh.write(summarize(res, cmd))
    return 0


if __name__ == "__main__":
    sys.exit(main())
