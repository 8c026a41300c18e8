"""Write the regression fixtures of tests/golden/ from the FP64 oracle only.

The paper prints no worked example (its only figure is absent from the text), so
these fixtures are not the paper's numbers: they freeze oracle outputs on tiny
seeded cases so that a later change to the oracle's arithmetic shows up as a
diff.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def cpx(a):
    return [[float(z.real), float(z.imag)] for z in np.asarray(a)]


def main():
    rng = np.random.default_rng(W.SEED)
    b, a, c, d = W.random_system(9, rng)
    J = np.array([0, 3, 5, 8], np.int64)
    bw, aw, cw, dw = oracle.nshape_reduce(b, a, c, d, J, order=1)
    table1 = {"source": "oracle Table 1 restatement (Sec. 4), order (RD+JD)+(RU+JU)",
              "n": 9, "J": J.tolist(), "b": cpx(b), "a": cpx(a), "c": cpx(c), "d": cpx(d),
              "reduced_b": cpx(bw), "reduced_a": cpx(aw), "reduced_c": cpx(cw), "reduced_d": cpx(dw),
              "x": cpx(oracle.nshape_solve(b, a, c, d, J))}
    with open(os.path.join(HERE, "table1_n9.json"), "w") as f:
        json.dump(table1, f, indent=1)
    cfg = W.free_packet_config()
    psi = oracle.cn_run(oracle.Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"]), W.initial_state(cfg),
                        cfg["nsteps"])
    idx = list(range(0, cfg["n"], 256)) + [cfg["n"] - 1]
    free = {"source": "oracle CN stepper (Sec. 2), free packet N=4096, dx=0.1, dt=0.01, 100 steps",
            "index": idx, "psi": cpx(psi[idx])}
    with open(os.path.join(HERE, "free_packet_n4096_100.json"), "w") as f:
        json.dump(free, f, indent=1)


if __name__ == "__main__":
    main()
