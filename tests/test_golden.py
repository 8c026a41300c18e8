"""Regression fixtures written by tests/golden/make_golden.py from the oracle
(the paper prints no worked example): the oracle must keep reproducing them."""
import json
import os

import numpy as np

import oracle
import workloads as W

G = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def arr(v):
    v = np.asarray(v, dtype=np.float64)
    return v[:, 0] + 1j * v[:, 1]


def test_table1_fixture():
    g = json.load(open(os.path.join(G, "table1_n9.json")))
    b, a, c, d = arr(g["b"]), arr(g["a"]), arr(g["c"]), arr(g["d"])
    J = np.array(g["J"], np.int64)
    red = oracle.nshape_reduce(b, a, c, d, J, order=1)
    for got, key in zip(red, ("reduced_b", "reduced_a", "reduced_c", "reduced_d")):
        assert np.allclose(got, arr(g[key]), rtol=1e-15, atol=1e-15)
    assert np.allclose(oracle.nshape_solve(b, a, c, d, J), arr(g["x"]), rtol=1e-15, atol=1e-15)


def test_free_packet_fixture():
    g = json.load(open(os.path.join(G, "free_packet_n4096_100.json")))
    cfg = W.free_packet_config()
    psi = oracle.cn_run(oracle.Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"]), W.initial_state(cfg),
                        cfg["nsteps"])
    assert np.allclose(psi[g["index"]], arr(g["psi"]), rtol=1e-14, atol=1e-16)
