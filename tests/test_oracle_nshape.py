"""Pins for the oracle's literal Table 1 restatement (Sec. 4 of the paper).

The N-shaped partition method is an exact direct solver, so every variant
(partition count, unequal blocks, nesting depth, stage order) must reproduce
a dense LU solve to round-off.  The structural claims of Sec. 4 (fill-in
columns J_w / J_{w+1}, the reduced tridiagonal system on the joint lines) are
checked against the exact solution: every transformed row must hold as an
equation using only the columns the paper says remain non-zero.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def dense(b, a, c):
    n = len(a)
    return np.diag(a) + np.diag(b[1:], -1) + np.diag(c[:-1], 1)


def rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def random_joints(n, P, rng):
    """Joint lines with unequal gaps >= 2 (Sec. 4.1.1: blocks may differ in size)."""
    extra = n - 1 - 2 * P
    assert extra >= 0
    gaps = 2 + rng.multinomial(extra, rng.dirichlet(np.full(P, 0.5)))
    return np.concatenate([[0], np.cumsum(gaps)]).astype(np.int64)


@pytest.mark.parametrize("n,P", [(3, 1), (5, 2), (9, 1), (9, 3), (17, 8), (64, 16), (65, 32), (200, 3)])
@pytest.mark.parametrize("order", [0, 1])
def test_nshape_equals_dense_default_joints(n, P, order):
    rng = np.random.default_rng(100 * n + P)
    b, a, c, d = W.random_system(n, rng)
    J = oracle.default_joints(n, P)
    x = oracle.nshape_solve(b, a, c, d, J, order=order)
    assert rel(x, np.linalg.solve(dense(b, a, c), d)) <= 1e-13
    assert rel(x, oracle.thomas(b, a, c, d)) <= 1e-13


@pytest.mark.parametrize("seed", range(6))
def test_nshape_unequal_blocks(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 120))
    P = int(rng.integers(1, (n - 1) // 2))
    J = random_joints(n, P, rng)
    b, a, c, d = W.random_system(n, rng)
    x = oracle.nshape_solve(b, a, c, d, J)
    assert rel(x, np.linalg.solve(dense(b, a, c), d)) <= 1e-13


@pytest.mark.parametrize("n,P,nested", [(257, 64, [16]), (257, 64, [16, 4]), (1000, 250, [60, 12, 3]),
                                        (101, 50, [25, 12, 6, 3, 1])])
def test_nshape_nested_iteration(n, P, nested):
    # Eq. (iteration): the reduced system is solved again by the N-shaped method
    rng = np.random.default_rng(n + P)
    b, a, c, d = W.random_system(n, rng)
    J = oracle.default_joints(n, P)
    x = oracle.nshape_solve(b, a, c, d, J, nested_P=nested)
    assert rel(x, oracle.thomas(b, a, c, d)) <= 1e-13


def test_nshape_cn_matrix():
    cfg = W.free_packet_config()
    prob = oracle.Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"])
    b, a, c = oracle.cn_matrix(prob)
    bs, as_, cs = oracle.cn_matrix(prob, dt_sign=-1)
    d = oracle.tridiag_apply(bs, as_, cs, W.initial_state(cfg))
    J = oracle.default_joints(cfg["n"], cfg["n_parts"])
    x = oracle.nshape_solve(b, a, c, d, J, nested_P=[4])
    assert rel(x, oracle.thomas(b, a, c, d)) <= 1e-14


def test_stage_order_commutes_bitwise():
    # Sec. 5.2.1: JD needs only RD, so (RD+JD)+(RU+JU) equals (RD+RU)+(JU+JD) exactly
    rng = np.random.default_rng(11)
    n = 77
    b, a, c, d = W.random_system(n, rng)
    J = random_joints(n, 9, rng)
    r0 = oracle.nshape_reduce(b, a, c, d, J, order=0)
    r1 = oracle.nshape_reduce(b, a, c, d, J, order=1)
    for u, v in zip(r0, r1):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("P", [1, 2, 5, 13])
def test_structure_after_reduction(P):
    rng = np.random.default_rng(P)
    n = 60
    b, a, c, d = W.random_system(n, rng)
    J = random_joints(n, P, rng)
    x = np.linalg.solve(dense(b, a, c), d)
    bw, aw, cw, dw = oracle.nshape_reduce(b, a, c, d, J)
    # interior rows: b_i in column J_w, c_i in column J_{w+1} (Sec. 4.1.2, Fig. 1b-d)
    for w in range(P):
        for i in range(J[w] + 1, J[w + 1]):
            lhs = bw[i] * x[J[w]] + aw[i] * x[i] + cw[i] * x[J[w + 1]]
            assert abs(lhs - dw[i]) <= 1e-12 * (abs(dw[i]) + abs(aw[i] * x[i]) + 1)
    # joint lines: a tridiagonal system of size P+1 (Fig. 1e)
    for w in range(P + 1):
        i = J[w]
        lhs = aw[i] * x[i]
        if w > 0:
            lhs += bw[i] * x[J[w - 1]]
        if w < P:
            lhs += cw[i] * x[J[w + 1]]
        assert abs(lhs - dw[i]) <= 1e-12 * (abs(dw[i]) + abs(aw[i] * x[i]) + 1)
    # RS then SS reproduce x (Table 1)
    psiJ = oracle.nshape_rs(bw, aw, cw, dw, J)
    assert rel(psiJ, x[J]) <= 1e-13
    assert rel(oracle.nshape_substitute(bw, aw, cw, dw, J, psiJ), x) <= 1e-13


def test_gap_two_blocks_and_single_block():
    # gap 2: RD and RU are empty, JU/JD use the single interior row; P=1: 2x2 reduced system
    rng = np.random.default_rng(5)
    n = 21
    b, a, c, d = W.random_system(n, rng)
    J = np.arange(0, n, 2, dtype=np.int64)
    assert rel(oracle.nshape_solve(b, a, c, d, J), np.linalg.solve(dense(b, a, c), d)) <= 1e-13
    x1 = oracle.nshape_solve(b, a, c, d, np.array([0, n - 1]))
    assert rel(x1, np.linalg.solve(dense(b, a, c), d)) <= 1e-13


def test_linearity_of_solve():
    rng = np.random.default_rng(9)
    n = 50
    b, a, c, d1 = W.random_system(n, rng)
    d2 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    J = oracle.default_joints(n, 7)
    al, be = 0.3 - 1.2j, -2.0 + 0.5j
    lhs = oracle.nshape_solve(b, a, c, al * d1 + be * d2, J)
    rhs = al * oracle.nshape_solve(b, a, c, d1, J) + be * oracle.nshape_solve(b, a, c, d2, J)
    assert rel(lhs, rhs) <= 1e-14
