"""The partition model (Sec. 4.3) against the paper's closed forms: Eq.
optimal_nblocks (one iteration), Eq. optimal-P-multistage (equal split for
alpha = beta), a brute-force minimisation of the model, and recovery of known
constants by the least-squares fit.  Host only."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2205_00856_b300 import partition as pm


@pytest.mark.parametrize("n,L,nbl1", [(300000, 1, 512), (300000, 2, 4096), (300000, 3, 20000), (1 << 24, 2, 1 << 16),
                                      (1000, 4, 200), (50, 1, 100)])
def test_level_blocks_structure(n, L, nbl1):
    blocks = pm.level_blocks(n, L, nbl1)
    assert len(blocks) == L and min(blocks) >= 3
    counts, base = pm.level_counts(n, blocks)
    # level 0 thread count close to the request unless the minimum block length binds
    if (n - 1) / nbl1 >= 3:
        assert 0.6 * nbl1 <= counts[0] <= 1.6 * nbl1
    rows = n
    for m, c in zip(blocks, counts):
        assert c == math.ceil((rows - 1) / m)
        rows = c + 1
    assert base == rows


def test_one_iteration_optimum_is_eq_optimal_nblocks():
    for n, a, b in [(3e5, 1.0, 1.0), (3e5, 0.2, 3.0), (2 ** 24, 5.0, 0.5)]:
        o = pm.optimum(n, 1, a, b)
        assert o["nbl1"] == pytest.approx(math.sqrt(a / b) * math.sqrt(n), rel=1e-12)
        # t* = alpha n / n_bl + beta n_bl at n_bl = delta sqrt(n) = 2 sqrt(alpha beta n)
        assert o["time"] == pytest.approx(2 * math.sqrt(a * b * n), rel=1e-12)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 6])
def test_equal_constants_give_eq_optimal_p_multistage(L):
    n = 3e5
    o = pm.optimum(n, L, 1.0, 1.0)
    assert o["ratio"] == pytest.approx(n ** (1.0 / (L + 1)), rel=1e-12)
    assert o["rs_rows"] == pytest.approx(o["ratio"], rel=1e-12)  # n_bl(i)/n_bl(i+1) ~ n_bl(n_it)
    assert o["nbl1"] == pytest.approx(pm.paper_optimum_nbl1(n, L), rel=1e-12)
    # t* = (alpha n_it + beta) n^(1/(n_it+1)) with alpha = beta = 1
    assert o["time"] == pytest.approx((L + 1) * n ** (1.0 / (L + 1)), rel=1e-12)


@pytest.mark.parametrize("L,a,b", [(1, 0.3, 2.0), (2, 1.0, 4.0), (3, 2.0, 0.7)])
def test_optimum_matches_brute_force_minimisation(L, a, b):
    n = 3e5

    def t(logr):  # ratios r_i = n_bl(i)/n_bl(i+1) free, RS rows n / prod r
        r = np.exp(logr)
        return a * np.sum(r) + b * n / np.prod(r)

    res = minimize(t, np.full(L, math.log(10.0)), method="Nelder-Mead",
                   options={"xatol": 1e-10, "fatol": 1e-12, "maxiter": 20000})
    o = pm.optimum(n, L, a, b)
    assert res.fun == pytest.approx(o["time"], rel=1e-6)
    assert np.allclose(np.exp(res.x), o["ratio"], rtol=1e-3)


def test_fit_recovers_constants():
    rng = np.random.default_rng(0)
    n = 300000
    truth = dict(alpha=2e-4, beta=6e-4, c0=0.01, c1=0.004)
    recs = []
    for L in (1, 2, 3):
        for nbl1 in (32, 90, 256, 724, 2048, 5793, 16384, 46341):
            blocks = pm.level_blocks(n, L, nbl1)
            ms = pm.model_time(n, blocks, truth["alpha"], truth["beta"], truth["c0"], truth["c1"])
            recs.append({"n": n, "blocks": blocks, "ms": ms * (1 + 0.002 * rng.standard_normal())})
    f = pm.fit(recs)
    assert f["alpha_ms"] == pytest.approx(truth["alpha"], rel=0.03)
    assert f["beta_ms"] == pytest.approx(truth["beta"], rel=0.03)
    assert f["delta"] == pytest.approx(math.sqrt(truth["alpha"] / truth["beta"]), rel=0.03)
    assert f["r2_relative"] > 0.99


def test_features_sum_block_lengths():
    n = 1001
    x = pm.features(n, [10, 4])
    # level 0: 1000/10 = 100 blocks; level 1: 101 rows, 25 blocks; RS 26 rows
    assert x[0] == pytest.approx(1001 / 100 + 101 / 25)
    assert x[1] == 26 and x[2] == 1 and x[3] == 2
