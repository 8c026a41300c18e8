"""Seeded random configurations of the CN step against the FP64 oracle: sizes from 3
to 60000 (ragged tails, single-block and base-only levels), level-0 and level block
sizes 3..32 (level 1 on its own or not), both arithmetics, store and recompute modes,
the three potential kinds, default and explicit nesting; the states kept by
cn_step_states end on the plain step's result bitwise.  Tolerance as the other parity tests (rel L2 <= 1e-11)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_00856_b300 as cnb  # noqa: E402

DEV = torch.device("cuda:0")


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(np.exp(rng.uniform(np.log(3), np.log(60000))))
    n = max(n, 3)
    c = dict(n=n, dx=float(rng.choice([0.05, 0.1, 0.2])), dt=float(rng.choice([0.005, 0.01, 0.02])),
             block=int(rng.integers(3, 33)), level_block=int(rng.integers(3, 33)),
             arith=int(rng.integers(0, 2)), flags=int(rng.choice([0, cnb.FLAG_RECOMPUTE, cnb.FLAG_COEFF_TABLE])),
             pot=int(rng.choice([cnb.POT_NONE, cnb.POT_SOFTCOULOMB, cnb.POT_COSSERIES])),
             nsteps=int(rng.integers(1, 12)), field=bool(rng.integers(0, 2)))
    c["x_min"] = -(n // 2) * c["dx"] + float(rng.uniform(-1, 1))
    c["cos_a"] = rng.uniform(-0.5, 0.5, int(rng.integers(1, 9)))
    c["explicit"] = None
    if seed % 4 == 3 and n > 40:
        # an explicit depth: first block up to 64 rows, then what fits
        m0 = int(rng.integers(3, 65))
        levels = [m0]
        rows = (n - 1 + m0 - 1) // m0 + 1
        while rows > 40 and len(levels) < 3:
            ml = int(rng.integers(3, 17))
            levels.append(ml)
            rows = (rows - 1 + ml - 1) // ml + 1
        c["explicit"] = levels
    c["psi0"] = W.gaussian(n, c["dx"], c["x_min"], float(rng.uniform(-2, 2)), max(0.5, 0.02 * n * c["dx"]),
                           float(rng.uniform(-1, 1)))
    c["E"] = 0.05 * np.sin(np.arange(c["nsteps"]) * 0.7 + seed) if c["field"] else None
    c["level1_block"] = int(rng.choice([0, int(rng.integers(3, 33))]))  # drawn last: earlier draws unchanged
    return c


@pytest.mark.parametrize("seed", range(200))
def test_random_configuration_vs_oracle(seed):
    c = _case(seed)
    n = c["n"]
    kw = dict(pot=c["pot"], soft_s=2.0, arith=c["arith"], flags=c["flags"])
    okw = dict(pot=c["pot"], soft_s=2.0)
    if c["pot"] == cnb.POT_COSSERIES:
        kw.update(cos_a=c["cos_a"], L=n * c["dx"])
        okw.update(cos_a=c["cos_a"], L=n * c["dx"])
    if c["explicit"] is not None:
        if c["flags"] == cnb.FLAG_RECOMPUTE and c["explicit"][0] > 32:
            c["flags"] = kw["flags"] = 0
        plan = cnb.Plan(n, c["dx"], c["dt"], c["x_min"], levels=c["explicit"], **kw)
    else:
        plan = cnb.Plan(n, c["dx"], c["dt"], c["x_min"], block=c["block"], level_block=c["level_block"],
                        level1_block=c["level1_block"], **kw)
    E_dev = None if c["E"] is None else torch.from_numpy(c["E"]).to(DEV)
    out = plan.step(torch.from_numpy(c["psi0"]).to(DEV), c["nsteps"], E_mid=E_dev).cpu().numpy()
    # every state kept: the last equals the plain step's result bitwise
    states = plan.step_states(torch.from_numpy(c["psi0"]).to(DEV), c["nsteps"], E_mid=E_dev).cpu().numpy()
    plan.check()
    plan.close()
    assert np.array_equal(states[-1], out)
    ref = oracle.cn_run(oracle.Problem(n, c["dx"], c["dt"], c["x_min"], **okw), c["psi0"], c["nsteps"], E_mid=c["E"])
    err = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    assert err <= 1e-11, {k: c[k] for k in ("n", "block", "level_block", "level1_block", "arith", "flags", "pot",
                                            "nsteps", "explicit")} | {"err": err}
