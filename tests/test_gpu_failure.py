"""Device-side failure reporting without a GPU fault: a bounded wait on an mbarrier
that nothing completes (the wait the TMA-staged substitution uses) returns
CN_ERR_TIMEOUT through a status word, the kernel ends normally and the context
stays usable; a zero pivot is covered in test_gpu_parity."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2205_00856_b300 as cnb  # noqa: E402


def test_bounded_wait_reports_timeout_and_context_survives():
    for polls in (1, 64, 4096):
        assert cnb.diag_wait_timeout(polls) == 5  # CN_ERR_TIMEOUT
    with pytest.raises(cnb.CNError):
        cnb._check(cnb.diag_wait_timeout(0), "diag")  # invalid argument, checked on the host
    # the context still runs the solver correctly
    cfg = W.free_packet_config()
    psi0 = W.initial_state(cfg)
    plan = cnb.Plan(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"], arith=cnb.ARITH_DF64)
    out = plan.step(torch.from_numpy(psi0).to("cuda"), 10).cpu().numpy()
    assert plan.status() == 0
    ref = oracle.cn_run(oracle.Problem(cfg["n"], cfg["dx"], cfg["dt"], cfg["x_min"]), psi0, 10)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-11
