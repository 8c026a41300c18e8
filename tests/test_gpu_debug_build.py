"""The CN_DEBUG build (libcn_b300_debug.so): every global-memory access of the
kernels is checked against the buffers the enqueuing call registered, and an
access outside all of them is recorded and skipped (include/cn.h,
cn_debug_report) -- the stand-in for a memory sanitizer.  Runs in a fresh
process (the package loads one library per process): the planted-access self
test, then every entry point over configurations that reach every kernel --
ragged sizes, the large-grid blocks with the coefficient table, long blocks
with device scratch and the serial RS stage, few long blocks on one CTA each
(prefix scans) with the RS stage on one warp, recompute mode, the adjoint, the
host-buffer step, a batch, slabs with tiny and uneven joint lines, the
no-allocation solve and the control-field maps -- with no violation reported,
and the results against the oracle."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    import oracle
    import workloads as W
    import paper_2205_00856_b300 as cnb
    from paper_2205_00856_b300.sharded import step_slabs
    cnb.use_debug_library()
    assert cnb.version().endswith("debug"), cnb.version()
    assert cnb.load().cn_debug_selftest() == 0
    dev = torch.device("cuda:0")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    def clean(what):
        st, addr, nb = cnb.debug_report()
        assert st == 0, (what, st, hex(addr), nb)

    def rel(x, y):
        return float(np.linalg.norm(x - y) / np.linalg.norm(y))

    for arith in (cnb.ARITH_F64, cnb.ARITH_DF64):
        m0, m1, ml = cnb.LARGE_GRID_BLOCKS[arith]
        for n, kw in ((100003, {{}}), (1 << 21, dict(block=m0, level1_block=m1, level_block=ml,
                                                    flags=cnb.FLAG_COEFF_TABLE)),
                      (1 << 20, dict(flags=cnb.FLAG_PERSISTENT_LEVELS)), (1 << 20, dict(flags=cnb.FLAG_LEVEL_LAUNCHES)),
                      (200001, dict(levels=[40, 20])), (70001, dict(flags=cnb.FLAG_RECOMPUTE)),
                      (20011, dict(levels=[300, 8])), (5001, dict(levels=[1024]))):
            cfg = W.soft_coulomb_config(n=n, nsteps=5)
            prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
            psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n)
            E = W.field_midpoints(5, cfg["dt"], t0=120.0)
            p = cnb.Plan(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=cnb.POT_SOFTCOULOMB, soft_s=2.0, arith=arith, **kw)
            out = p.step(T(psi0), 5, E_mid=T(E)).cpu().numpy()
            p.check()
            clean(("step", arith, n))
            assert rel(out, oracle.cn_run(prob, psi0, 5, E_mid=E)) <= 1e-11
            p.step(T(psi0), 1, E_mid=T(E))
            p.step_states(T(psi0), 3, E_mid=T(E))
            b, a, c, d = (T(v) for v in W.random_system(n, np.random.default_rng(n)))
            p.solve_tridiag(b, a, c, d)
            g = torch.zeros(1, dtype=torch.float64, device=dev)
            psi1 = p.step(T(psi0), 1, E_mid=T(E))
            p.adjoint_step(T(psi0), psi1, psi1.clone(), g, E_mid=T(E))
            if n <= 200001:
                p.step_host(psi0, 2, E_mid=E[:2])
            p.check()
            clean(("all entry points", arith, n))
            p.close()
        sizes = [1500, 30011, 4097, 250003]
        cos_a = np.random.default_rng(9).uniform(-0.5, 0.5, (len(sizes), 8))
        bt = cnb.Batch(sizes, 0.1, 0.01, pot=cnb.POT_COSSERIES, cos_a=cos_a, arith=arith)
        bt.step(T(np.concatenate([W.full_support_state(k, 0.1, -(k // 2) * 0.1, seed=k) for k in sizes])), 3)
        bt.check()
        clean(("batch", arith))
        bt.close()
        n = 20001
        cfg = W.soft_coulomb_config(n=n, nsteps=4)
        psi0 = W.full_support_state(n, cfg["dx"], cfg["x_min"], seed=n)
        E = W.field_midpoints(4, cfg["dt"], t0=140.0)
        for joints, kw in ((None, {{}}), ([0, 2, 5, 4000, 4003, 13001, n - 4, n - 1], dict(block=13, level_block=8))):
            G = 4 if joints is None else len(joints) - 1
            sl = [cnb.Slab(n, cfg["dx"], cfg["dt"], cfg["x_min"], G, r, joints=joints, pot=cnb.POT_SOFTCOULOMB,
                           soft_s=2.0, arith=arith, **kw) for r in range(G)]
            ps = [T(psi0[s.lo:s.hi + 1]) for s in sl]
            step_slabs(sl, ps, 4, E_mid=T(E))
            full = np.empty(n, np.complex128)
            for s, v in zip(sl, ps):
                full[s.lo:s.hi + 1] = v.cpu().numpy()
                s.check()
                s.close()
            clean(("slabs", arith, joints))
            prob = oracle.Problem(n, cfg["dx"], cfg["dt"], cfg["x_min"], pot=oracle.POT_SOFTCOULOMB, soft_s=2.0)
            assert rel(full, oracle.cn_run(prob, psi0, 4, E_mid=E)) <= 1e-11
        for n in (3, 9, 130, 1025, 100003):
            b, a, c, d = W.random_system(n, np.random.default_rng(n))
            x = cnb.solve_tridiag_noalloc(T(b), T(a), T(c), T(d), arith=arith).cpu().numpy()
            clean(("noalloc", arith, n))
            assert rel(x, oracle.thomas(b, a, c, d)) <= 1e-12
    u = torch.rand(50, dtype=torch.float64, device=dev)
    Em = cnb.field_from_controls(u, 4.0, 0.0, 0.02, 200)
    cnb.field_grad_to_controls(Em, 4.0, 0.0, 0.02, 50)
    torch.cuda.synchronize()
    clean("controls")
    print("DEBUG BUILD OK")
""")


@pytest.mark.gpu
def test_debug_build_reports_no_out_of_bounds_access():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "DEBUG BUILD OK" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])


def test_default_build_has_no_checks():
    """The default build reports that it checks nothing (CN_ERR_UNSUPPORTED)."""
    import paper_2205_00856_b300 as cnb
    lib = cnb.load()
    assert lib.cn_debug_selftest() == 2
    assert cnb.debug_report()[0] == 2
    assert not cnb.version().endswith("debug")
