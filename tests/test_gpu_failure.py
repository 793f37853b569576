"""Failure detection of the bounded device waits, without a GPU fault.

The persistent MD kernel's grid barrier gives up after a time limit, flags
MD_E_TIMEOUT in the status word the host reads, and every CTA leaves the
kernel.  md_barrier_selftest makes one CTA leave instead of arriving (a
missing arrival, nothing else skipped) with a 20 ms limit: the call must
report the timeout within a bounded time, and the device must stay usable.
bf16_gemm_selftest does the same for an mbarrier wait of the tensor-core
GEMM: one completion signal is withheld, the wait runs out, the kernel
drains its MMAs and frees its tensor memory, and a normal GEMM afterwards
is correct.
"""

import time

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _system(mdlg, prec, n=20_000, seed=3):
    L = inputs.box_length(n, 0.1)
    st = inputs.lattice_gas_state(n, L, 5.0, seed=seed)
    p = mdlg.make_params(n, L, precision=prec, lg_every=(50,), lx=(int(L),))
    return mdlg.System(p, st.x, st.y, st.vx, st.vy)


@pytest.mark.parametrize("prec", [0, 1])
def test_grid_barrier_wait_runs_out_and_is_reported(mdlg, prec):
    s = _system(mdlg, prec)
    s.step(20)
    s.sync()
    t0 = time.perf_counter()
    rc = s.barrier_selftest(0.02)
    dt = time.perf_counter() - t0
    assert rc == mdlg.MD_E_TIMEOUT, rc
    assert dt < 2.0, dt
    s.close()
    # the context stays usable: a fresh system runs and reports no error
    f = _system(mdlg, prec, seed=4)
    e0 = f.energy()
    f.step(200)
    f.sync()
    e1 = f.energy()
    assert np.all(np.isfinite(e1))
    assert abs((e1[0] + e1[1]) - (e0[0] + e0[1])) < 1e-2 * abs(e0[0] + e0[1])
    f.close()


def test_barrier_selftest_rejects_bad_limits(mdlg):
    s = _system(mdlg, 1)
    for lim in (0.0, -1.0, 5.0):
        assert s.barrier_selftest(lim) == mdlg.MD_E_ARG
    s.step(10)
    s.sync()
    s.close()


def test_mbarrier_wait_runs_out_and_is_reported(mdlg):
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    A = torch.randn((256, 256), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((128, 256), device="cuda", generator=g).to(torch.bfloat16)
    t0 = time.perf_counter()
    rc = mdlg.bf16_gemm_selftest(A, B, limit_s=0.02)
    assert rc == mdlg.MD_E_TIMEOUT, rc
    assert time.perf_counter() - t0 < 2.0
    # the device is usable and the tensor memory was released
    for _ in range(3):
        Cm, st = mdlg.bf16_gemm_tn(A, B)
        torch.cuda.synchronize()
        assert st.item() == 0
        ref = A.float() @ B.float().T
        assert torch.max(torch.abs(Cm - ref)).item() < 1e-3 * torch.max(torch.abs(ref)).item()
