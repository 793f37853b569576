"""Block-bootstrap error bars of the measured equilibrium on the GPU
(feq_bootstrap) against the oracle on the same block histograms (the same
definition and draws, rounded operation by operation: equal bits), and
against the spread of P over independent replicas (statistics)."""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ensemble(mdlg, R, n, seed, block_windows=1, windows=24):
    L = inputs.box_length(n, 0.0784)
    states = [inputs.lattice_gas_state(n, L, 20.0, seed=seed + r) for r in range(R)]
    cat = [np.concatenate([getattr(st, f) for st in states]) for f in ("x", "y", "vx", "vy")]
    p = mdlg.make_params(n, L, precision=mdlg.MD_FP32_CELLOFF, W=4, n_equil=2000, lg_every=(400, 200),
                         lx=(int(round(L)),), block_windows=block_windows)
    s = mdlg.System([p] * R, *cat)
    s.step(2000 + windows * 400)
    return s, p


@pytest.mark.parametrize("block_windows,sym", [(1, False), (2, True)])
def test_bootstrap_matches_oracle(mdlg, orc, block_windows, sym):
    s, p = _ensemble(mdlg, 6, 4096, seed=40, block_windows=block_windows, windows=40)
    for lg in (0, 1):
        sig = mdlg.feq_bootstrap(s, lg, 0, symmetrize=sym, n_resamples=300, seed=77)
        for r in range(6):
            h, w = mdlg.hist_blocks(s, r, lg, 0)
            ref = orc.bootstrap_feq(h.astype(np.int64), w, 4, float(p.n), sym=sym, B=300, seed=77, rep=r)
            assert np.array_equal(sig[r], ref), (lg, r, np.max(np.abs(sig[r] - ref)))
            assert w.sum() == s.hist_raw(r, lg, 0)[2]
    s.close()


def test_bootstrap_agrees_with_replica_spread(mdlg):
    """64 replicas of one (phi, T): the standard deviation of each replica's
    P0 over the replicas is the statistical error of one replica, which the
    bootstrap over that replica's windows estimates."""
    R = 64
    # blocks of 16 windows (3.2 tau): windows are correlated over a few mean
    # free times at phi = 0.0784, T = 20 (blocks of 4 windows, 0.8 tau,
    # understated the spread by a factor of 1.8), so blocks must be longer
    s, p = _ensemble(mdlg, R, 4096, seed=70, block_windows=16, windows=512)
    c0 = 40
    P0 = np.array([s.feq_measured(r, 0, 0)[0][c0] for r in range(R)])
    sig = mdlg.feq_bootstrap(s, 0, 0, n_resamples=400, seed=3)[:, c0]
    ratio = P0.std(ddof=1) / np.sqrt(np.mean(sig ** 2))
    # the replica spread itself carries a relative error of about 1/sqrt(2 (R-1))
    assert 0.65 < ratio < 1.5, ratio
    s.close()
