"""Exact checkpoint and resume through the C-ABI: k steps, save, load into a
fresh system of the same parameters (created from another state), m more
steps must give the bits of k + m steps straight -- positions, velocities,
snapshots, every histogram and overflow on both engines, and the FP64
moment sums too on the global engine.  The resident engine sums a slab's
moment terms in its slot order, which a load resets: there the moments must
agree to 4 ulp."""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _setup(mdlg, prec, R, seed):
    Ns, phis, Ts = inputs.ensemble_params(R, seed=seed, n_min=3000, n_max=20000)
    params, cat = [], [[], [], [], []]
    for r in range(R):
        L = inputs.box_length(int(Ns[r]), float(phis[r]))
        st = inputs.lattice_gas_state(int(Ns[r]), L, float(Ts[r]), seed=300 + r)
        params.append(mdlg.make_params(int(Ns[r]), L, precision=prec, W=4, lg_every=(150, 400),
                                       lx=(int(round(L)), int(round(L / 2))), skin=0.4))
        for a, f in zip(cat, ("x", "y", "vx", "vy")):
            a.append(getattr(st, f))
    return params, [np.concatenate(a) for a in cat]


def _observe(mdlg, s, params):
    R = len(params)
    return {"state": s.get_state(),
            "snap": [[t.cpu().numpy() for t in s.get_snapshot(k)] for k in range(2)],
            "hist": [[[s.hist_raw(r, k, d) for d in range(2)] for k in range(2)] for r in range(R)],
            "feq": [[s.feq_measured(r, k, 0)[2] for k in range(2)] for r in range(R)],
            "step": s.info().step}


def _eq(a, b, mom_ulps=0):
    assert a["step"] == b["step"]
    for u, v in zip(a["state"], b["state"]):
        assert np.array_equal(u, v)
    for k in range(2):
        for u, v in zip(a["snap"][k], b["snap"][k]):
            assert np.array_equal(u, v)
    for ha, hb in zip(a["hist"], b["hist"]):
        for k in range(2):
            for d in range(2):
                assert np.array_equal(ha[k][d][0], hb[k][d][0]) and ha[k][d][1:] == hb[k][d][1:]
    for fa, fb in zip(a["feq"], b["feq"]):
        for k in range(2):
            assert fa[k].n_windows == fb[k].n_windows
            for x, y in ((fa[k].mu2, fb[k].mu2), (fa[k].mu4, fb[k].mu4)):
                assert abs(x - y) <= mom_ulps * np.spacing(abs(y)), (x, y)


@pytest.mark.parametrize("prec,engine", [(0, "global"), (1, "global"), (1, "resident")])
def test_checkpoint_resume_is_exact(mdlg, prec, engine):
    params, cat = _setup(mdlg, prec, 4, seed=5)
    shape = (0, 0, 4) if engine == "resident" else (256, 1, 3)
    a = mdlg.System(params, *cat)
    a.tune(*shape)
    a.step(1000)
    a.step(1000)
    ref = _observe(mdlg, a, params)
    a.close()
    b = mdlg.System(params, *cat)
    b.tune(*shape)
    b.step(1000)
    ck = b.checkpoint()
    b.close()
    # a fresh system from another state takes the checkpoint
    other = [c[::-1].copy() for c in cat]
    c = mdlg.System(params, *other)
    c.tune(*shape)
    c.restore(ck)
    c.step(1000)
    _eq(ref, _observe(mdlg, c, params), mom_ulps=4 if engine == "resident" else 0)
    c.close()


def test_checkpoint_rejects_other_parameters(mdlg):
    params, cat = _setup(mdlg, 1, 2, seed=6)
    a = mdlg.System(params, *cat)
    a.step(10)
    ck = a.checkpoint()
    a.close()
    p2, c2 = _setup(mdlg, 1, 3, seed=6)
    b = mdlg.System(p2, *c2)
    with pytest.raises(mdlg.MDError):
        b.restore(ck)
    bad = ck.copy()
    bad[:8] = 0
    with pytest.raises(mdlg.MDError):
        b.restore(bad)
    b.close()
