"""The shared-memory-resident engine (md_tune staging 4) against the global
engine and the oracle, through the C-ABI.

The resident engine keeps one rebuild bound per replica; the global engine
keeps one for its whole batch, which for a batch of one replica is the same
rule.  Both sum every force over the same pairs in the same order with the
same arithmetic, so each replica of a resident batch must follow, bit for
bit, the trajectory the global engine gives that replica alone (positions,
velocities, snapshots, integer histograms), whatever the slab plan and the
splitting of md_step calls.  Only the FP64 moment sums are grouped
differently: they must agree to 1e-12 relative.  The global engine itself
is checked against the oracle elsewhere; the resident engine's own list
forces are also checked against the oracle here.
"""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs
import _bars

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _batch(mdlg, spec, seed0, lg_every=(100, 250), dx=(1.0, 2.0), skin=0.4):
    params, cat = [], [[], [], [], []]
    for r, (n, phi, T) in enumerate(spec):
        L = inputs.box_length(n, phi)
        st = inputs.lattice_gas_state(n, L, T, seed=seed0 + r)
        params.append(mdlg.make_params(n, L, precision=mdlg.MD_FP32_CELLOFF, W=4, lg_every=lg_every,
                                       lx=tuple(int(round(L / d)) for d in dx), skin=skin))
        for a, f in zip(cat, ("x", "y", "vx", "vy")):
            a.append(getattr(st, f))
    return params, [np.concatenate(a) for a in cat]


def _run(mdlg, params, cat, engine, chunks):
    s = mdlg.System(params, *cat)
    if engine == "resident":
        s.tune(0, 0, 4)
    else:
        s.tune(256, 1, 3)
    for c in chunks:
        s.step(c)
    R = len(params)
    out = {"state": s.get_state(), "snap": [[t.cpu().numpy() for t in s.get_snapshot(k)] for k in range(2)]}
    out["hist"] = [[[s.hist_raw(r, k, d) for d in range(2)] for k in range(2)] for r in range(R)]
    out["mom"] = [[_bars.moment_sums(s, r, k, params[r].n) for k in range(2)] for r in range(R)]
    s.close()
    return out


def _alone(mdlg, params, cat, chunks):
    """Each replica run alone on the global engine, results concatenated in
    replica order."""
    base = np.concatenate([[0], np.cumsum([p.n for p in params])])
    outs = []
    for r, p in enumerate(params):
        sl = slice(base[r], base[r + 1])
        outs.append(_run(mdlg, [p], [a[sl] for a in cat], "global", chunks))
    return {"state": [np.concatenate([o["state"][q] for o in outs]) for q in range(4)],
            "snap": [[np.concatenate([o["snap"][k][q] for o in outs]) for q in range(3)] for k in range(2)],
            "hist": [o["hist"][0] for o in outs], "mom": [o["mom"][0] for o in outs]}


def _same(a, b):
    for u, v in zip(a["state"], b["state"]):
        assert np.array_equal(u, v)
    for k in range(2):
        for u, v in zip(a["snap"][k], b["snap"][k]):
            assert np.array_equal(u, v)
    for ha, hb in zip(a["hist"], b["hist"]):
        for k in range(2):
            for d in range(2):
                assert np.array_equal(ha[k][d][0], hb[k][d][0]) and ha[k][d][1:] == hb[k][d][1:]
    for ma, mb in zip(a["mom"], b["mom"]):
        for k in range(2):
            assert np.all(np.abs(ma[k] - mb[k]) <= 1e-12 * np.abs(mb[k]))


@pytest.mark.parametrize("spec", [
    [(5000, 0.2, 5.0)],                        # one slab
    [(60000, 0.25, 8.0)],                      # one replica over many slabs
])
def test_resident_equals_global_engine_single_replica(mdlg, spec):
    params, cat = _batch(mdlg, spec, seed0=70)
    a = _run(mdlg, params, cat, "global", (800,))
    b = _run(mdlg, params, cat, "resident", (300, 1, 499))
    _same(a, b)


@pytest.mark.parametrize("R,seed", [(3, 21), (16, 11)])
def test_resident_batch_equals_replicas_alone(mdlg, R, seed):
    """R replicas of the bench's draw recipe (16: about 360k particles) on
    the resident engine against each replica alone on the global engine."""
    Ns, phis, Ts = inputs.ensemble_params(R, seed=seed)
    spec = [(int(n), float(p), float(t)) for n, p, t in zip(Ns, phis, Ts)]
    params, cat = _batch(mdlg, spec, seed0=900)
    a = _alone(mdlg, params, cat, (1000,))
    b = _run(mdlg, params, cat, "resident", (600, 400))
    _same(a, b)


def test_resident_list_forces_match_oracle(mdlg, orc):
    """The resident engine's own force pass at consecutive steps across a
    rebuild, one replica over several slabs, against the oracle (FP32 bar,
    allowances of _bars.py)."""
    n, phi, T = 30_000, 0.25, 5.0
    L = inputs.box_length(n, phi)
    st = inputs.lattice_gas_state(n, L, T, seed=31)
    p = mdlg.make_params(n, L, precision=mdlg.MD_FP32_CELLOFF, lg_every=(100,), lx=(int(round(L)),), skin=0.4)
    s = mdlg.System(p, st.x, st.y, st.vx, st.vy)
    s.tune(0, 0, 4)
    s.step(200)
    info = s.rep_info(0)
    nc, h, Le = int(info.ncell), float(info.h), float(info.L_eff)
    r0 = s.info().n_rebuilds
    worst = 0.0
    for _ in range(60):
        cell, ox, oy = (t.cpu().numpy() for t in s.get_raw())
        gx, gy = s.step_forces(1)
        x, y = _bars.decode(cell, ox, oy, nc, h)
        ofx, ofy, _, ofa = orc.forces_cells(x, y, Le)
        allow = _bars.force_allowance(x, y, Le, h, True)
        worst = max(worst, _bars.force_ratio(gx, gy, ofx, ofy, ofa, allow, 1e-5))
    assert worst <= 1.0, worst
    assert s.info().n_rebuilds - r0 >= 1
    s.close()


def test_resident_rejects_fp64(mdlg):
    L = inputs.box_length(2000, 0.1)
    st = inputs.lattice_gas_state(2000, L, 5.0, seed=1)
    s = mdlg.System(mdlg.make_params(2000, L, precision=mdlg.MD_FP64), st.x, st.y, st.vx, st.vy)
    with pytest.raises(mdlg.MDError):
        s.tune(0, 0, 4)
    s.close()
