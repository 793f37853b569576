"""mdlg_bin_noalloc, the binning entry point for callers that cannot
allocate device memory while they run (memory owned by a framework's caching
allocator or a fixed budget, or a loop that must not stall on allocator
calls), against mdlg_bin on the same inputs: two calls in a row with
different sizes, so that partials left in the shared scratch array by the
first call would show in the second.  Named to be collected last; it also
passes on its own."""

import numpy as np
import pytest

from paper_2101_01160_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _snap(n, seed, f64):
    ncell, h = 33, 101.283 / 33
    if not f64:
        h = float(np.float32(h))
    s = inputs.random_celloff_snapshots(n, ncell, h, seed=seed, max_step=6.0, f64=f64,
                                        ties=min(n, 300), lattice_dx=ncell * h / 101)
    return [torch.from_numpy(s[k]).cuda() for k in ("cell0", "ox0", "oy0", "cell1", "ox1", "oy1")], ncell, h


@pytest.mark.parametrize("f64", [False, True])
def test_noalloc_matches_mdlg_bin_twice(mdlg, f64):
    cases = [(262_147, 11), (1_000, 12)]          # many CTAs, then few
    outs = []
    for n, seed in cases:
        arrs, ncell, h = _snap(n, seed, f64)
        outs.append((arrs, ncell, h, mdlg.mdlg_bin(*arrs, ncell, h, 101, 4, noalloc=True)))
    for arrs, ncell, h, (hist, ovf, mom) in outs:
        rh, ro, rm = mdlg.mdlg_bin(*arrs, ncell, h, 101, 4)
        torch.cuda.synchronize()
        assert torch.equal(hist, rh)
        assert torch.equal(ovf, ro)
        assert torch.equal(mom, rm)           # same grid, same summation order: identical bits


def test_noalloc_rejects_bad_args(mdlg):
    c = torch.zeros(4, dtype=torch.int32, device="cuda")
    o = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(mdlg.MDError):
        mdlg.mdlg_bin(c, o, o, c, o, o, 10, 1.0, 10, 11, noalloc=True)   # W > MD_MAX_W
