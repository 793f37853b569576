"""Host-side argument checks of the Python binding (no GPU): snapshot
arrays and fields go to the C ABI as bare pointers, so the binding refuses
mismatched lengths, dtypes, shapes and devices before any library call."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2101_01160_gb300 import mdlg  # noqa: E402


def _snap(n=8, cell=torch.int32, off=torch.float32):
    return [torch.zeros(n, dtype=cell), torch.zeros(n, dtype=off), torch.zeros(n, dtype=off)]


@pytest.mark.parametrize("fn,extra", [(mdlg.mdlg_bin, (4, 2)), (mdlg.disp_hist, (0.1, 16)),
                                      (mdlg.site_occupation, (4, 2))])
def test_snapshot_checks(fn, extra):
    a, b = _snap(), _snap()
    with pytest.raises(ValueError, match="one length"):
        fn(*a, *_snap(9), 3, 1.0, *extra)
    with pytest.raises(ValueError, match="int32"):
        fn(*_snap(cell=torch.int64), *b, 3, 1.0, *extra)
    with pytest.raises(ValueError, match="float32 or all float64"):
        fn(*a, *_snap(off=torch.float64), 3, 1.0, *extra)
    with pytest.raises(ValueError, match="float32 or all float64"):
        fn(*_snap(off=torch.float16), *_snap(off=torch.float16), 3, 1.0, *extra)
    with pytest.raises(ValueError, match="torch tensors"):
        fn(*[np.zeros(8, np.int32), np.zeros(8, np.float32), np.zeros(8, np.float32)], *b, 3, 1.0, *extra)
    with pytest.raises(ValueError, match="contiguous"):
        fn(torch.zeros((2, 4), dtype=torch.int32), *a[1:], *b, 3, 1.0, *extra)
    # well-formed but on the host: refused too
    with pytest.raises(ValueError, match="CUDA"):
        fn(*a, *b, 3, 1.0, *extra)


def test_field_checks():
    a, b = _snap(), _snap()
    with pytest.raises(ValueError, match="MD_MAX_W"):
        mdlg.site_occupation(*a, *b, 3, 1.0, 4, 11)
    with pytest.raises(ValueError, match="2\\^31"):
        mdlg.site_occupation(*a, *b, 3, 1.0, 20_000, 10)
    n = torch.zeros((9, 3, 3), dtype=torch.int32)
    with pytest.raises(ValueError, match="shape"):
        mdlg.collision(n, n, 2)                      # 25 classes expected
    with pytest.raises(ValueError, match="shape"):
        mdlg.collision(n, torch.zeros((9, 3, 4), dtype=torch.int32), 1)
    with pytest.raises(ValueError, match="int32"):
        mdlg.collision(n, n.to(torch.int64), 1)
    with pytest.raises(ValueError, match="CUDA"):
        mdlg.collision(n, n, 1)


def test_set_state_checks():
    """md_set_state reads n_total FP64 values per array from host or device
    memory, so the binding refuses shorter host arrays and non-FP64,
    non-contiguous or mis-sized device tensors before the call."""
    import types

    fake = types.SimpleNamespace(n_total=8, h=None)
    ok = [np.zeros(8) for _ in range(4)]
    with pytest.raises(ValueError, match="hold 8 values"):
        mdlg.System.set_state(fake, np.zeros(7), *ok[1:])
    if torch.cuda.is_available():
        dev = [torch.zeros(8, dtype=torch.float64, device="cuda") for _ in range(4)]
        with pytest.raises(ValueError, match="float64 of 8"):
            mdlg.System.set_state(fake, dev[0].float(), *dev[1:])
        with pytest.raises(ValueError, match="float64 of 8"):
            mdlg.System.set_state(fake, torch.zeros(16, dtype=torch.float64, device="cuda")[::2], *dev[1:])
