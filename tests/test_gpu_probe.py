"""The 64-byte segment read probe (a measurement hook, not part of the method):
argument checks and a clean run on finite data (its one output is written only
for a NaN)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cw():
    import paper_1207_6365_gb300 as cw
    cw.load()
    return cw


def test_probe_runs_and_leaves_out_untouched(cw):
    a = torch.ones(1 << 20, device="cuda")
    out = torch.zeros(1, device="cuda")
    for seq in (False, True):
        for k in (1, 4, 8):
            cw.probe_gather64(a, (1 << 20) // 16 + 1000, seq, k, out)   # wraps past the end by the mask
    cw.probe_gather64(a, 0, False, 4, out)
    torch.cuda.synchronize()
    assert float(out[0]) == 0.0
    a[123] = float("nan")
    cw.probe_gather64(a, 1 << 16, True, 4, out)   # consecutive segments cover element 123
    torch.cuda.synchronize()
    assert out[0].isnan()


def test_probe_rejects_bad_arguments(cw):
    a = torch.ones(48, device="cuda")   # three segments: not a power of two
    with pytest.raises(cw.CWError):
        cw.probe_gather64(a, 3)
    b = torch.ones(64, device="cuda")
    for k in (0, 9):
        with pytest.raises(cw.CWError):
            cw.probe_gather64(b, 4, False, k)
    with pytest.raises(cw.CWError):
        cw.probe_gather64(b, -1)
