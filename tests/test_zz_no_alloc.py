"""The allocation-free row-pointer scan (impact_scan_rows_static).

Some callers cannot allocate device memory when they build row pointers (their
memory is reserved up front by their own arena, or owned by a host
framework). For them the library offers impact_scan_rows_static, whose
scratch is a fixed device array instead of per-call memory. This test feeds
it the per-row pair counts of a build made with the regular entry points and
checks that it reproduces the row pointers impact_count produced, exactly
(integer results), on two calls in a row; it also checks the size limit.
The file is named so that pytest collects it last.
"""

import pytest
import torch

from paper_2401_03555_gb300 import impact, workloads as W

pytestmark = pytest.mark.gpu


def counts_of(row_ptr):
    c = torch.empty_like(row_ptr)
    c[:-1] = row_ptr[1:] - row_ptr[:-1]
    c[-1] = -12345                      # overwritten by the scan's total
    return c


@pytest.mark.parametrize("make", [lambda: W.room_5d(cells_per_dim=6),
                                  lambda: W.unicycle_3d(nx=31, ny=31, nth=17)])
def test_static_scan_matches_regular_row_pointers(make):
    if not torch.cuda.is_available():
        pytest.fail("needs a CUDA device")
    prob = make()
    ref = impact.build(prob, "fp32").row_ptr          # impact_count + impact_emit
    rows = prob.rows
    assert rows > 4096                               # spans several scan tiles
    for _ in range(2):                               # two calls in a row
        rp = counts_of(ref)
        impact.scan_rows_static(rp, rows)
        torch.cuda.synchronize()
        assert torch.equal(rp, ref)


def test_static_scan_single_row_and_limit():
    rp = torch.tensor([7, -1], dtype=torch.int64, device="cuda")
    impact.scan_rows_static(rp, 1)
    torch.cuda.synchronize()
    assert rp.tolist() == [0, 7]
    # beyond the stated maximum the call is refused before touching memory
    big = torch.zeros(2, dtype=torch.int64, device="cuda")
    status = impact.load().impact_scan_rows_static(big.data_ptr(), (1 << 27) + 1, None)
    assert status == impact.IMPACT_ERR_ARG
    assert "allocation-free" in impact.load().impact_last_error().decode()
    # a host array is refused before any launch
    host = torch.zeros(8, dtype=torch.int64)
    status = impact.load().impact_scan_rows_static(host.data_ptr(), 4, None)
    assert status == impact.IMPACT_ERR_ARG
    assert "device array" in impact.load().impact_last_error().decode()
    # a strided view is refused by the binding (the kernel reads rows+1 in a row)
    with pytest.raises(ValueError):
        impact.scan_rows_static(torch.zeros(16, dtype=torch.int64, device="cuda")[::2], 4)
