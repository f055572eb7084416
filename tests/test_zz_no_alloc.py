"""The allocation-free contraction table (tgba_table_noalloc) against the regular one.

Some callers cannot let a library allocate device memory: a process whose device memory is
handed out by a fixed-size pool that refuses allocations made behind its back, or a
latency-critical loop that cannot afford the implicit device synchronisation of cudaMalloc
and cudaFree.  tgba_table_noalloc serves them from a statically sized work area instead.  This
test checks that it returns the same table and vacuum element as tgba_table, on two calls in a
row (the work area keeps the previous call's contents), for two chain lengths and fields.
It lives in a file of its own, collected last.
"""
import numpy as np
import pytest
import torch

from paper_2410_04204_gb300 import tgba

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def noalloc(L, h):
    table = torch.empty(4 * L * L, dtype=torch.float64, device="cuda")
    c0 = torch.empty(2, dtype=torch.float64, device="cuda")
    tgba.tgba_table_noalloc(L, h, table, c0)          # through the C ABI
    torch.cuda.synchronize()
    return table.cpu().numpy(), complex(*c0.cpu().numpy())


def reference(L, h):
    b = tgba.tgba_build_basis(L, h, [0], 2)
    try:
        table = torch.empty(4 * L * L, dtype=torch.float64, device="cuda")
        c0 = tgba.tgba_table(b, table)
        return table.cpu().numpy(), c0
    finally:
        tgba.tgba_basis_free(b)


@pytest.mark.parametrize("L,h", [(24, 1.0), (40, 0.7), (64, 1.0)])
def test_noalloc_table_matches_regular_entry_point(L, h):
    """L = 64 is the size limit: there the work matrix fills the static array exactly."""
    want_t, want_c0 = reference(L, h)
    for _ in range(2):
        got_t, got_c0 = noalloc(L, h)
        assert np.abs(got_t - want_t).max() <= 1e-10 * np.abs(want_t).max()
        assert abs(got_c0 - want_c0) <= 1e-10 * abs(want_c0)


def test_noalloc_calls_take_no_device_memory():
    """After a first call (which may load the library's device code, static arrays included),
    repeated calls leave the device's free memory and torch's allocator unchanged."""
    L = 64
    table = torch.empty(4 * L * L, dtype=torch.float64, device="cuda")
    c0 = torch.empty(2, dtype=torch.float64, device="cuda")
    tgba.tgba_table_noalloc(L, 1.0, table, c0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for h in (0.5, 1.0, 1.5):
        tgba.tgba_table_noalloc(L, h, table, c0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_chains_beyond_its_work_area():
    with pytest.raises(tgba.TgbaError) as e:
        tgba.tgba_table_noalloc(66, 1.0, torch.empty(4 * 66 * 66, dtype=torch.float64, device="cuda"),
                                torch.empty(2, dtype=torch.float64, device="cuda"))
    assert e.value.code == tgba.TGBA_ELIMIT
