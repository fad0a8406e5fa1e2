"""psf_sysmat_rows_set_noalloc: the row generator for callers that may not
allocate device memory (a fixed device budget reserved at start-up, or no
tolerance for the device synchronisation an allocation implies).  Its scratch
is a fixed device array inside the library, so it must give exactly the rows
of psf_sysmat_rows_set, on repeated calls, and refuse sets that do not fit.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test; it must also pass on its own in a
fresh process."""
import ctypes as C

import pytest
import torch

from paper_1607_06170_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1607_06170_gb300 import build, psf

    build.build()
    assert torch.cuda.is_available()
    return psf


def _noalloc(P, w, buffers):
    """Size query then fill, through the C ABI of the no-allocation entry point."""
    s, i, l = P.scanner(w["scanner"]), P.image(w["image"]), P.lor_set(w["lors"])
    row_ptr, col, val = buffers
    nnz = C.c_int64()
    L = P.lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.psf_sysmat_rows_set_noalloc(C.byref(s), C.byref(i), C.byref(l),
                                        C.c_void_p(row_ptr.data_ptr()), None, None, 0,
                                        C.byref(nnz), st)
    assert rc == 0, P.strerror(rc)
    assert nnz.value <= col.numel()
    rc = L.psf_sysmat_rows_set_noalloc(C.byref(s), C.byref(i), C.byref(l),
                                        C.c_void_p(row_ptr.data_ptr()),
                                        C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()),
                                        col.numel(), C.byref(nnz), st)
    assert rc == 0, P.strerror(rc)
    torch.cuda.synchronize()
    return nnz.value


@pytest.mark.parametrize("name", ["RING3D_SMALL", "RING3D"])
def test_matches_allocating_entry_point_twice(P, name):
    w = I.workload(name)
    ref_ptr, ref_col, ref_val = P.sysmat_rows_set(w["scanner"], w["image"], w["lors"])
    torch.cuda.synchronize()
    n = ref_ptr.numel() - 1
    bufs = (torch.full((n + 1,), -1, dtype=torch.int64, device="cuda"),
            torch.zeros(ref_col.numel(), dtype=torch.int32, device="cuda"),
            torch.zeros(ref_val.numel(), dtype=torch.float32, device="cuda"))
    for _ in range(2):  # the shared array keeps the previous call's contents
        nnz = _noalloc(P, w, bufs)
        assert nnz == ref_col.numel()
        assert torch.equal(bufs[0], ref_ptr)
        assert torch.equal(bufs[1], ref_col)
        torch.testing.assert_close(bufs[2], ref_val, rtol=0, atol=0)
        bufs[1].zero_()
        bufs[2].zero_()


def test_rejects_sets_beyond_the_scratch(P):
    # 2048 crystals per ring x 256 rings, every pair: far beyond the fixed scratch
    s = I.scanner(64, 32, 16, 16, 2.0, 2.0, 10.0, 0.0, 0.0, 700.0, 0.0, 0.087)
    w = dict(scanner=s, image=I.image(64, 64, 64, 1.0, 1.0, 1.0),
             lors=dict(fan_half=1023, max_ring_diff=255))
    n, _ = P.lor_set_size(w["scanner"], w["lors"])
    assert n > ((1 << 20) - 64) // 8 * 2048  # PSF_NOALLOC_MAX_ROWS
    si, ii, li = P.scanner(s), P.image(w["image"]), P.lor_set(w["lors"])
    nnz = C.c_int64(-1)
    row_ptr = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = P.lib().psf_sysmat_rows_set_noalloc(C.byref(si), C.byref(ii), C.byref(li),
                                              C.c_void_p(row_ptr.data_ptr()), None, None, 0,
                                              C.byref(nnz), None)
    assert rc == -6
    assert "scratch" in P.strerror(rc)
