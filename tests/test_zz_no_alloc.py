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


# Driver-API view of the device's default memory pool, the pool the library's
# stream-ordered allocations come from (attribute values from cuda.h).
_RESERVED_CUR, _USED_CUR, _USED_HIGH = 5, 7, 8


class _Pool:
    def __init__(self):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuCtxGetDevice(C.byref(dev)) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = C.c_uint64(0)  # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_HIGH, C.byref(zero)) == 0

    def free_bytes(self):
        free, total = C.c_size_t(), C.c_size_t()
        assert self.cu.cuMemGetInfo_v2(C.byref(free), C.byref(total)) == 0
        return free.value


def test_allocates_nothing(P):
    """The property the entry point exists for: neither the size query nor the
    fill draws on the device's default memory pool (whose high-water mark
    registers a stream-ordered allocation even after it is freed), and the free
    device memory does not change.  The same check registers the allocating
    psf_sysmat_rows_set (the control)."""
    w = I.workload("RING3D_SMALL")
    ref_ptr, ref_col, _ = P.sysmat_rows_set(w["scanner"], w["image"], w["lors"])
    n = ref_ptr.numel() - 1
    bufs = (torch.empty(n + 1, dtype=torch.int64, device="cuda"),
            torch.empty(ref_col.numel(), dtype=torch.int32, device="cuda"),
            torch.empty(ref_col.numel(), dtype=torch.float32, device="cuda"))
    _noalloc(P, w, bufs)  # warm-up: module load, symbol address look-up
    torch.cuda.synchronize()
    pool = _Pool()
    pool.reset_high()
    high0, res0, free0 = pool.get(_USED_HIGH), pool.get(_RESERVED_CUR), pool.free_bytes()
    _noalloc(P, w, bufs)  # size query + fill
    torch.cuda.synchronize()
    assert pool.get(_USED_HIGH) == high0
    assert pool.get(_RESERVED_CUR) == res0
    assert pool.free_bytes() == free0
    assert torch.equal(bufs[1], ref_col)
    # control: the allocating entry point moves the high-water mark
    pool.reset_high()
    high1 = pool.get(_USED_HIGH)
    P.sysmat_rows_set(w["scanner"], w["image"], w["lors"], buffers=bufs)
    torch.cuda.synchronize()
    assert pool.get(_USED_HIGH) > high1


def _call_size_query(P, w, row_ptr):
    si, ii, li = P.scanner(w["scanner"]), P.image(w["image"]), P.lor_set(w["lors"])
    nnz = C.c_int64(-1)
    rc = P.lib().psf_sysmat_rows_set_noalloc(C.byref(si), C.byref(ii), C.byref(li),
                                              C.c_void_p(row_ptr.data_ptr()), None, None, 0,
                                              C.byref(nnz), None)
    return rc


NOALLOC_MAX_ROWS = 268_417_024  # PSF_NOALLOC_MAX_ROWS in psf.h
ENOSCRATCH = -6


def test_rejects_sets_beyond_the_row_limit(P):
    # 2048 crystals per ring x 256 rings, every pair: far beyond the row limit
    s = I.scanner(64, 32, 16, 16, 2.0, 2.0, 10.0, 0.0, 0.0, 700.0, 0.0, 0.087)
    w = dict(scanner=s, image=I.image(64, 64, 64, 1.0, 1.0, 1.0),
             lors=dict(fan_half=1023, max_ring_diff=255))
    n, _ = P.lor_set_size(w["scanner"], w["lors"])
    assert n > NOALLOC_MAX_ROWS
    row_ptr = torch.full((4,), 7, dtype=torch.int64, device="cuda")
    rc = _call_size_query(P, w, row_ptr)
    assert rc == ENOSCRATCH
    assert "scratch" in P.strerror(rc)
    assert (row_ptr == 7).all()  # nothing was enqueued


def test_rejects_sets_whose_ring_pair_table_overflows(P):
    # few transaxial pairs (4 blocks of 2 crystals, fan 0) but 128 rings with
    # every ring difference: 16,384 ring pairs, whose z-axis table (80 bytes
    # each) alone is larger than the 1 MiB array, while the row count is far
    # below the row limit
    s = I.scanner(4, 2, 16, 8, 2.0, 2.0, 10.0, 0.0, 0.0, 10.0, 0.0, 0.087)
    w = dict(scanner=s, image=I.image(8, 8, 8, 1.0, 1.0, 1.0),
             lors=dict(fan_half=0, max_ring_diff=127))
    n, _ = P.lor_set_size(w["scanner"], w["lors"])
    assert 0 < n <= NOALLOC_MAX_ROWS and 80 * 128 * 128 > (1 << 20)
    row_ptr = torch.full((n + 1,), 7, dtype=torch.int64, device="cuda")
    rc = _call_size_query(P, w, row_ptr)
    assert rc == ENOSCRATCH
    torch.cuda.synchronize()
    assert (row_ptr == 7).all()  # rejected before any device work
