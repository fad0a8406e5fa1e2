"""The C-ABI library loads and exports every entry point declared in
include/psf.h; host-side validation rejects bad arguments before any device
work (no GPU needed for these calls)."""
import ctypes as C
import os
import re

import pytest

from paper_1607_06170_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1607_06170_gb300 import build, psf

    build.build()
    return psf


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "psf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(psf_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    lib = C.CDLL(L.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.FUNCTIONS)


def test_strerror_and_sizes(L):
    assert L.strerror(0) == "ok"
    assert "invalid" in L.strerror(-1)
    t = L.table_desc(I.workload("RING3D")["table"])
    a, b = C.c_int64(), C.c_int64()
    assert L.lib().psf_table_size(C.byref(t), C.byref(a), C.byref(b)) == 0
    assert a.value == 32 * 8 * 8 * 8 * 16 * 6 and b.value == 32 * 8 * 8 * 8 * 17


def test_lor_set_sizes_match_the_input_module(L):
    for name in ["RING2D", "RING3D_SMALL", "RING3D"]:
        w = I.workload(name)
        n, k = L.lor_set_size(w["scanner"], w["lors"])
        assert n == I.n_lors(w)
        s = w["scanner"]
        tp = I.transaxial_pairs(s, w["lors"]["fan_half"])
        assert k == int((tp[:, 0] < s["nt_block"]).sum()) * (2 * w["lors"]["max_ring_diff"] + 1)
    assert I.n_lors(I.workload("RING3D")) == 44_732_688


@pytest.mark.parametrize("field,value", [("n_blocks", 2), ("radius", 1.0), ("mu", 0.0),
                                         ("xtal_w_t", -1.0)])
def test_bad_scanner_rejected_on_host(L, field, value):
    s = dict(I.workload("RING2D")["scanner"])
    s[field] = value
    sc, tb = L.scanner(s), L.table_desc(I.workload("RING2D")["table"])
    rc = L.lib().psf_response_build(C.byref(sc), C.byref(tb), C.c_void_p(16), C.c_void_p(16),
                                    None)
    assert rc == -1


def test_table_reach_is_checked(L):
    w = I.workload("RING2D")
    t = dict(w["table"])
    t["max_off_t"] = 8   # the 78.75-degree node reaches 27 crystals
    sc, tb = L.scanner(w["scanner"]), L.table_desc(t)
    rc = L.lib().psf_response_build(C.byref(sc), C.byref(tb), C.c_void_p(16), C.c_void_p(16),
                                    None)
    assert rc == -1


def test_unequal_block_ring_gap_rejected(L):
    s = dict(I.workload("RING3D")["scanner"])
    s["block_gap_a"] = 1.0
    sc, ls = L.scanner(s), L.lor_set(I.workload("RING3D")["lors"])
    n, k = C.c_int64(), C.c_int64()
    assert L.lib().psf_lor_set_size(C.byref(sc), C.byref(ls), C.byref(n), C.byref(k)) == -1
