"""Thin ctypes binding of libpsf.so (the C ABI declared in include/psf.h).

Argument marshalling only: tensors are passed as device pointers together
with torch's current CUDA stream; every step of the computation runs in the
library's kernels.  There is no fallback: if the library is missing or the
process has no GPU the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpsf.so")

PSF_F32, PSF_BF16, PSF_F16 = 0, 1, 2
NORM_NONE, NORM_EFF, NORM_UNIT = 0, 1, 2
_DT = {"f32": PSF_F32, "bf16": PSF_BF16, "f16": PSF_F16}
_TORCH_DT = {PSF_F32: torch.float32, PSF_BF16: torch.bfloat16, PSF_F16: torch.float16}

FUNCTIONS = [
    "psf_strerror", "psf_table_size", "psf_response_build", "psf_bin_spread",
    "psf_lor_set_size", "psf_lor_set_list", "psf_lor_set_classes", "psf_sysmat_rows",
    "psf_sysmat_rows_set", "psf_sysmat_rows_set_noalloc", "psf_sysmat_rows_set_typed",
    "psf_matrix_create", "psf_matrix_set_spread", "psf_matrix_destroy", "psf_forward",
    "psf_back", "psf_em_ratio", "psf_em_update", "psf_timing_enable", "psf_timing_read",
    "psf_matrix_autotune", "psf_matrix_set_launch", "psf_sensitivity", "psf_back_sens",
    "psf_spread_topn", "psf_matrix_set_spread_topn", "psf_event_rows", "psf_histogram",
    "psf_forward_masked", "psf_sino_bins", "psf_voxel_homog", "psf_matrix_set_stencil_form",
    "psf_matrix_check", "psf_matrix_build_sparse_adjoint", "psf_bin_spread_classes",
    "psf_set_wait_limit", "psf_matrix_create_otf", "psf_matrix_set_image",
    "psf_spread_topn_bf16", "psf_matrix_set_spread_topn_bf16",
]


class PSFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class Scanner(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("nt_block", C.c_int32), ("na_block", C.c_int32),
                ("n_block_rings", C.c_int32), ("xtal_w_t", C.c_double), ("xtal_w_a", C.c_double),
                ("depth", C.c_double), ("gap_t", C.c_double), ("gap_a", C.c_double),
                ("radius", C.c_double), ("block_gap_a", C.c_double), ("mu", C.c_double)]


class TableDesc(C.Structure):
    _fields_ = [("n_ang_t", C.c_int32), ("n_ang_a", C.c_int32), ("n_sub_t", C.c_int32),
                ("n_sub_a", C.c_int32), ("max_off_t", C.c_int32), ("max_off_a", C.c_int32),
                ("ang_max_t_deg", C.c_double), ("ang_max_a_deg", C.c_double)]


class Image(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("reserved", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class LorSet(C.Structure):
    _fields_ = [("fan_half", C.c_int32), ("max_ring_diff", C.c_int32)]


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_SIGS = {
    "psf_strerror": (C.c_char_p, [C.c_int]),
    "psf_table_size": (C.c_int, [_P, _P, _P]),
    "psf_response_build": (C.c_int, [_P, _P, _P, _P, _P]),
    "psf_bin_spread": (C.c_int, [_P, _P, _P, _P, _P, _I64, _I32, _I32, _I32, _P, _P]),
    "psf_bin_spread_classes": (C.c_int, [_P, _P, _P, _P, _P, _P, _I32, _I32, _I32, _P, _P]),
    "psf_lor_set_size": (C.c_int, [_P, _P, _P, _P]),
    "psf_lor_set_list": (C.c_int, [_P, _P, _P, _P]),
    "psf_lor_set_classes": (C.c_int, [_P, _P, _P, _P]),
    "psf_sysmat_rows": (C.c_int, [_P, _P, _P, _I64, _P, _I32, _I32, _I32, _P, _P, _P, _P, _I64,
                                  _P, _P]),
    "psf_sysmat_rows_set": (C.c_int, [_P, _P, _P, _P, _P, _P, _I64, _P, _P]),
    "psf_sysmat_rows_set_noalloc": (C.c_int, [_P, _P, _P, _P, _P, _P, _I64, _P, _P]),
    "psf_sysmat_rows_set_typed": (C.c_int, [_P, _P, _P, _I32, _P, _P, _P, _P, _I64, _P, _P]),
    "psf_matrix_create": (C.c_int, [_P, _I64, _I64, _P, _P, _P, _I32, _P, _P]),
    "psf_matrix_set_spread": (C.c_int, [_P, _P, _P, _I32, _I32, _P]),
    "psf_matrix_destroy": (C.c_int, [_P]),
    "psf_forward": (C.c_int, [_P, _P, _P, _P]),
    "psf_back": (C.c_int, [_P, _P, _P, _P]),
    "psf_em_ratio": (C.c_int, [_P, _P, _P, _I64, _P]),
    "psf_em_update": (C.c_int, [_P, _P, _P, C.c_float, _I64, _P]),
    "psf_timing_enable": (C.c_int, [_I32]),
    "psf_timing_read": (C.c_int, [_I32, _P, _P, _P]),
    "psf_matrix_autotune": (C.c_int, [_P, _P, _P, _P]),
    "psf_matrix_set_launch": (C.c_int, [_P, _I32, _I32]),
    "psf_sensitivity": (C.c_int, [_P, _P, _P]),
    "psf_back_sens": (C.c_int, [_P, _P, _P, _P, _P]),
    "psf_spread_topn": (C.c_int, [_P, _I64, _I32, _I32, _I32, _P, _P, _P]),
    "psf_matrix_set_spread_topn": (C.c_int, [_P, _P, _P, _I32, _I32, _I32, _P, _P]),
    "psf_event_rows": (C.c_int, [_P, _P, _P, _I64, _P, _P]),
    "psf_histogram": (C.c_int, [_P, _I64, C.c_float, _P, _I64, _P]),
    "psf_forward_masked": (C.c_int, [_P, _P, _P, _P, _P]),
    "psf_sino_bins": (C.c_int, [_P, _P, _P, _P, _P]),
    "psf_voxel_homog": (C.c_int, [_P, _P, _P, _P, _P, _P, _I32, _I32, _P, _P]),
    "psf_matrix_set_stencil_form": (C.c_int, [_P, _I32]),
    "psf_matrix_set_image": (C.c_int, [_P, _P]),
    "psf_spread_topn_bf16": (C.c_int, [_P, _I64, _I32, _P, _P, _P]),
    "psf_matrix_set_spread_topn_bf16": (C.c_int, [_P, _P, _P, _I32, _I32, _I32, _P, _P, _P]),
    "psf_matrix_check": (C.c_int, [_P, _P]),
    "psf_set_wait_limit": (C.c_int, [_I64]),
    "psf_matrix_build_sparse_adjoint": (C.c_int, [_P, _P]),
    "psf_matrix_create_otf": (C.c_int, [_P, _P, _P, _P, _P]),
}

_lock = threading.Lock()
_lib = None


def lib() -> C.CDLL:
    """Load libpsf.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().psf_strerror(int(code)).decode()


def timing_enable(on: bool = True):
    """Clear the kernel-time accumulators and switch event timing on or off."""
    _ok(lib().psf_timing_enable(1 if on else 0), "psf_timing_enable")


def timing_read() -> dict:
    """{kernel name: (launches, total ms)} accumulated since timing_enable()."""
    out = {}
    name, n, ms = C.c_char_p(), C.c_int64(), C.c_double()
    i = 0
    while lib().psf_timing_read(i, C.byref(name), C.byref(n), C.byref(ms)) == 0:
        out[name.value.decode()] = (n.value, ms.value)
        i += 1
    return out


def _ok(rc: int, where: str):
    if rc != 0:
        raise PSFError(rc, where)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def scanner(d: dict) -> Scanner:
    return Scanner(int(d["n_blocks"]), int(d["nt_block"]), int(d["na_block"]),
                   int(d["n_block_rings"]), float(d["xtal_w_t"]), float(d["xtal_w_a"]),
                   float(d["depth"]), float(d["gap_t"]), float(d["gap_a"]), float(d["radius"]),
                   float(d["block_gap_a"]), float(d["mu"]))


def table_desc(d: dict) -> TableDesc:
    return TableDesc(int(d["n_ang_t"]), int(d["n_ang_a"]), int(d["n_sub_t"]), int(d["n_sub_a"]),
                     int(d["max_off_t"]), int(d["max_off_a"]), float(d["ang_max_t_deg"]),
                     float(d["ang_max_a_deg"]))


def image(d: dict) -> Image:
    return Image(int(d["nx"]), int(d["ny"]), int(d["nz"]), 0, float(d["dx"]), float(d["dy"]),
                 float(d["dz"]), float(d["ox"]), float(d["oy"]), float(d["oz"]))


def lor_set(d: dict) -> LorSet:
    return LorSet(int(d["fan_half"]), int(d["max_ring_diff"]))


# ------------------------------------------------------------------ calls
def response_build(sc: dict, tb: dict, device="cuda"):
    """P-SPIR table (float32) and FP64 counting-rate prefix sums."""
    s, t = scanner(sc), table_desc(tb)
    shp = (t.n_ang_t, t.n_ang_a, t.n_sub_t, t.n_sub_a)
    T = torch.empty(shp + (t.max_off_t, t.max_off_a), dtype=torch.float32, device=device)
    eta = torch.empty(shp + (t.max_off_t + 1,), dtype=torch.float64, device=device)
    _ok(lib().psf_response_build(C.byref(s), C.byref(t), _ptr(T), _ptr(eta), _stream()),
        "psf_response_build")
    return T, eta


def bin_spread(sc: dict, tb: dict, T, eta, lors, half_t: int, half_a: int,
               norm: int = NORM_EFF, out=None):
    """Homogenization spread [n, E, E] of each LOR (int32 [n, 2] crystal ids)."""
    s, t = scanner(sc), table_desc(tb)
    n = lors.shape[0]
    E = (2 * half_t + 1) * (2 * half_a + 1)
    if out is None:
        out = torch.empty((n, E, E), dtype=torch.float32, device=lors.device)
    _ok(lib().psf_bin_spread(C.byref(s), C.byref(t), _ptr(T), _ptr(eta), _ptr(lors), n,
                             half_t, half_a, norm, _ptr(out), _stream()), "psf_bin_spread")
    return out


def bin_spread_classes(sc: dict, tb: dict, T, eta, ls: dict, class_lors, half_t: int,
                       half_a: int, norm: int = NORM_EFF, out=None):
    """Spreads [n_classes, E, E] of every class of a structured set (class_lors
    from lor_set_classes): ring differences d >= 0 computed, d < 0 as their
    axial mirrors (psf_bin_spread_classes)."""
    s, t, l = scanner(sc), table_desc(tb), lor_set(ls)
    n = class_lors.shape[0]
    E = (2 * half_t + 1) * (2 * half_a + 1)
    if out is None:
        out = torch.empty((n, E, E), dtype=torch.float32, device=class_lors.device)
    _ok(lib().psf_bin_spread_classes(C.byref(s), C.byref(t), _ptr(T), _ptr(eta), C.byref(l),
                                     _ptr(class_lors), half_t, half_a, norm, _ptr(out),
                                     _stream()), "psf_bin_spread_classes")
    return out


def set_wait_limit(cycles: int):
    """Cycle limit of the library's bounded device waits (psf_set_wait_limit);
    negative: give up at once (tests of the timeout path)."""
    _ok(lib().psf_set_wait_limit(int(cycles)), "psf_set_wait_limit")


WAIT_LIMIT_DEFAULT = 1 << 31


def spread_topn(spread, half_t: int, half_a: int, n_keep: int):
    """Top-N truncation of spreads [n, E, E] (psf_spread_topn): kept window
    indices int32 [n, n_keep] in rank order and their rescaled weights."""
    n = spread.shape[0]
    idx = torch.empty((n, n_keep), dtype=torch.int32, device=spread.device)
    w = torch.empty((n, n_keep), dtype=torch.float32, device=spread.device)
    _ok(lib().psf_spread_topn(_ptr(spread), n, half_t, half_a, n_keep, _ptr(idx), _ptr(w),
                              _stream()), "psf_spread_topn")
    return idx, w


def spread_topn_bf16(w):
    """Top-N weights [n, N] (FP32) as BF16 codes with one FP32 scale per row
    (psf_spread_topn_bf16): weight = code x scale."""
    n, N = w.shape
    w16 = torch.empty((n, N), dtype=torch.bfloat16, device=w.device)
    scale = torch.empty(n, dtype=torch.float32, device=w.device)
    _ok(lib().psf_spread_topn_bf16(_ptr(w), n, N, _ptr(w16), _ptr(scale), _stream()),
        "psf_spread_topn_bf16")
    return w16, scale


def event_rows(sc: dict, ls: dict, events):
    """Row of each event (int32 [n, 2] crystal ids) in the set, -1 outside."""
    s, l = scanner(sc), lor_set(ls)
    rows = torch.empty(events.shape[0], dtype=torch.int64, device=events.device)
    _ok(lib().psf_event_rows(C.byref(s), C.byref(l), _ptr(events), events.shape[0], _ptr(rows),
                             _stream()), "psf_event_rows")
    return rows


def voxel_homog(sc: dict, tb: dict, T, eta, im: dict, ls: dict, k: int, half_t: int,
                out=None):
    """Voxel-driven homogenization matrix (dense [n_lors, nx*ny], psf_voxel_homog)."""
    s, t, i, l = scanner(sc), table_desc(tb), image(im), lor_set(ls)
    n, _ = lor_set_size(sc, ls)
    if out is None:
        out = torch.empty((n, im["nx"] * im["ny"]), dtype=torch.float32, device=T.device)
    _ok(lib().psf_voxel_homog(C.byref(s), C.byref(t), _ptr(T), _ptr(eta), C.byref(i),
                              C.byref(l), int(k), int(half_t), _ptr(out), _stream()),
        "psf_voxel_homog")
    return out


def sino_bins(sc: dict, ls: dict, device="cuda"):
    """Sinogram (view, bin) of every transaxial pair of the set (int32 [ntp] each)."""
    s, l = scanner(sc), lor_set(ls)
    n, _ = lor_set_size(sc, ls)
    ntp = n // len_ring_pairs(sc, ls)
    view = torch.empty(ntp, dtype=torch.int32, device=device)
    bins = torch.empty(ntp, dtype=torch.int32, device=device)
    _ok(lib().psf_sino_bins(C.byref(s), C.byref(l), _ptr(view), _ptr(bins), _stream()),
        "psf_sino_bins")
    return view, bins


def len_ring_pairs(sc: dict, ls: dict) -> int:
    """Ordered ring pairs of the set (|ra - rb| <= max_ring_diff)."""
    nr = sc["na_block"] * sc["n_block_rings"]
    d = ls["max_ring_diff"]
    return sum(min(nr - 1, r + d) - max(0, r - d) + 1 for r in range(nr))


def histogram(rows, n_rows: int, weight: float = 1.0, out=None):
    """weight x events per row (float [n_rows])."""
    out = torch.empty(n_rows, dtype=torch.float32, device=rows.device) if out is None else out
    _ok(lib().psf_histogram(_ptr(rows), rows.numel(), float(weight), _ptr(out), n_rows,
                            _stream()), "psf_histogram")
    return out


def lor_set_size(sc: dict, ls: dict):
    s, l = scanner(sc), lor_set(ls)
    n, k = C.c_int64(), C.c_int64()
    _ok(lib().psf_lor_set_size(C.byref(s), C.byref(l), C.byref(n), C.byref(k)),
        "psf_lor_set_size")
    return n.value, k.value


def lor_set_list(sc: dict, ls: dict, device="cuda"):
    n, _ = lor_set_size(sc, ls)
    s, l = scanner(sc), lor_set(ls)
    out = torch.empty((n, 2), dtype=torch.int32, device=device)
    _ok(lib().psf_lor_set_list(C.byref(s), C.byref(l), _ptr(out), _stream()), "psf_lor_set_list")
    return out


def lor_set_classes(sc: dict, ls: dict, device="cuda"):
    _, k = lor_set_size(sc, ls)
    s, l = scanner(sc), lor_set(ls)
    out = torch.empty((k, 2), dtype=torch.int32, device=device)
    _ok(lib().psf_lor_set_classes(C.byref(s), C.byref(l), _ptr(out), _stream()),
        "psf_lor_set_classes")
    return out


def sysmat_rows(sc: dict, im: dict, lors, spread=None, half_t: int = 0, half_a: int = 0,
                dtype: str = "f32", buffers=None):
    """CSR rows (row_ptr int64, col int32, val, row_scale or None).

    Without `buffers`: a size query, then the fill into buffers of exactly the
    required size.  With buffers=(row_ptr, col, val, row_scale) of sufficient
    capacity: one call that fills them (PSFError with PSF_ECAPACITY if short).
    """
    s, i = scanner(sc), image(im)
    n = lors.shape[0]
    dt = _DT[dtype]
    dev = lors.device
    nnz = C.c_int64()
    L = lib()
    if buffers is not None:
        row_ptr, col, val, row_scale = buffers
        _ok(L.psf_sysmat_rows(C.byref(s), C.byref(i), _ptr(lors), n, _ptr(spread), half_t,
                              half_a, dt, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(row_scale),
                              col.numel(), C.byref(nnz), _stream()), "psf_sysmat_rows")
        return row_ptr, col[: nnz.value], val[: nnz.value], row_scale
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    row_scale = None if dt == PSF_F32 else torch.empty(n, dtype=torch.float32, device=dev)
    _ok(L.psf_sysmat_rows(C.byref(s), C.byref(i), _ptr(lors), n, _ptr(spread), half_t, half_a,
                          dt, _ptr(row_ptr), None, None, _ptr(row_scale), 0, C.byref(nnz),
                          _stream()), "psf_sysmat_rows(size)")
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(nnz.value, 1), dtype=_TORCH_DT[dt], device=dev)
    _ok(L.psf_sysmat_rows(C.byref(s), C.byref(i), _ptr(lors), n, _ptr(spread), half_t, half_a,
                          dt, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(row_scale), nnz.value,
                          C.byref(nnz), _stream()), "psf_sysmat_rows")
    return row_ptr, col[: nnz.value], val[: nnz.value], row_scale


def sysmat_rows_set(sc: dict, im: dict, ls: dict, buffers=None, device="cuda"):
    """Geometric rows of a structured LOR set (row_ptr, col, val), rows in set
    order.  buffers=(row_ptr, col, val) of sufficient capacity are filled in
    one call; otherwise a size query precedes the fill."""
    s, i, l = scanner(sc), image(im), lor_set(ls)
    nnz = C.c_int64()
    L = lib()
    if buffers is not None:
        row_ptr, col, val = buffers
        _ok(L.psf_sysmat_rows_set(C.byref(s), C.byref(i), C.byref(l), _ptr(row_ptr), _ptr(col),
                                  _ptr(val), col.numel(), C.byref(nnz), _stream()),
            "psf_sysmat_rows_set")
        return row_ptr, col[: nnz.value], val[: nnz.value]
    n, _ = lor_set_size(sc, ls)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=device)
    _ok(L.psf_sysmat_rows_set(C.byref(s), C.byref(i), C.byref(l), _ptr(row_ptr), None, None, 0,
                              C.byref(nnz), _stream()), "psf_sysmat_rows_set(size)")
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=device)
    val = torch.empty(max(nnz.value, 1), dtype=torch.float32, device=device)
    _ok(L.psf_sysmat_rows_set(C.byref(s), C.byref(i), C.byref(l), _ptr(row_ptr), _ptr(col),
                              _ptr(val), nnz.value, C.byref(nnz), _stream()), "psf_sysmat_rows_set")
    return row_ptr, col[: nnz.value], val[: nnz.value]


def sysmat_rows_set_typed(sc: dict, im: dict, ls: dict, dtype: str = "bf16", buffers=None,
                          device="cuda"):
    """Geometric rows of a structured set with values in `dtype` ("f32",
    "bf16", "f16"): (row_ptr, col, val, row_scale); row_scale is None for
    "f32", else the per-row FP32 scale (value = stored x scale).  buffers =
    (row_ptr, col, val, row_scale) of sufficient capacity are filled in one
    call; otherwise a size query precedes the fill."""
    s, i, l = scanner(sc), image(im), lor_set(ls)
    dt = _DT[dtype]
    nnz = C.c_int64()
    L = lib()
    if buffers is not None:
        row_ptr, col, val, row_scale = buffers
        _ok(L.psf_sysmat_rows_set_typed(C.byref(s), C.byref(i), C.byref(l), dt, _ptr(row_ptr),
                                        _ptr(col), _ptr(val), _ptr(row_scale), col.numel(),
                                        C.byref(nnz), _stream()), "psf_sysmat_rows_set_typed")
        return row_ptr, col[: nnz.value], val[: nnz.value], row_scale
    n, _ = lor_set_size(sc, ls)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=device)
    _ok(L.psf_sysmat_rows_set_typed(C.byref(s), C.byref(i), C.byref(l), dt, _ptr(row_ptr), None,
                                    None, None, 0, C.byref(nnz), _stream()),
        "psf_sysmat_rows_set_typed(size)")
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=device)
    val = torch.empty(max(nnz.value, 1), dtype=_TORCH_DT[dt], device=device)
    row_scale = None if dt == PSF_F32 else torch.empty(n, dtype=torch.float32, device=device)
    _ok(L.psf_sysmat_rows_set_typed(C.byref(s), C.byref(i), C.byref(l), dt, _ptr(row_ptr),
                                    _ptr(col), _ptr(val), _ptr(row_scale), nnz.value,
                                    C.byref(nnz), _stream()), "psf_sysmat_rows_set_typed")
    return row_ptr, col[: nnz.value], val[: nnz.value], row_scale


class Matrix:
    """Projector plan over CSR tensors (kept alive by this object)."""

    def __init__(self, row_ptr, col, val, n_cols: int, row_scale=None):
        dt = {torch.float32: PSF_F32, torch.bfloat16: PSF_BF16, torch.float16: PSF_F16}[val.dtype]
        self._keep = [row_ptr, col, val, row_scale]
        self.n_rows = row_ptr.shape[0] - 1
        self.n_cols = int(n_cols)
        self.topn = 0  # kept entries per class spread of a top-N plan
        self.dtype_name = {PSF_F32: "f32", PSF_BF16: "bf16", PSF_F16: "f16"}[dt]
        self._h = C.c_void_p()
        _ok(lib().psf_matrix_create(C.byref(self._h), self.n_rows, self.n_cols, _ptr(row_ptr),
                                    _ptr(col), _ptr(val), dt, _ptr(row_scale), _stream()),
            "psf_matrix_create")

    @classmethod
    def traced(cls, sc: dict, im: dict, ls: dict):
        """A plan without stored rows whose geometric rows (those of the
        structured set on this image) are traced whenever a projection needs
        them (psf_matrix_create_otf)."""
        self = cls.__new__(cls)
        s, i, l = scanner(sc), image(im), lor_set(ls)
        self._keep = []
        n, _ = lor_set_size(sc, ls)
        self.n_rows = n
        self.n_cols = int(im["nx"]) * int(im["ny"]) * int(im["nz"])
        self.topn = 0
        self.dtype_name = "f32"
        self._h = C.c_void_p()
        _ok(lib().psf_matrix_create_otf(C.byref(self._h), C.byref(s), C.byref(i), C.byref(l),
                                        _stream()), "psf_matrix_create_otf")
        return self

    def set_spread(self, sc: dict, ls: dict, half_t: int, half_a: int, class_spread):
        self._spread = class_spread  # the plan keeps the pointer; keep the tensor alive
        s, l = scanner(sc), lor_set(ls)
        _ok(lib().psf_matrix_set_spread(self._h, C.byref(s), C.byref(l), half_t, half_a,
                                        _ptr(class_spread)), "psf_matrix_set_spread")
        self.topn = 0
        return self

    def set_spread_topn(self, sc: dict, ls: dict, half_t: int, half_a: int, idx, w,
                        scale=None):
        """Factored form with top-N class spreads (outputs of spread_topn); with
        BF16 weights and their per-class scale (spread_topn_bf16) when scale is
        given."""
        self._spread = (idx, w, scale)  # the plan keeps the pointers; keep them alive
        s, l = scanner(sc), lor_set(ls)
        if scale is None:
            _ok(lib().psf_matrix_set_spread_topn(self._h, C.byref(s), C.byref(l), half_t,
                                                 half_a, idx.shape[1], _ptr(idx), _ptr(w)),
                "psf_matrix_set_spread_topn")
        else:
            _ok(lib().psf_matrix_set_spread_topn_bf16(self._h, C.byref(s), C.byref(l), half_t,
                                                      half_a, idx.shape[1], _ptr(idx), _ptr(w),
                                                      _ptr(scale)),
                "psf_matrix_set_spread_topn_bf16")
        self.topn = int(idx.shape[1])
        return self

    def build_sparse_adjoint(self):
        """Transpose of the top-N S, so S^T of sparse inputs scatters from their
        nonzero entries (psf_matrix_build_sparse_adjoint)."""
        _ok(lib().psf_matrix_build_sparse_adjoint(self._h, _stream()),
            "psf_matrix_build_sparse_adjoint")
        return self

    def autotune(self):
        """Pick the stored-row projector launches by timing the candidates;
        returns ((chunk, threads) forward, (chunk, threads) back): chunk -1 =
        streaming tiles, 0 = grid-stride kernels, > 0 = work queue."""
        c, t = (C.c_int32 * 2)(), (C.c_int32 * 2)()
        _ok(lib().psf_matrix_autotune(self._h, c, t, _stream()), "psf_matrix_autotune")
        return (c[0], t[0]), (c[1], t[1])

    def set_launch(self, chunk: int, threads: int = 256):
        """Stored-row projector launch: chunk 0 = grid-stride kernels, -1 the
        streaming forward, -2 the bulk-staged kernels, else the work-queue
        kernels taking `chunk` rows per warp."""
        _ok(lib().psf_matrix_set_launch(self._h, int(chunk), int(threads)),
            "psf_matrix_set_launch")
        return self

    def check(self):
        """Raise if a bounded device wait of this plan gave up (psf_matrix_check)."""
        _ok(lib().psf_matrix_check(self._h, _stream()), "psf_matrix_check")
        return self

    def set_stencil_form(self, form: int):
        """Stencil form of a factored plan (0 default, 1 plain, 2 register-blocked, 3, 4, 5)."""
        _ok(lib().psf_matrix_set_stencil_form(self._h, int(form)), "psf_matrix_set_stencil_form")
        return self

    def set_image(self, im: dict):
        """Declare the voxel grid of the columns (psf_matrix_set_image)."""
        i = image(im)
        _ok(lib().psf_matrix_set_image(self._h, C.byref(i)), "psf_matrix_set_image")
        return self

    def forward(self, x, out=None):
        if out is None:
            out = torch.empty(self.n_rows, dtype=torch.float32, device=x.device)
        _ok(lib().psf_forward(self._h, _ptr(x), _ptr(out), _stream()), "psf_forward")
        return out

    def forward_masked(self, x, mask, out=None):
        """A x on the rows with mask != 0, 0 elsewhere (psf_forward_masked)."""
        if out is None:
            out = torch.empty(self.n_rows, dtype=torch.float32, device=x.device)
        _ok(lib().psf_forward_masked(self._h, _ptr(x), _ptr(mask), _ptr(out), _stream()),
            "psf_forward_masked")
        return out

    def sensitivity(self, out=None, device="cuda"):
        """A^T 1 (psf_sensitivity)."""
        if out is None:
            out = torch.empty(self.n_cols, dtype=torch.float32, device=device)
        _ok(lib().psf_sensitivity(self._h, _ptr(out), _stream()), "psf_sensitivity")
        return out

    def back_sens(self, y, out=None, sens=None):
        """(A^T y, A^T 1) with one pass over the rows (psf_back_sens)."""
        if out is None:
            out = torch.empty(self.n_cols, dtype=torch.float32, device=y.device)
        if sens is None:
            sens = torch.empty(self.n_cols, dtype=torch.float32, device=y.device)
        _ok(lib().psf_back_sens(self._h, _ptr(y), _ptr(out), _ptr(sens), _stream()),
            "psf_back_sens")
        return out, sens

    def back(self, y, out=None):
        if out is None:
            out = torch.empty(self.n_cols, dtype=torch.float32, device=y.device)
        _ok(lib().psf_back(self._h, _ptr(y), _ptr(out), _stream()), "psf_back")
        return out

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.psf_matrix_destroy(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass


def em_ratio(y, yhat, out=None):
    out = torch.empty_like(y) if out is None else out
    _ok(lib().psf_em_ratio(_ptr(y), _ptr(yhat), _ptr(out), y.numel(), _stream()), "psf_em_ratio")
    return out


def em_update(x, bp, sens, floor: float):
    _ok(lib().psf_em_update(_ptr(x), _ptr(bp), _ptr(sens), float(floor), x.numel(), _stream()),
        "psf_em_update")
    return x
