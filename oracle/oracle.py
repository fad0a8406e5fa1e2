"""ctypes marshalling for ``psf_oracle.c`` (test infrastructure only).

Every function takes the plain description dicts produced by the seeded input
module (scanner, table, image) and numpy arrays, and returns numpy arrays in
float64.  See ``psf_oracle.c`` for the paper passages each step follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

NORM_NONE, NORM_EFF, NORM_UNIT = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpsf_oracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Scanner(C.Structure):
    _fields_ = [("R", C.c_int), ("Nb", C.c_int), ("Na", C.c_int), ("NBR", C.c_int),
                ("wt", C.c_double), ("wa", C.c_double), ("depth", C.c_double),
                ("gt", C.c_double), ("ga", C.c_double), ("radius", C.c_double),
                ("bga", C.c_double), ("mu", C.c_double)]


class _Table(C.Structure):
    _fields_ = [("Kt", C.c_int), ("Ka", C.c_int), ("Pt", C.c_int), ("Pa", C.c_int),
                ("Mt", C.c_int), ("Ma", C.c_int),
                ("amax_t_deg", C.c_double), ("amax_a_deg", C.c_double)]


class _Image(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class _Entry(C.Structure):
    _fields_ = [("dt", C.c_int), ("da", C.c_int), ("val", C.c_double)]


_P = C.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            sig = {
                "orc_sigma": (C.c_double, [_P]),
                "orc_node": (C.c_int, [C.c_double, C.c_double, C.c_int]),
                "orc_gap_eq": (None, [_P, C.c_double, C.c_double, _P, _P, _P]),
                "orc_face_point": (None, [_P, C.c_int, C.c_double, C.c_double, _P]),
                "orc_trace_response": (None, [_P, C.c_double, C.c_double, C.c_double,
                                              C.c_double, C.c_int, C.c_int, _P, _P]),
                "orc_table_build": (None, [_P, _P, _P, _P]),
                "orc_composed": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, _P, _P,
                                           C.c_int, _P]),
                "orc_spread": (None, [_P, _P, _P, _P, C.c_int64, C.c_int, C.c_int, C.c_int, _P]),
                "orc_siddon": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
                "orc_slabclip": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
                "orc_rows_geom_count": (None, [_P, _P, _P, C.c_int64, _P]),
                "orc_rows_geom_fill": (None, [_P, _P, _P, C.c_int64, _P, _P, _P]),
                "orc_window_pair": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int,
                                              C.c_int, C.c_int, _P, _P]),
                "orc_rows_psf_dense": (None, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_int,
                                              C.c_int, _P, C.c_int64, _P]),
                "orc_csr_fwd": (None, [C.c_int64, _P, _P, _P, _P, _P]),
                "orc_csr_back": (None, [C.c_int64, _P, _P, _P, _P, C.c_int64, _P]),
                "orc_spread_apply": (None, [_P, C.c_int64, _P, _P, C.c_int, C.c_int, _P, _P, _P]),
                "orc_spread_adjoint": (None, [_P, C.c_int64, _P, _P, C.c_int, C.c_int, _P, _P, _P]),
                "orc_spread_topn": (None, [C.c_int64, _P, C.c_int, C.c_int, C.c_int, _P, _P]),
                "orc_sino_index": (None, [_P, C.c_int, C.c_int, C.c_int, _P, _P]),
                "orc_voxel_homog": (None, [_P, _P, _P, _P, C.c_int, C.c_int, _P, C.c_int64, _P,
                                           _P]),
                "orc_lor_normal": (None, [_P, C.c_int, C.c_int, _P, _P]),
                "orc_threads": (C.c_int, []),
                "orc_tie_margin": (None, [_P, _P, _P, _P, C.c_int64, _P]),
                "orc_tie_stats": (None, [_P, _P, _P, _P, C.c_int64, C.c_double, _P, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _scanner(s: dict) -> _Scanner:
    return _Scanner(int(s["n_blocks"]), int(s["nt_block"]), int(s["na_block"]),
                    int(s["n_block_rings"]), float(s["xtal_w_t"]), float(s["xtal_w_a"]),
                    float(s["depth"]), float(s["gap_t"]), float(s["gap_a"]),
                    float(s["radius"]), float(s["block_gap_a"]), float(s["mu"]))


def _table(t: dict) -> _Table:
    return _Table(int(t["n_ang_t"]), int(t["n_ang_a"]), int(t["n_sub_t"]), int(t["n_sub_a"]),
                  int(t["max_off_t"]), int(t["max_off_a"]),
                  float(t["ang_max_t_deg"]), float(t["ang_max_a_deg"]))


def _image(im: dict) -> _Image:
    return _Image(int(im["nx"]), int(im["ny"]), int(im["nz"]), float(im["dx"]),
                  float(im["dy"]), float(im["dz"]), float(im["ox"]), float(im["oy"]),
                  float(im["oz"]))


def _lors(lors) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(lors, dtype=np.int32).reshape(-1, 2))
    return a


def threads() -> int:
    return int(_load().orc_threads())


def sigma(scanner: dict) -> float:
    """Half gap AB = BC between neighbouring blocks (Fig. 6)."""
    s = _scanner(scanner)
    return float(_load().orc_sigma(C.byref(s)))


def node(angle_rad: float, amax_deg: float, K: int) -> int:
    return int(_load().orc_node(float(angle_rad), float(amax_deg), int(K)))


def gap_eq(scanner: dict, alpha: float, nu: float):
    """(beta, AP1, run) of Eq. 2 and Eq. 4 for entry distance nu = CP0."""
    s = _scanner(scanner)
    out = np.zeros(3)
    _load().orc_gap_eq(C.byref(s), float(alpha), float(nu), _ptr(out[0:]), _ptr(out[1:]),
                       _ptr(out[2:]))
    return float(out[0]), float(out[1]), float(out[2])


def face_point(scanner: dict, xid: int, off_t: float = 0.0, off_a: float = 0.0) -> np.ndarray:
    s = _scanner(scanner)
    P = np.zeros(3)
    _load().orc_face_point(C.byref(s), int(xid), float(off_t), float(off_a), _ptr(P))
    return P


def trace_response(scanner: dict, alpha_t: float, theta: float, u: float, v: float,
                   Mx: int, My: int):
    """First-interaction probabilities of one ray in a flat array (Sec. 2.1.1)."""
    s = _scanner(scanner)
    T = np.zeros((Mx, My))
    eta = np.zeros(1)
    _load().orc_trace_response(C.byref(s), float(alpha_t), float(theta), float(u), float(v),
                               int(Mx), int(My), _ptr(T), _ptr(eta))
    return T, float(eta[0])


def table_build(scanner: dict, table: dict):
    """P-SPIR table T[Kt,Ka,Pt,Pa,Mt,Ma] and eta[Kt,Ka,Pt,Pa] (Sec. 2.1.1, 2.1.3)."""
    s, t = _scanner(scanner), _table(table)
    shp = (t.Kt, t.Ka, t.Pt, t.Pa)
    T = np.zeros(shp + (t.Mt, t.Ma))
    eta = np.zeros(shp)
    _load().orc_table_build(C.byref(s), C.byref(t), _ptr(T), _ptr(eta))
    return T, eta


def composed(scanner: dict, table: dict, T: np.ndarray, xid: int, ipt: int, ipa: int,
             direction):
    """Response around crystal xid with two-block penetration (Sec. 2.1.2)."""
    s, t = _scanner(scanner), _table(table)
    T = np.ascontiguousarray(T, dtype=np.float64)
    cap = 4 * t.Mt * t.Ma + 16
    out = (_Entry * cap)()
    eta = np.zeros(1)
    d = np.ascontiguousarray(np.asarray(direction, dtype=np.float64))
    n = _load().orc_composed(C.byref(s), C.byref(t), _ptr(T), int(xid), int(ipt), int(ipa),
                             _ptr(d), out, cap, _ptr(eta))
    return [(out[k].dt, out[k].da, out[k].val) for k in range(n)], float(eta[0])


def spread(scanner: dict, table: dict, T: np.ndarray, lors, Wt: int, Wa: int,
           norm: int = NORM_EFF) -> np.ndarray:
    """Homogenization spread w[n, E, E] of each LOR (Eq. 10-12)."""
    s, t = _scanner(scanner), _table(table)
    T = np.ascontiguousarray(T, dtype=np.float64)
    L = _lors(lors)
    E = (2 * Wt + 1) * (2 * Wa + 1)
    w = np.zeros((L.shape[0], E, E))
    _load().orc_spread(C.byref(s), C.byref(t), _ptr(T), _ptr(L), L.shape[0], int(Wt), int(Wa),
                       int(norm), _ptr(w))
    return w


def tie_margin(scanner: dict, table: dict, T: np.ndarray, lors) -> np.ndarray:
    """Per LOR, the smallest distance of a rounding decision to its boundary
    (see orc_tie_margin); LORs below working precision have several correct
    spreads."""
    s, t = _scanner(scanner), _table(table)
    T = np.ascontiguousarray(T, dtype=np.float64)
    L = _lors(lors)
    out = np.zeros(L.shape[0])
    _load().orc_tie_margin(C.byref(s), C.byref(t), _ptr(T), _ptr(L), L.shape[0], _ptr(out))
    return out


def tie_count(scanner: dict, table: dict, T: np.ndarray, lors, tau: float):
    """Per LOR, (smallest margin, number of sub-LORs with a decision closer than
    tau to its boundary)."""
    s, t = _scanner(scanner), _table(table)
    T = np.ascontiguousarray(T, dtype=np.float64)
    L = _lors(lors)
    m = np.zeros(L.shape[0])
    c = np.zeros(L.shape[0], dtype=np.int64)
    _load().orc_tie_stats(C.byref(s), C.byref(t), _ptr(T), _ptr(L), L.shape[0], float(tau),
                          _ptr(m), _ptr(c))
    return m, c


def _trace(fn, image: dict, a, b):
    im = _image(image)
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    cap = im.nx * im.ny * im.nz if fn == "orc_slabclip" else im.nx + im.ny + im.nz + 8
    idx = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap)
    n = getattr(_load(), fn)(C.byref(im), _ptr(a), _ptr(b), _ptr(idx), _ptr(ln), cap)
    if n < 0:
        raise RuntimeError("oracle tracer capacity exceeded")
    return idx[:n].copy(), ln[:n].copy()


def siddon(image: dict, a, b):
    """Parametric chord lengths of segment a->b (sorted voxel index, mm)."""
    return _trace("orc_siddon", image, a, b)


def slabclip(image: dict, a, b):
    """Brute per-voxel slab clipping of segment a->b (small grids)."""
    return _trace("orc_slabclip", image, a, b)


def rows_geom(scanner: dict, image: dict, lors):
    """Geometric matrix G in CSR (row_ptr int64, col int64, val float64)."""
    s, im = _scanner(scanner), _image(image)
    L = _lors(lors)
    n = L.shape[0]
    counts = np.zeros(n, dtype=np.int64)
    lib = _load()
    lib.orc_rows_geom_count(C.byref(s), C.byref(im), _ptr(L), n, _ptr(counts))
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    col = np.zeros(int(ptr[-1]), dtype=np.int64)
    val = np.zeros(int(ptr[-1]))
    lib.orc_rows_geom_fill(C.byref(s), C.byref(im), _ptr(L), n, _ptr(ptr), _ptr(col), _ptr(val))
    return ptr, col, val


def window_pair(scanner: dict, id1: int, id2: int, Wt: int, Wa: int, e1: int, e2: int):
    s = _scanner(scanner)
    X = C.c_int()
    Y = C.c_int()
    r = _load().orc_window_pair(C.byref(s), int(id1), int(id2), int(Wt), int(Wa), int(e1),
                                int(e2), C.byref(X), C.byref(Y))
    return None if r else (X.value, Y.value)


def pair_row_map(scanner: dict, lors) -> np.ndarray:
    """Dense map (X*Ncrys + Y, both orders) -> row index of the LOR list, else -1."""
    nc = int(scanner["n_blocks"]) * int(scanner["nt_block"]) * int(scanner["na_block"]) * int(
        scanner["n_block_rings"])
    L = _lors(lors)
    m = np.full(nc * nc, -1, dtype=np.int64)
    r = np.arange(L.shape[0], dtype=np.int64)
    m[L[:, 0].astype(np.int64) * nc + L[:, 1]] = r
    m[L[:, 1].astype(np.int64) * nc + L[:, 0]] = r
    return m


def rows_psf_dense(scanner: dict, lors, G, w: np.ndarray, Wt: int, Wa: int, nvox: int):
    """Dense PSF matrix A = S G over the LOR list (small problems)."""
    s = _scanner(scanner)
    L = _lors(lors)
    ptr, col, val = G
    w = np.ascontiguousarray(w, dtype=np.float64)
    pr = pair_row_map(scanner, L)
    A = np.zeros((L.shape[0], nvox))
    _load().orc_rows_psf_dense(C.byref(s), L.shape[0], _ptr(L), _ptr(ptr), _ptr(col), _ptr(val),
                               _ptr(w), int(Wt), int(Wa), _ptr(pr), int(nvox), _ptr(A))
    return A


def csr_fwd(G, x: np.ndarray) -> np.ndarray:
    ptr, col, val = G
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = ptr.shape[0] - 1
    y = np.zeros(n)
    _load().orc_csr_fwd(n, _ptr(ptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def csr_back(G, y: np.ndarray, nvox: int) -> np.ndarray:
    ptr, col, val = G
    y = np.ascontiguousarray(y, dtype=np.float64)
    x = np.zeros(nvox)
    _load().orc_csr_back(ptr.shape[0] - 1, _ptr(ptr), _ptr(col), _ptr(val), _ptr(y), nvox,
                         _ptr(x))
    return x


def spread_apply(scanner: dict, lors, w: np.ndarray, Wt: int, Wa: int, p: np.ndarray):
    """y = S p: each geometric LOR's value spread onto its window's measured pairs."""
    s = _scanner(scanner)
    L = _lors(lors)
    w = np.ascontiguousarray(w, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    y = np.zeros(L.shape[0])
    _load().orc_spread_apply(C.byref(s), L.shape[0], _ptr(L), _ptr(w), int(Wt), int(Wa),
                             _ptr(pair_row_map(scanner, L)), _ptr(p), _ptr(y))
    return y


def spread_adjoint(scanner: dict, lors, w: np.ndarray, Wt: int, Wa: int, r: np.ndarray):
    """q = S^T r."""
    s = _scanner(scanner)
    L = _lors(lors)
    w = np.ascontiguousarray(w, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    q = np.zeros(L.shape[0])
    _load().orc_spread_adjoint(C.byref(s), L.shape[0], _ptr(L), _ptr(w), int(Wt), int(Wa),
                               _ptr(pair_row_map(scanner, L)), _ptr(r), _ptr(q))
    return q


def voxel_homog(scanner: dict, table: dict, T: np.ndarray, image: dict, lors, k: int, Wt: int):
    """Voxel-driven homogenization of a planar scanner (Sec. 2.3 Eq. 11-12):
    the dense matrix A (n_lors x nvox, rows of the LOR list) from k lines per
    pixel centre, and each pixel's smallest decision margin."""
    s, tb, im = _scanner(scanner), _table(table), _image(image)
    L = _lors(lors)
    T = np.ascontiguousarray(T, dtype=np.float64)
    nvox = int(image["nx"]) * int(image["ny"])
    A = np.zeros((L.shape[0], nvox))
    margin = np.zeros(nvox)
    _load().orc_voxel_homog(C.byref(s), C.byref(tb), _ptr(T), C.byref(im), int(k), int(Wt),
                            _ptr(pair_row_map(scanner, L)), L.shape[0], _ptr(A), _ptr(margin))
    return A, margin


def sino_index(scanner: dict, pairs, fan_half: int):
    """(view, bin) of each transaxial pair (a, b), a < b (int [n, 2])."""
    sc = _scanner(scanner)
    P = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    out = np.zeros((P.shape[0], 2), dtype=np.int64)
    v, b = C.c_int(), C.c_int()
    f = _load().orc_sino_index
    for k, (a, bb) in enumerate(P):
        f(C.byref(sc), int(a), int(bb), int(fan_half), C.byref(v), C.byref(b))
        out[k] = (v.value, b.value)
    return out


def lor_normal(scanner: dict, a: int, b: int):
    """(phi in [0, pi), signed axis distance) of the line joining the face
    centres of transaxial crystals a and b."""
    sc = _scanner(scanner)
    ph, d = C.c_double(), C.c_double()
    _load().orc_lor_normal(C.byref(sc), int(a), int(b), C.byref(ph), C.byref(d))
    return ph.value, d.value


def spread_topn(w: np.ndarray, Wt: int, Wa: int, N: int):
    """Top-N truncation of each LOR's spread (n x E x E): the truncated,
    rescaled weights (same shape) and the kept window indices in rank order
    (n x N int32)."""
    E = (2 * Wt + 1) * (2 * Wa + 1)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1, E * E)
    n = w.shape[0]
    if not 1 <= N <= E * E:
        raise ValueError("N must be in 1 .. window size")
    out = np.zeros_like(w)
    idx = np.zeros((n, N), dtype=np.int32)
    _load().orc_spread_topn(n, _ptr(w), int(Wt), int(Wa), int(N), _ptr(out), _ptr(idx))
    return out.reshape(n, E, E), idx


def topn_bf16(w: np.ndarray):
    """Top-N weights (n x N) in their BF16 storage form for the list-mode
    projector (a reading: the paper's list-mode step keeps the top-N weights;
    16-bit storage with one scale per spread is this build's choice): scale =
    the largest |w| of a row in FP32 (1 when all are 0), code = w / scale
    (FP32 division) rounded to the nearest BF16, ties to even.  Returns the
    codes' bit patterns (uint16, n x N), the scales (float32, n) and the
    dequantized weights code x scale (float64, n x N)."""
    w32 = np.ascontiguousarray(w, dtype=np.float32)
    mx = np.abs(w32).max(axis=1) if w32.shape[1] else np.zeros(w32.shape[0], np.float32)
    sc = np.where(mx > 0, mx, np.float32(1.0)).astype(np.float32)
    q = (w32 / sc[:, None]).astype(np.float32)
    b = q.view(np.uint32).astype(np.uint64)
    # round to nearest even on the 16 bits dropped: add 0x7fff plus the kept
    # part's lowest bit, then truncate
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
    deq = (r.astype(np.uint32) << 16).view(np.float32).astype(np.float64) * sc[:, None]
    return r, sc, deq


def mlem(fwd, back, y: np.ndarray, nvox: int, iters: int, x0=None):
    """MLEM (the EM iteration OSEM is built on, Sec. 3).

    sens = A^T 1; x <- x * A^T(y / A x) / sens.  Voxels with
    sens < 1e-12 * max(sens) are held at 0, and 0/0 in the ratio is 0.
    """
    y = np.asarray(y, dtype=np.float64)
    sens = back(np.ones_like(y))
    live = sens >= 1e-12 * sens.max()
    x = np.where(live, 1.0, 0.0) if x0 is None else np.array(x0, dtype=np.float64)
    for _ in range(iters):
        yh = fwd(x)
        ratio = np.divide(y, yh, out=np.zeros_like(y), where=yh > 0)
        bp = back(ratio)
        x = np.where(live, x * bp / np.where(live, sens, 1.0), 0.0)
    return x


def listmode_osem(fwd, back, event_rows: np.ndarray, n_lors: int, n_subsets: int, iters: int,
                  x0=None):
    """List-mode OSEM (the next step named in Sec. 5; subsets of events as
    the OSEM subsets of Sec. 3), event by event: the events are split into
    n_subsets consecutive subsets and for each subset
        x_j <- x_j / (s_j / n_subsets) * sum_{e in subset} a_ej / sum_k a_ek x_k,
    s = A^T 1, the per-event terms a_e / (a_e x) gathered one event at a time
    into LOR space and back-projected once.  Events with row -1 (not in the
    set) or a zero forward projection contribute nothing; voxels with
    s < 1e-12 max(s) are held at 0."""
    rows = np.asarray(event_rows, dtype=np.int64)
    sens = back(np.ones(n_lors))
    live = sens >= 1e-12 * sens.max()
    x = np.where(live, 1.0, 0.0) if x0 is None else np.array(x0, dtype=np.float64)
    n_ev = rows.shape[0]
    bounds = [n_ev * j // n_subsets for j in range(n_subsets + 1)]
    for _ in range(iters):
        for j in range(n_subsets):
            yh = fwd(x)
            r = np.zeros(n_lors)
            for m in rows[bounds[j]:bounds[j + 1]]:
                if m >= 0 and yh[m] > 0:
                    r[m] += 1.0 / yh[m]
            bp = back(r)
            x = np.where(live, x * bp / np.where(live, sens / n_subsets, 1.0), 0.0)
    return x


def poisson_loglik(fwd, y: np.ndarray, x: np.ndarray) -> float:
    """L(x) = sum y log(Ax) - Ax (the log y! term dropped)."""
    yh = fwd(x)
    pos = yh > 0
    return float(np.sum(y[pos] * np.log(yh[pos])) - np.sum(yh))


def poisson_grad(fwd, back, y: np.ndarray, x: np.ndarray) -> np.ndarray:
    """grad L = A^T(y / Ax) - A^T 1."""
    yh = fwd(x)
    ratio = np.divide(y, yh, out=np.zeros_like(yh), where=yh > 0)
    return back(ratio) - back(np.ones_like(yh))
