"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances and where they come from:
  * response table: |d| <= 1e-5 |ref| + TABLE_ATOL.  FP32 box bounds and
    crossing depths carry absolute errors of a few 1e-6 mm, so a path clipped
    through a crystal corner (tens of micrometres long) has a length error
    near 2e-5 mm; the probability error is then below mu * 2.3e-5 = 2e-6;
  * spread: |d| <= 1e-5 |ref| + SPREAD_ATOL_REL * max|ref| per LOR (products of
    table values inherit the table's absolute floor, and FP32 sums of
    products leave a residue near 1e-7 of the largest term where the exact
    sum cancels to zero);
  * chords: voxel sets bit-exact after removing voxels with chord < 1e-6 mm on
    either side, values |d| <= 1e-4 |ref| + 1e-6 mm;
  * PSF rows and projections: |d| <= 1e-4 |ref| + 1e-6 * (row scale).
"""
import numpy as np

SET_THR_MM = 1e-6
TABLE_ATOL = 2e-6
SPREAD_ATOL_REL = 1e-6


def assert_close(got, ref, rtol, atol, what=""):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    err = np.abs(got - ref)
    bad = err > rtol * np.abs(ref) + atol
    if bad.any():
        i = np.flatnonzero(bad.reshape(-1))[:5]
        raise AssertionError(
            f"{what}: {bad.sum()} / {bad.size} outside tolerance; first at {i}: "
            f"got {got.reshape(-1)[i]}, ref {ref.reshape(-1)[i]}")
    den = np.abs(ref) + atol
    ratio = np.divide(err, den, out=np.zeros_like(err), where=den > 0)  # err is 0 where den is
    return float(np.max(ratio)) if err.size else 0.0


def csr_keys(ptr, col, ncol):
    ptr = np.asarray(ptr, dtype=np.int64)
    rows = np.repeat(np.arange(len(ptr) - 1, dtype=np.int64), np.diff(ptr))
    return rows * ncol + np.asarray(col, dtype=np.int64)


def compare_chord_rows(gpu, ref, ncol, rtol=1e-4, atol=1e-6, thr=SET_THR_MM):
    """Geometric rows: sorted columns, bit-exact voxel sets (chords >= thr on
    both sides), chord values within tolerance.  Returns (max rel err, n)."""
    gptr, gcol, gval = [np.asarray(a) for a in gpu]
    rptr, rcol, rval = [np.asarray(a) for a in ref]
    assert len(gptr) == len(rptr)
    # columns strictly ascending inside each GPU row
    d = np.diff(gcol.astype(np.int64))
    starts = gptr[1:-1]
    inner = np.ones(len(gcol), dtype=bool)
    inner[starts[starts < len(gcol)]] = False
    assert np.all(d[inner[1:]] > 0), "GPU columns not strictly ascending within rows"
    gk = csr_keys(gptr, gcol, ncol)
    rk = csr_keys(rptr, rcol, ncol)
    gm, rm = gval >= thr, rval >= thr
    gk2, rk2 = gk[gm], rk[rm]
    only_g = np.setdiff1d(gk2, rk2)
    only_r = np.setdiff1d(rk2, gk2)
    # a voxel right at the exemption threshold may sit on either side of it
    near = lambda k, keys, vals: np.isin(k, keys[np.abs(vals - thr) < 1e-9])
    assert np.all(near(only_g, rk, rval) | near(only_g, gk, gval)), f"GPU extra voxels {only_g[:5]}"
    assert np.all(near(only_r, gk, gval) | near(only_r, rk, rval)), f"GPU missing voxels {only_r[:5]}"
    common, gi, ri = np.intersect1d(gk2, rk2, return_indices=True)
    err = assert_close(gval[gm][gi], rval[rm][ri], rtol, atol, "chords")
    return err, len(common)
