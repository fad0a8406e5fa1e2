"""Pins of the oracle's geometric rows (chord lengths), PSF rows A = S G and
projectors / MLEM (Sec. 2.3, Sec. 3)."""
import math

import numpy as np
import pytest

from paper_1607_06170_gb300 import inputs as I

IM2 = I.image(16, 12, 1, 1.0, 1.5, 1.0)
IM3 = I.image(9, 7, 6, 1.0, 1.3, 0.9)


def test_axis_aligned_chords(orc):
    # A ray along x inside one row crosses every voxel of that row fully.
    idx, ln = orc.siddon(IM2, [-100.0, 0.3, 0.0], [100.0, 0.3, 0.0])
    assert len(idx) == 16
    np.testing.assert_allclose(ln, 1.0, rtol=1e-13)
    assert ln.sum() == pytest.approx(16.0, rel=1e-13)
    iy = int(math.floor((0.3 - IM2["oy"]) / IM2["dy"]))
    np.testing.assert_array_equal(idx, iy * 16 + np.arange(16))
    # along y: chords equal dy
    idx, ln = orc.siddon(IM2, [0.2, -50.0, 0.0], [0.2, 50.0, 0.0])
    np.testing.assert_allclose(ln, 1.5, rtol=1e-13)
    assert len(idx) == 12


def test_ray_on_a_grid_plane_belongs_to_upper_voxel(orc):
    # y = 0 is the plane between rows 5 and 6 (half-open voxels [lo, hi)).
    idx, ln = orc.siddon(IM2, [-100.0, 0.0, 0.0], [100.0, 0.0, 0.0])
    assert np.all(idx // 16 == 6)
    # the top boundary plane belongs to no voxel
    top = IM2["oy"] + 12 * 1.5
    idx, _ = orc.siddon(IM2, [-100.0, top, 0.0], [100.0, top, 0.0])
    assert len(idx) == 0
    idx, _ = orc.slabclip(IM2, [-100.0, top, 0.0], [100.0, top, 0.0])
    assert len(idx) == 0


@pytest.mark.parametrize("eps", [0.0, 1e-13, -1e-13])
def test_ray_within_rounding_of_a_plane_is_on_it(orc, eps):
    # A LOR on a grid plane by symmetry, tilted or shifted by rounding noise,
    # still belongs wholly to the voxel row above the plane, in both tracers.
    for fn in (orc.siddon, orc.slabclip):
        idx, ln = fn(IM2, [-100.0, 3.0 + eps, 0.0], [100.0, 3.0 - eps, 0.0])
        iy = int(round((3.0 - IM2["oy"]) / IM2["dy"]))
        assert np.all(idx // 16 == iy) and len(idx) == 16
        np.testing.assert_allclose(ln, 1.0, rtol=1e-12)
    # a genuinely tilted ray (1e-6 voxel) is not snapped
    idx, _ = orc.siddon(IM2, [-100.0, 3.0 + 1e-6, 0.0], [100.0, 3.0 - 1e-6, 0.0])
    assert set(idx // 16) == {iy - 1, iy}


def _compare(a, b, tol_set=1e-9):
    ia, la = a
    ib, lb = b
    ka, kb = ia[la > tol_set], ib[lb > tol_set]
    np.testing.assert_array_equal(ka, kb)
    np.testing.assert_allclose(la[la > tol_set], lb[lb > tol_set], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("im", [IM2, IM3])
def test_two_tracers_agree_random(orc, im):
    g = np.random.default_rng(5)
    for _ in range(300):
        a = g.uniform(-20, 20, 3)
        b = g.uniform(-20, 20, 3)
        if im["nz"] == 1:
            a[2] = b[2] = g.uniform(-0.4, 0.4)
        _compare(orc.siddon(im, a, b), orc.slabclip(im, a, b))


def test_two_tracers_agree_on_ring_lors(orc):
    w = I.workload("RING2D")
    s, im = w["scanner"], w["image"]
    for a, b in I.workload_lors(w)[::3]:
        p, q = orc.face_point(s, a), orc.face_point(s, b)
        _compare(orc.siddon(im, p, q), orc.slabclip(im, p, q))


def test_quarter_turn_permutes_voxels(orc):
    # R = 8: rotating both crystals by two blocks turns the LOR by 90 degrees,
    # which maps voxel (ix, iy) to (n-1-iy, ix) on a centred square grid.
    w = I.workload("RING2D")
    s, im = w["scanner"], w["image"]
    n = im["nx"]
    Nb = s["nt_block"]
    for a, b in I.workload_lors(w)[::7]:
        if b + 2 * Nb >= 64:
            continue
        i0, l0 = orc.siddon(im, orc.face_point(s, a), orc.face_point(s, b))
        i1, l1 = orc.siddon(im, orc.face_point(s, a + 2 * Nb), orc.face_point(s, b + 2 * Nb))
        m0 = {(n - 1 - (v // n)) + n * (v % n): L for v, L in zip(i0, l0) if L > 1e-9}
        m1 = {v: L for v, L in zip(i1, l1) if L > 1e-9}
        assert m0.keys() == m1.keys()
        for k in m0:
            assert m0[k] == pytest.approx(m1[k], rel=1e-10, abs=1e-12)


@pytest.fixture(scope="module")
def ring2d(orc):
    w = I.workload("RING2D")
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    T, _ = orc.table_build(s, t)
    L = I.workload_lors(w)
    W = orc.spread(s, t, T, L, Wt, Wa)
    G = orc.rows_geom(s, im, L)
    nv = im["nx"] * im["ny"] * im["nz"]
    A = orc.rows_psf_dense(s, L, G, W, Wt, Wa, nv)
    return dict(w=w, T=T, L=L, W=W, G=G, A=A, nv=nv)


def test_rows_match_spread_applied_to_geometric_projection(orc, ring2d):
    # A = S G: forming the rows and applying S after G give the same projector.
    d = ring2d
    s = d["w"]["scanner"]
    x = I.phantom_discs(d["w"]["image"], 0).reshape(-1).astype(np.float64)
    y1 = d["A"] @ x
    y2 = orc.spread_apply(s, d["L"], d["W"], 3, 0, orc.csr_fwd(d["G"], x))
    np.testing.assert_allclose(y1, y2, rtol=1e-12, atol=1e-12)
    r = np.random.default_rng(6).uniform(size=len(d["L"]))
    b1 = d["A"].T @ r
    b2 = orc.csr_back(d["G"], orc.spread_adjoint(s, d["L"], d["W"], 3, 0, r), d["nv"])
    np.testing.assert_allclose(b1, b2, rtol=1e-12, atol=1e-12)


def test_rows_scatter_by_hand(orc, ring2d):
    # One geometric LOR's row, spread by hand over its window, lands on the
    # rows of the neighbouring pairs with the spread weights (Sec. 2.3).
    d = ring2d
    s = d["w"]["scanner"]
    L, W, G = d["L"], d["W"], d["G"]
    pr = orc.pair_row_map(s, L)
    g = 777
    Ag = np.zeros_like(d["A"])
    ptr, col, val = G
    for e1 in range(7):
        for e2 in range(7):
            if W[g, e1, e2] == 0:
                continue
            pair = orc.window_pair(s, L[g, 0], L[g, 1], 3, 0, e1, e2)
            if pair is None:
                continue
            m = pr[pair[0] * 64 + pair[1]]
            Ag[m, col[ptr[g]:ptr[g + 1]]] += W[g, e1, e2] * val[ptr[g]:ptr[g + 1]]
    # compare with the contribution of g alone, obtained from the oracle by
    # zeroing every other LOR's spread
    W1 = np.zeros_like(W)
    W1[g] = W[g]
    A1 = orc.rows_psf_dense(s, L, G, W1, 3, 0, d["nv"])
    np.testing.assert_allclose(A1, Ag, rtol=1e-13, atol=0)


def test_dot_product_identity(orc, ring2d):
    d = ring2d
    g = np.random.default_rng(7)
    ptr = np.zeros(len(d["L"]) + 1, dtype=np.int64)
    nz = d["A"] != 0
    np.cumsum(nz.sum(1), out=ptr[1:])
    rows, cols = np.nonzero(nz)
    Acsr = (ptr, cols.astype(np.int64), d["A"][rows, cols])
    for _ in range(4):
        x = g.uniform(size=d["nv"])
        y = g.uniform(size=len(d["L"]))
        lhs = orc.csr_fwd(Acsr, x) @ y
        rhs = x @ orc.csr_back(Acsr, y, d["nv"])
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_mlem_count_identity(orc, ring2d):
    # MLEM keeps sum_v sens_v x_v^{k+1} = sum_m y_m over LORs seen by the image.
    d = ring2d
    A = d["A"]
    x_true = I.phantom_discs(d["w"]["image"], 0).reshape(-1).astype(np.float64)
    y = A @ x_true
    fwd = lambda x: A @ x
    back = lambda r: A.T @ r
    sens = back(np.ones(len(y)))
    for it in [1, 3]:
        x = orc.mlem(fwd, back, y, d["nv"], it)
        assert (sens * x).sum() == pytest.approx(y[A.sum(1) > 0].sum(), rel=1e-10)


def test_loglik_gradient_by_finite_differences(orc, ring2d):
    d = ring2d
    A = d["A"]
    g = np.random.default_rng(8)
    x = g.uniform(0.5, 1.5, d["nv"])
    y = g.poisson(20.0 * (A @ x) / (A @ x).mean()).astype(np.float64)
    fwd = lambda v: A @ v
    back = lambda r: A.T @ r
    grad = orc.poisson_grad(fwd, back, y, x)
    h = 1e-3
    vox = g.choice(np.nonzero(A.sum(0) > 0)[0], 16, replace=False)
    for v in vox:
        e = np.zeros(d["nv"])
        e[v] = h
        fd = (orc.poisson_loglik(fwd, y, x + e) - orc.poisson_loglik(fwd, y, x - e)) / (2 * h)
        assert fd == pytest.approx(grad[v], rel=1e-5, abs=1e-6 * np.abs(grad).max())
