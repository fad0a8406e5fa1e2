"""Pins of the oracle's event-by-event list-mode OSEM (the next step named in
Sec. 5; OSEM subsets as in Sec. 3) on the planar ring with its dense PSF
matrix: one subset reduces to MLEM on the event histogram, and every
sub-iteration keeps the EM count identity sum_j (s_j / n_subsets) x_j =
(events of the subset with a positive forward projection)."""
import numpy as np
import pytest

from paper_1607_06170_gb300 import inputs as I


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
    rng = np.random.default_rng(1607)
    # events: rows drawn in proportion to the phantom's projection, plus a few
    # pairs outside the set (-1)
    y = A @ I.phantom_discs(im, 0).reshape(-1).astype(np.float64)
    rows = rng.choice(len(L), size=3000, p=y / y.sum()).astype(np.int64)
    rows[rng.choice(3000, 30, replace=False)] = -1
    return dict(A=A, rows=rows, n_lors=len(L), nv=nv)


def test_one_subset_is_mlem_on_the_histogram(orc, ring2d):
    A, rows = ring2d["A"], ring2d["rows"]
    fwd, back = (lambda v: A @ v), (lambda r: A.T @ r)
    x_lm = orc.listmode_osem(fwd, back, rows, ring2d["n_lors"], 1, 3)
    y = np.bincount(rows[rows >= 0], minlength=ring2d["n_lors"]).astype(np.float64)
    x_ml = orc.mlem(fwd, back, y, ring2d["nv"], 3)
    np.testing.assert_allclose(x_lm, x_ml, rtol=1e-11, atol=1e-12 * x_ml.max())


@pytest.mark.parametrize("n_sub", [2, 5])
def test_subset_count_identity_and_weighting(orc, ring2d, n_sub):
    """A sub-iteration over subset S alone (one subset) gives
    sum_j s_j x_j = #{e in S : (A x)_e > 0}; with n_sub subsets each
    sub-iteration is n_sub times that update (sensitivity s / n_sub)."""
    A, rows = ring2d["A"], ring2d["rows"]
    fwd, back = (lambda v: A @ v), (lambda r: A.T @ r)
    sens = back(np.ones(ring2d["n_lors"]))
    live = sens >= 1e-12 * sens.max()
    x = np.where(live, 1.0, 0.0)
    n_ev = len(rows)
    for j in range(n_sub):
        sub = rows[n_ev * j // n_sub: n_ev * (j + 1) // n_sub]
        yh = fwd(x)
        expect = sum(1 for m in sub if m >= 0 and yh[m] > 0)
        x1 = orc.listmode_osem(fwd, back, sub, ring2d["n_lors"], 1, 1, x0=x)
        assert np.sum(sens * x1) == pytest.approx(expect, rel=1e-10)
        x = n_sub * x1
    x_all = orc.listmode_osem(fwd, back, rows, ring2d["n_lors"], n_sub, 1)
    np.testing.assert_allclose(x_all, x, rtol=1e-11, atol=1e-13 * x.max())


def test_event_order_within_a_subset(orc, ring2d):
    A, rows = ring2d["A"], ring2d["rows"]
    fwd, back = (lambda v: A @ v), (lambda r: A.T @ r)
    perm = np.random.default_rng(3).permutation(len(rows))
    # permuting events inside each of 3 subsets changes nothing
    n = len(rows)
    b = [n * j // 3 for j in range(4)]
    shuffled = np.concatenate([rows[b[j]:b[j + 1]][np.argsort(perm[b[j]:b[j + 1]])]
                               for j in range(3)])
    x1 = orc.listmode_osem(fwd, back, rows, ring2d["n_lors"], 3, 2)
    x2 = orc.listmode_osem(fwd, back, shuffled, ring2d["n_lors"], 3, 2)
    np.testing.assert_allclose(x1, x2, rtol=1e-12, atol=1e-14 * x1.max())
