"""Pins of the oracle's voxel-driven homogenization (Sec. 2.3, Eq. 11-12,
Figs. 7-8) on the planar ring: the quarter-turn and mirror symmetries of the
scanner map the matrix onto itself, every column is a sub-probability, and the
matrix converges as the number of lines k grows."""
import numpy as np
import pytest

from paper_1607_06170_gb300 import inputs as I

K = 60  # 3 degree steps: no line meets a node boundary of this table exactly


@pytest.fixture(scope="module")
def ring2d(orc):
    w = I.workload("RING2D")
    s, t, im = w["scanner"], w["table"], w["image"]
    T, _ = orc.table_build(s, t)
    L = I.workload_lors(w)
    A, margin = orc.voxel_homog(s, t, T, im, L, K, w["window"][0])
    return dict(w=w, T=T, L=L, A=A, margin=margin, pr=orc.pair_row_map(s, L))


def _permuted(ring2d, cmap, pmap):
    """A with its rows and columns permuted by a crystal map and a pixel map."""
    L, pr, A = ring2d["L"], ring2d["pr"], ring2d["A"]
    nc = I.n_crystals(ring2d["w"]["scanner"])
    rows = pr[cmap[L[:, 0]].astype(np.int64) * nc + cmap[L[:, 1]]]
    assert (rows >= 0).all()
    B = np.zeros_like(A)
    B[np.ix_(rows, pmap)] = A
    return B


def test_margins(ring2d):
    assert ring2d["margin"].min() > 1e-5


def test_quarter_turn(ring2d):
    s, im = ring2d["w"]["scanner"], ring2d["w"]["image"]
    nt, nx, ny = I.n_transaxial(s), im["nx"], im["ny"]
    assert s["n_blocks"] % 4 == 0 and nx == ny
    cmap = (np.arange(nt) + nt // 4) % nt  # two blocks = 90 degrees
    iy, ix = np.divmod(np.arange(nx * ny), nx)
    pmap = ix * nx + (nx - 1 - iy)  # (x, y) -> (-y, x)
    B = _permuted(ring2d, cmap, pmap)
    np.testing.assert_allclose(B, ring2d["A"], rtol=1e-11, atol=1e-14)


def test_mirror(ring2d):
    s, im = ring2d["w"]["scanner"], ring2d["w"]["image"]
    R, nb, nx, ny = s["n_blocks"], s["nt_block"], im["nx"], im["ny"]
    b, i = np.divmod(np.arange(R * nb), nb)
    cmap = ((R - b) % R) * nb + (nb - 1 - i)  # reflection in the x axis
    iy, ix = np.divmod(np.arange(nx * ny), nx)
    pmap = (ny - 1 - iy) * nx + ix
    B = _permuted(ring2d, cmap, pmap)
    np.testing.assert_allclose(B, ring2d["A"], rtol=1e-11, atol=1e-14)


def test_columns_are_sub_probabilities(ring2d):
    A = ring2d["A"]
    assert (A >= 0).all()
    col = A.sum(0)
    assert col.max() <= 1.0
    assert col.min() > 0.0  # every pixel of this image is seen by some line


def test_converges_with_k(orc, ring2d):
    """The projection of the disc phantom settles as k grows (Sec. 2.3: the
    result approaches a steady state): its change halves at least from k to 4k
    toward k = 3840."""
    w = ring2d["w"]
    s, t, im = w["scanner"], w["table"], w["image"]
    x = I.phantom_discs(im, 0).reshape(-1).astype(np.float64)
    ys = {k: orc.voxel_homog(s, t, ring2d["T"], im, ring2d["L"], k, w["window"][0])[0] @ x
          for k in (60, 240, 960, 3840)}
    ref = ys[3840]
    d = [np.linalg.norm(ys[k] - ref) / np.linalg.norm(ref) for k in (60, 240, 960)]
    assert d[2] < 0.5 * d[1] < 0.25 * d[0]
    assert d[2] < 0.05
