"""Pins of the oracle's top-N truncation of a LOR's spread (Sec. 4.3, Table 3:
the extended bins kept in descending order of proportion, up to N), with the
readings stated in the oracle: ranking over the whole window, ties to the
smaller offset |dt1|+|da1|+|dt2|+|da2| and then the lower window index, kept
weights rescaled to the untruncated window total."""
import numpy as np
import pytest

from paper_1607_06170_gb300 import inputs as I


def _dist(Wt, Wa):
    """|dt1|+|da1|+|dt2|+|da2| of every window index e1*E + e2."""
    W2a = 2 * Wa + 1
    E = (2 * Wt + 1) * W2a
    e1, e2 = np.divmod(np.arange(E * E), E)
    off = lambda e: np.abs(e // W2a - Wt) + np.abs(e % W2a - Wa)
    return off(e1) + off(e2)


def _brute_order(w, Wt, Wa):
    """Rank order by an independent route: a stable lexicographic sort."""
    e = np.arange(w.size)
    return np.lexsort((e, _dist(Wt, Wa), -np.maximum(w, 0.0)))


@pytest.mark.parametrize("Wt,Wa,N", [(3, 3, 1), (3, 3, 25), (2, 1, 7), (1, 1, 81), (3, 0, 10)])
def test_topn_matches_brute_order_and_sum(orc, Wt, Wa, N):
    E = (2 * Wt + 1) * (2 * Wa + 1)
    rng = np.random.default_rng(160706 + N)
    # FP32-representable weights with many exact ties (a few distinct levels)
    w = (rng.integers(0, 6, size=(5, E, E)) / 8.0).astype(np.float32).astype(np.float64)
    out, idx = orc.spread_topn(w, Wt, Wa, N)
    for g in range(w.shape[0]):
        order = _brute_order(w[g].reshape(-1), Wt, Wa)
        np.testing.assert_array_equal(idx[g], order[:N])
        kept = np.zeros(E * E, bool)
        kept[order[:N]] = True
        o = out[g].reshape(-1)
        assert np.all(o[~kept] == 0.0)
        # rescaled to the untruncated total (or left as is when nothing is kept)
        tot, ks = w[g].sum(), w[g].reshape(-1)[kept].sum()
        if ks > 0:
            assert o.sum() == pytest.approx(tot, rel=1e-13)
            np.testing.assert_allclose(o[kept], w[g].reshape(-1)[kept] * (tot / ks), rtol=1e-14)
        else:
            assert np.all(o == 0.0)


def test_full_window_is_identity(orc):
    Wt, Wa = 3, 3
    E = (2 * Wt + 1) * (2 * Wa + 1)
    w = np.random.default_rng(7).random((4, E, E))
    out, idx = orc.spread_topn(w, Wt, Wa, E * E)
    np.testing.assert_allclose(out, w, rtol=1e-13)
    assert sorted(idx[0].tolist()) == list(range(E * E))


def test_tie_rules(orc):
    Wt = Wa = 1
    E = 9
    w = np.ones((1, E, E))
    _, idx = orc.spread_topn(w, Wt, Wa, 5)
    # all weights equal: the centre (no offset) first, then the four
    # one-offset entries by index: e1 = 4 with e2 in {1, 3, 5, 7}, ... e1 in {1, 3}
    d = _dist(Wt, Wa)
    assert idx[0, 0] == 4 * E + 4 and d[idx[0, 0]] == 0
    assert all(d[i] == 1 for i in idx[0, 1:])
    assert list(idx[0, 1:]) == sorted(idx[0, 1:])
    assert idx[0, 1] == 1 * E + 4  # the lowest index with one unit of offset
    # a larger weight beats any offset; a negative weight ranks as zero
    w2 = np.zeros((1, E, E))
    w2[0, 0, 0] = 0.5   # offset 4
    w2[0, 4, 4] = -1.0  # centre, negative
    _, idx2 = orc.spread_topn(w2, Wt, Wa, 2)
    assert idx2[0, 0] == 0
    assert idx2[0, 1] == 4 * E + 4  # zero-weight entries by offset: the centre next


def test_real_spreads_keep_the_largest(orc):
    """On oracle spreads of the planar ring: the kept weights are the N largest
    and the window total is unchanged."""
    w = I.workload("RING2D")
    s, t = w["scanner"], w["table"]
    Wt, Wa = w["window"]
    T, _ = orc.table_build(s, t)
    L = I.workload_lors(w)[:40]
    W = orc.spread(s, t, T, L, Wt, Wa).astype(np.float32).astype(np.float64)
    N = 5
    out, idx = orc.spread_topn(W, Wt, Wa, N)
    for g in range(W.shape[0]):
        wg = W[g].reshape(-1)
        thr = np.sort(wg)[::-1][N - 1]
        assert np.all(wg[idx[g]] >= thr)
        assert np.sum(wg > thr) <= N
        assert out[g].sum() == pytest.approx(wg.sum(), rel=1e-12)


def test_topn_bf16_matches_library_rounding(orc):
    """The oracle's BF16 storage of top-N weights: its codes equal torch's
    round-to-nearest-even conversion of the same FP32 quotients (a library
    routine), ties included, and code x scale reproduces each weight within
    half a BF16 unit (at most 2^-8 of it)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4242)
    w = rng.random((300, 5)).astype(np.float32) * rng.choice([1e-6, 1e-2, 1.0, 30.0], (300, 1))
    w[7] = 0.0  # an all-zero row keeps scale 1
    w[11, 1:] = w[11, 0]  # equal weights
    # a row whose largest weight is 1 (quotients = weights) with values exactly
    # between two BF16 numbers: ties to the even code, down and up
    w[20] = np.array([1.0, 0.5 + 2.0 ** -9, 0.5 + 3 * 2.0 ** -9, 0.25 + 2.0 ** -10, 0.75],
                     dtype=np.float32)
    codes, sc, deq = orc.topn_bf16(w)
    q = w / np.where(np.abs(w).max(1) > 0, np.abs(w).max(1), 1.0).astype(np.float32)[:, None]
    want = torch.from_numpy(q.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy()
    np.testing.assert_array_equal(codes.view(np.int16), want)
    assert sc[7] == 1.0 and (deq[7] == 0).all()
    np.testing.assert_array_equal(codes[20], [0x3F80, 0x3F00, 0x3F02, 0x3E80, 0x3F40])
    nz = w != 0
    assert (np.abs(deq[nz] - w[nz]) <= 2.0 ** -8 * np.abs(w[nz]) * (1 + 1e-6)).all()
