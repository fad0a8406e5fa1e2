"""Top-N truncated spreads (Sec. 4.3, Table 3) on the GPU against the FP64
oracle: the selection (psf_spread_topn) and the factored projector with top-N
class spreads (psf_matrix_set_spread_topn).

Both sides rank the same FP32 spreads (the oracle's class spreads rounded to
FP32, or seeded FP32 arrays with many exact ties), so the kept index sets
must agree exactly; the rescaled weights agree to FP32 rounding."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import assert_close

pytestmark = pytest.mark.gpu
NAME = "RING3D_SMALL"


@pytest.fixture(scope="module")
def P():
    from paper_1607_06170_gb300 import build, psf

    build.build()
    return psf


def _class_lors(w):
    """One representative LOR per spread class, in class order (transaxial
    pairs with a in block 0, then ring differences -Dm..Dm)."""
    s, Dm = w["scanner"], w["lors"]["max_ring_diff"]
    nt = I.n_transaxial(s)
    tp = I.transaxial_pairs(s, w["lors"]["fan_half"])
    tp = tp[tp[:, 0] < s["nt_block"]]
    out = []
    for a, b in tp:
        for d in range(-Dm, Dm + 1):
            ra = max(0, -d)
            out.append((ra * nt + a, (ra + d) * nt + b))
    return np.array(out, dtype=np.int32), {(int(a), int(b)): k for k, (a, b) in enumerate(tp)}


def _lor_classes(w, L, tp_index):
    """Class index of every LOR of the list: block rotation of the first
    crystal into block 0, ring difference."""
    s, Dm = w["scanner"], w["lors"]["max_ring_diff"]
    nt, nb = I.n_transaxial(s), s["nt_block"]
    a, ra = L[:, 0] % nt, L[:, 0] // nt
    b, rb = L[:, 1] % nt, L[:, 1] // nt
    a0 = a % nb
    b0 = b - (a - a0)
    t = np.array([tp_index[(int(x), int(y))] for x, y in zip(a0, b0)])
    return t * (2 * Dm + 1) + (rb - ra + Dm)


@pytest.fixture(scope="module")
def ref(orc):
    w = I.workload(NAME)
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    T, _ = orc.table_build(s, t)
    C, tp_index = _class_lors(w)
    WC = orc.spread(s, t, T, C, Wt, Wa).astype(np.float32)  # the shared FP32 input
    L = I.workload_lors(w)
    return dict(w=w, WC=WC, L=L, cls=_lor_classes(w, L, tp_index), G=orc.rows_geom(s, im, L),
                nv=im["nx"] * im["ny"] * im["nz"])


@pytest.mark.parametrize("N", [1, 5, 25, 64])
def test_selection_class_spreads(P, ref, orc, N):
    Wt, Wa = ref["w"]["window"]
    idx, wk = P.spread_topn(torch.from_numpy(ref["WC"]).cuda(), Wt, Wa, N)
    out_o, idx_o = orc.spread_topn(ref["WC"].astype(np.float64), Wt, Wa, N)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    wo = np.take_along_axis(out_o.reshape(len(idx_o), -1), idx_o.astype(np.int64), 1)
    assert_close(wk.cpu().numpy(), wo, 2e-7, 1e-30, f"top-{N} weights")


@pytest.mark.parametrize("Wt,Wa,N", [(3, 3, 64), (2, 1, 10), (1, 3, 7), (3, 0, 49)])
def test_selection_ties(P, orc, Wt, Wa, N):
    """Seeded FP32 spreads with many exact ties (and some negative entries):
    the tie rules decide most picks."""
    E = (2 * Wt + 1) * (2 * Wa + 1)
    rng = np.random.default_rng(1607 + N)
    w = (rng.integers(-1, 5, size=(300, E, E)) / 4.0).astype(np.float32)
    idx, wk = P.spread_topn(torch.from_numpy(w).cuda(), Wt, Wa, N)
    out_o, idx_o = orc.spread_topn(w.astype(np.float64), Wt, Wa, N)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    wo = np.take_along_axis(out_o.reshape(len(idx_o), -1), idx_o.astype(np.int64), 1)
    assert_close(wk.cpu().numpy(), wo, 2e-7, 1e-30, "tied weights")


def test_selection_limits(P):
    w = torch.zeros((2, 49, 49), device="cuda")
    from paper_1607_06170_gb300.psf import PSFError

    for bad in (0, 65):
        with pytest.raises(PSFError):
            P.spread_topn(w, 3, 3, bad)
    with pytest.raises(PSFError):  # more entries kept than the window has
        P.spread_topn(torch.zeros((2, 1, 1), device="cuda"), 0, 0, 2)
    idx, wk = P.spread_topn(torch.zeros((0, 49, 49), device="cuda"), 3, 3, 5)
    assert idx.shape == (0, 5) and wk.shape == (0, 5)


@pytest.fixture(scope="module")
def plan(P, ref):
    w = ref["w"]
    s, im, ls = w["scanner"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    G = P.sysmat_rows_set(s, im, ls)
    return G


@pytest.mark.parametrize("N", [5, 64])
def test_topn_projector(P, ref, orc, plan, N):
    w = ref["w"]
    s, ls = w["scanner"], w["lors"]
    Wt, Wa = w["window"]
    E = (2 * Wt + 1) * (2 * Wa + 1)
    idx, wk = P.spread_topn(torch.from_numpy(ref["WC"]).cuda(), Wt, Wa, N)
    M = P.Matrix(plan[0], plan[1], plan[2], ref["nv"]).set_spread_topn(s, ls, Wt, Wa, idx, wk)
    # oracle: truncated class spreads, each LOR taking its class's
    out_o, _ = orc.spread_topn(ref["WC"].astype(np.float64), Wt, Wa, N)
    Wl = out_o[ref["cls"]]
    assert Wl.shape == (len(ref["L"]), E, E)
    x = I.random_image(w["image"], 910).reshape(-1)
    y = M.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.spread_apply(s, ref["L"], Wl, Wt, Wa, orc.csr_fwd(ref["G"], x))
    assert_close(y, yo, 2e-5, 1e-6 * yo.max(), f"top-{N} forward")
    r = I.random_lor_values(len(ref["L"]), 911)
    b = M.back(torch.from_numpy(r).cuda()).cpu().numpy()
    bo = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], Wl, Wt, Wa, r), ref["nv"])
    assert_close(b, bo, 2e-5, 1e-6 * bo.max(), f"top-{N} back")
    ones = np.ones(len(ref["L"]))
    so = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], Wl, Wt, Wa, ones), ref["nv"])
    sens = M.sensitivity().cpu().numpy()
    assert_close(sens, so, 2e-5, 1e-6 * so.max(), f"top-{N} sensitivity")
    xb, sb = M.back_sens(torch.from_numpy(r).cuda())
    assert_close(xb.cpu().numpy(), bo, 2e-5, 1e-6 * bo.max(), f"top-{N} back (pair pass)")
    assert_close(sb.cpu().numpy(), so, 2e-5, 1e-6 * so.max(), f"top-{N} sensitivity (pair pass)")
    # a sparse LOR vector (1 % nonzero, as one list-mode subset's counts): the
    # adjoint reads only the occupied entries
    rs = np.where(np.random.default_rng(912).random(len(ref["L"])) < 0.01, r, 0.0)
    assert 0 < np.count_nonzero(rs) <= len(rs) // 16
    bs = M.back(torch.from_numpy(rs.astype(np.float32)).cuda()).cpu().numpy()
    bso = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], Wl, Wt, Wa, rs), ref["nv"])
    assert_close(bs, bso, 2e-5, 1e-6 * bso.max(), f"top-{N} back of a sparse vector")
    # with the transpose of S: sparse inputs scatter from their nonzero entries,
    # dense ones keep the gather
    M.build_sparse_adjoint()
    bs2 = M.back(torch.from_numpy(rs.astype(np.float32)).cuda()).cpu().numpy()
    assert_close(bs2, bso, 2e-5, 1e-6 * bso.max(), f"top-{N} back of a sparse vector (transpose)")
    b2 = M.back(torch.from_numpy(r).cuda()).cpu().numpy()
    assert_close(b2, bo, 2e-5, 1e-6 * bo.max(), f"top-{N} back (transpose built)")
    xb2, sb2 = M.back_sens(torch.from_numpy(rs.astype(np.float32)).cuda())
    assert_close(xb2.cpu().numpy(), bso, 2e-5, 1e-6 * bso.max(), f"top-{N} pair pass, sparse")
    assert_close(sb2.cpu().numpy(), so, 2e-5, 1e-6 * so.max(), f"top-{N} pair pass sensitivity")
    xt = torch.from_numpy(x).cuda()
    mask = torch.from_numpy((rs != 0).astype(np.float32)).cuda()
    ym = M.forward_masked(xt, mask).cpu().numpy()
    assert_close(ym, np.where(rs != 0, yo, 0.0), 2e-5, 1e-6 * yo.max(),
                 f"top-{N} masked forward (transpose)")
    M.check()
    for k in range(3):
        xk = torch.from_numpy(I.random_image(w["image"], 920 + k).reshape(-1)).cuda()
        yk = torch.from_numpy(I.random_lor_values(len(ref["L"]), 930 + k)).cuda()
        lhs = torch.dot(M.forward(xk).double(), yk.double()).item()
        rhs = torch.dot(xk.double(), M.back(yk).double()).item()
        assert lhs == pytest.approx(rhs, rel=1e-5)


def test_topn_bf16_codes(P, orc):
    """psf_spread_topn_bf16 against the oracle's BF16 storage form on the same
    seeded FP32 weights: codes and scales bit-equal."""
    rng = I.rng(4343)
    w = (rng.random((2000, 5)) * rng.choice([1e-5, 1e-2, 1.0], (2000, 1))).astype(np.float32)
    w[3] = 0.0
    w16, sc = P.spread_topn_bf16(torch.from_numpy(w).cuda())
    codes, sco, _ = orc.topn_bf16(w)
    np.testing.assert_array_equal(w16.cpu().view(torch.int16).numpy(), codes.view(np.int16))
    np.testing.assert_array_equal(sc.cpu().numpy(), sco)


@pytest.mark.parametrize("N", [5, 25])
def test_topn_projector_bf16(P, ref, orc, plan, N):
    """The factored projector with BF16 top-N weights (one FP32 scale per
    class, FP32 products and sums) against the oracle with its own top-N
    weights in the same storage form (dequantized in FP64)."""
    w = ref["w"]
    s, ls = w["scanner"], w["lors"]
    Wt, Wa = w["window"]
    E = (2 * Wt + 1) * (2 * Wa + 1)
    idx, wk = P.spread_topn(torch.from_numpy(ref["WC"]).cuda(), Wt, Wa, N)
    w16, sc = P.spread_topn_bf16(wk)
    M = P.Matrix(plan[0], plan[1], plan[2], ref["nv"]).set_spread_topn(s, ls, Wt, Wa, idx, w16,
                                                                       scale=sc)
    out_o, idx_o = orc.spread_topn(ref["WC"].astype(np.float64), Wt, Wa, N)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    flat = out_o.reshape(len(idx_o), E * E)
    _, _, deq = orc.topn_bf16(np.take_along_axis(flat, idx_o.astype(np.int64), 1))
    Wq = np.zeros_like(flat)
    np.put_along_axis(Wq, idx_o.astype(np.int64), deq, 1)
    Wl = Wq.reshape(-1, E, E)[ref["cls"]]
    x = I.random_image(w["image"], 950).reshape(-1)
    y = M.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.spread_apply(s, ref["L"], Wl, Wt, Wa, orc.csr_fwd(ref["G"], x))
    assert_close(y, yo, 2e-5, 1e-6 * yo.max(), f"top-{N} BF16 forward")
    r = I.random_lor_values(len(ref["L"]), 951)
    b = M.back(torch.from_numpy(r).cuda()).cpu().numpy()
    bo = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], Wl, Wt, Wa, r), ref["nv"])
    assert_close(b, bo, 2e-5, 1e-6 * bo.max(), f"top-{N} BF16 back")
    ones = np.ones(len(ref["L"]))
    so = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], Wl, Wt, Wa, ones), ref["nv"])
    assert_close(M.sensitivity().cpu().numpy(), so, 2e-5, 1e-6 * so.max(),
                 f"top-{N} BF16 sensitivity")
    M.build_sparse_adjoint()
    rs = np.where(np.random.default_rng(952).random(len(ref["L"])) < 0.01, r, 0.0)
    bs = M.back(torch.from_numpy(rs.astype(np.float32)).cuda()).cpu().numpy()
    bso = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], Wl, Wt, Wa, rs), ref["nv"])
    assert_close(bs, bso, 2e-5, 1e-6 * bso.max(), f"top-{N} BF16 sparse back (transpose)")


def test_listmode_osem_topn_bf16(P, orc):
    """List-mode OSEM (the list-mode step after Sec. 5) with BF16 top-5 class
    weights against the oracle's event-by-event list-mode OSEM with the same
    weights in the same storage form, on the small list-mode ring; both sides
    rank the oracle's class spreads rounded to FP32."""
    from paper_1607_06170_gb300.torch_api import listmode_osem

    w = I.workload("RING3D_SMALL_LM")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    E = (2 * Wt + 1) * (2 * Wa + 1)
    Nk = w["listmode"]["n_keep"]
    n_sub, iters = 4, 2
    T, _ = orc.table_build(s, t)
    C, tp_index = _class_lors(w)
    WC = orc.spread(s, t, T, C, Wt, Wa).astype(np.float32)
    L = I.workload_lors(w)
    cls = _lor_classes(w, L, tp_index)
    G = orc.rows_geom(s, im, L)
    nv = im["nx"] * im["ny"] * im["nz"]
    ev = I.listmode_events(w, w["listmode"]["events"], w["index"]).numpy()
    nc = I.n_crystals(s)
    rows_o = orc.pair_row_map(s, L)[ev[:, 0].astype(np.int64) * nc + ev[:, 1]]
    # oracle weights: its top-N of the FP32 class spreads in BF16 storage form
    out_o, idx_o = orc.spread_topn(WC.astype(np.float64), Wt, Wa, Nk)
    flat = out_o.reshape(len(idx_o), E * E)
    _, _, deq = orc.topn_bf16(np.take_along_axis(flat, idx_o.astype(np.int64), 1))
    Wq = np.zeros_like(flat)
    np.put_along_axis(Wq, idx_o.astype(np.int64), deq, 1)
    Wl = Wq.reshape(-1, E, E)[cls]

    def fwd(v):
        return orc.spread_apply(s, L, Wl, Wt, Wa, orc.csr_fwd(G, v))

    def back(r):
        return orc.csr_back(G, orc.spread_adjoint(s, L, Wl, Wt, Wa, r), nv)

    xo = orc.listmode_osem(fwd, back, rows_o, len(L), n_sub, iters)
    Gd = P.sysmat_rows_set(s, im, ls)
    idx, wk = P.spread_topn(torch.from_numpy(WC).cuda(), Wt, Wa, Nk)
    w16, sc = P.spread_topn_bf16(wk)
    M = P.Matrix(Gd[0], Gd[1], Gd[2], nv).set_spread_topn(s, ls, Wt, Wa, idx, w16, scale=sc)
    M.build_sparse_adjoint()
    rows = P.event_rows(s, ls, torch.from_numpy(ev).cuda())
    np.testing.assert_array_equal(rows.cpu().numpy(), rows_o)
    x = listmode_osem(M, rows, n_sub, iters).cpu().numpy()
    rel = float(np.linalg.norm(x - xo) / np.linalg.norm(xo))
    print(f"\nlist-mode OSEM, BF16 top-{Nk} ({n_sub} subsets x {iters}): image rel. L2 vs "
          f"oracle {rel:.2e}")
    assert rel < 1e-4
    assert_close(x, xo, 1e-3, 1e-4 * xo.max(), "list-mode OSEM image (BF16 top-N)")
