"""List-mode OSEM on the GPU (psf_event_rows, psf_histogram, the factored
projector; torch_api.listmode_osem) against the oracle's event-by-event
list-mode OSEM, on the small 3D ring with seeded three-sphere events."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import assert_close

pytestmark = pytest.mark.gpu
NAME = "RING3D_SMALL_LM"
N_SUB, ITERS = 4, 2


@pytest.fixture(scope="module")
def P():
    from paper_1607_06170_gb300 import build, psf

    build.build()
    return psf


@pytest.fixture(scope="module")
def ref(orc):
    w = I.workload(NAME)
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    T, _ = orc.table_build(s, t)
    L = I.workload_lors(w)
    ev = I.listmode_events(w, w["listmode"]["events"], w["index"]).numpy()
    nc = I.n_crystals(s)
    rows = orc.pair_row_map(s, L)[ev[:, 0].astype(np.int64) * nc + ev[:, 1]]
    return dict(w=w, L=L, W=orc.spread(s, t, T, L, Wt, Wa), G=orc.rows_geom(s, im, L), ev=ev,
                rows=rows, nv=im["nx"] * im["ny"] * im["nz"])


@pytest.fixture(scope="module")
def gpu(P, ref):
    w = ref["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    WC = P.bin_spread(s, t, T, eta, P.lor_set_classes(s, ls), Wt, Wa)
    G = P.sysmat_rows_set(s, im, ls)
    M = P.Matrix(G[0], G[1], G[2], ref["nv"]).set_spread(s, ls, Wt, Wa, WC)
    rows = P.event_rows(s, ls, torch.from_numpy(ref["ev"]).cuda())
    torch.cuda.synchronize()
    return dict(M=M, rows=rows)


def test_event_rows(gpu, ref):
    np.testing.assert_array_equal(gpu["rows"].cpu().numpy(), ref["rows"])
    assert (ref["rows"] >= 0).all()  # the generator redraws pairs outside the set


def test_event_rows_outside_set(P, ref):
    """Pairs of one crystal, out-of-range ids and pairs beyond the fan or the
    ring difference map to -1; either crystal order maps to the same row."""
    w = ref["w"]
    s, ls = w["scanner"], w["lors"]
    nt, nc = I.n_transaxial(s), I.n_crystals(s)
    a, b = ref["L"][5]
    ev = np.array([[a, b], [b, a], [a, a], [-1, b], [a, nc], [0, 1],
                   [0, (ls["max_ring_diff"] + 1) * nt + nt // 2]], dtype=np.int32)
    rows = P.event_rows(s, ls, torch.from_numpy(ev).cuda()).cpu().numpy()
    assert rows[0] == 5 and rows[1] == 5
    assert (rows[2:] == -1).all()


def test_histogram(P, gpu):
    rows = gpu["rows"]
    n = gpu["M"].n_rows
    c = P.histogram(rows, n, 3.0).cpu().numpy()
    want = 3.0 * np.bincount(rows.cpu().numpy(), minlength=n)
    np.testing.assert_array_equal(c, want.astype(np.float32))
    bad = torch.tensor([-1, n, 0], dtype=torch.int64, device="cuda")
    c2 = P.histogram(bad, n, 1.0).cpu().numpy()
    assert c2[0] == 1.0 and c2.sum() == 1.0


def test_listmode_osem(gpu, ref, orc):
    from paper_1607_06170_gb300.torch_api import listmode_osem

    w = ref["w"]
    s = w["scanner"]
    Wt, Wa = w["window"]
    x = listmode_osem(gpu["M"], gpu["rows"], N_SUB, ITERS).cpu().numpy()

    def fwd(v):
        return orc.spread_apply(s, ref["L"], ref["W"], Wt, Wa, orc.csr_fwd(ref["G"], v))

    def back(r):
        return orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], ref["W"], Wt, Wa, r),
                            ref["nv"])

    xo = orc.listmode_osem(fwd, back, ref["rows"], len(ref["L"]), N_SUB, ITERS)
    rel = float(np.linalg.norm(x - xo) / np.linalg.norm(xo))
    print(f"\nlist-mode OSEM ({N_SUB} subsets x {ITERS}): image rel. L2 vs oracle {rel:.2e}")
    assert rel < 1e-4
    assert_close(x, xo, 1e-3, 1e-4 * xo.max(), "list-mode OSEM image")


def test_forward_masked(P, gpu, ref):
    """A x on the masked rows equals the plain forward there, 0 elsewhere
    (factored plan: the sources are found through S^T of the mask)."""
    M = gpu["M"]
    x = torch.from_numpy(I.random_image(ref["w"]["image"], 77).reshape(-1)).cuda()
    mask = P.histogram(gpu["rows"][:3000], M.n_rows, 1.0)
    y = M.forward_masked(x, mask).cpu().numpy()
    yf = M.forward(x).cpu().numpy()
    on = mask.cpu().numpy() != 0
    assert on.sum() > 100
    assert_close(y[on], yf[on], 1e-6, 1e-7 * yf.max(), "masked forward")
    assert (y[~on] == 0).all()



@pytest.fixture(scope="module")
def traced(P, ref):
    """A plan of the same set whose rows are traced on the fly (no stored G)."""
    w = ref["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    WC = P.bin_spread(s, t, T, eta, P.lor_set_classes(s, ls), Wt, Wa)
    return P.Matrix.traced(s, im, ls).set_spread(s, ls, Wt, Wa, WC)


def test_traced_rows_equal_stored_rows(P, gpu, traced, ref):
    """Forward, back, masked forward and sensitivity of the traced plan against
    the plan over the stored rows of the same set."""
    M, Mt = gpu["M"], traced
    x = torch.from_numpy(I.random_image(ref["w"]["image"], 78).reshape(-1)).cuda()
    r = torch.from_numpy(I.random_lor_values(M.n_rows, 79)).cuda()
    mask = P.histogram(gpu["rows"][:3000], M.n_rows, 1.0)
    for got, want in ((Mt.forward(x), M.forward(x)), (Mt.back(r), M.back(r)),
                      (Mt.forward_masked(x, mask), M.forward_masked(x, mask)),
                      (Mt.sensitivity(), M.sensitivity())):
        torch.testing.assert_close(got, want, rtol=1e-5, atol=1e-6 * want.abs().max().item())
    Mt.check()


def test_listmode_osem_traced_rows(gpu, traced, ref, orc):
    """List-mode OSEM with rows generated on the fly per subset (top-5 spreads,
    the subsets' sources and back-projected rows traced) against the oracle."""
    from paper_1607_06170_gb300 import psf as P
    from paper_1607_06170_gb300.torch_api import listmode_osem

    w = ref["w"]
    s, t, ls = w["scanner"], w["table"], w["lors"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    WC = P.bin_spread(s, t, T, eta, P.lor_set_classes(s, ls), Wt, Wa)
    idx, wt = P.spread_topn(WC, Wt, Wa, 5)
    Mt = traced.set_spread_topn(s, ls, Wt, Wa, idx, wt)
    Ms = P.Matrix(*[a for a in gpu["M"]._keep[:3]], ref["nv"]).set_spread_topn(s, ls, Wt, Wa,
                                                                             idx, wt)
    xt = listmode_osem(Mt, gpu["rows"], N_SUB, ITERS).cpu().numpy()
    xs = listmode_osem(Ms, gpu["rows"], N_SUB, ITERS).cpu().numpy()
    Mt.check()
    # the oracle's list-mode OSEM with the same top-5 class spreads (the GPU's
    # selection, so near-ties rank alike), expanded to every LOR of the list
    E = (2 * Wt + 1) * (2 * Wa + 1)
    idx_h, wt_h = idx.cpu().numpy(), wt.cpu().numpy().astype(np.float64)
    dense = np.zeros((len(idx_h), E * E))
    np.put_along_axis(dense, idx_h.astype(np.int64), wt_h, axis=1)
    Wo5 = dense.reshape(-1, E, E)[_lor_classes(w, ref["L"])]

    def fwd(v):
        return orc.spread_apply(s, ref["L"], Wo5, Wt, Wa, orc.csr_fwd(ref["G"], v))

    def back(r):
        return orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], Wo5, Wt, Wa, r), ref["nv"])

    xo = orc.listmode_osem(fwd, back, ref["rows"], len(ref["L"]), N_SUB, ITERS)
    rel = float(np.linalg.norm(xt - xo) / np.linalg.norm(xo))
    rel_s = float(np.linalg.norm(xt - xs) / np.linalg.norm(xs))
    print(f"\ntraced rows, top-5: image rel. L2 vs oracle {rel:.2e}, vs stored rows {rel_s:.2e}")
    assert rel < 1e-4 and rel_s < 1e-5


def _lor_classes(w, L):
    """Spread class of every LOR of the list (the first crystal rotated into
    block 0 by whole blocks, the ring difference kept), in the set's class
    order: transaxial pairs with the first crystal in block 0, then ring
    differences -Dm..Dm."""
    s, Dm = w["scanner"], w["lors"]["max_ring_diff"]
    nt, nb = I.n_transaxial(s), s["nt_block"]
    tp = I.transaxial_pairs(s, w["lors"]["fan_half"])
    tp = tp[tp[:, 0] < nb]
    index = {(int(a), int(b)): k for k, (a, b) in enumerate(tp)}
    a, ra = L[:, 0] % nt, L[:, 0] // nt
    b, rb = L[:, 1] % nt, L[:, 1] // nt
    a0 = a % nb
    t = np.array([index[(int(x), int(y))] for x, y in zip(a0, b - (a - a0))])
    return t * (2 * Dm + 1) + (rb - ra + Dm)
