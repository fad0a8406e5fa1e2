"""GPU parity on the planar ring (8 blocks x 8 crystals, 2016 LORs, 64 x 64
image): every stage of the hot path through the C ABI against the FP64
oracle, element by element."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import SPREAD_ATOL_REL, assert_close, compare_chord_rows

pytestmark = pytest.mark.gpu

MARGIN = 1e-5  # LORs with a rounding decision closer than this have several correct spreads


@pytest.fixture(scope="module")
def P():
    from paper_1607_06170_gb300 import build, psf

    build.build()
    assert torch.cuda.is_available()
    return psf


def _oracle(orc, name):
    w = I.workload(name)
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    T, eta = orc.table_build(s, t)
    L = I.workload_lors(w)
    out = dict(w=w, T=T, eta=eta, L=L, Wt=Wt, Wa=Wa)
    out["margin"] = orc.tie_margin(s, t, T, L)
    out["W"] = {n: orc.spread(s, t, T, L, Wt, Wa, n) for n in (0, 1, 2)}
    out["G"] = orc.rows_geom(s, im, L)
    out["nv"] = im["nx"] * im["ny"] * im["nz"]
    return out


def _gpu(P, name):
    w = I.workload(name)
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    L = torch.from_numpy(I.workload_lors(w)).cuda()
    W = {n: P.bin_spread(s, t, T, eta, L, Wt, Wa, n) for n in (0, 1, 2)}
    G = P.sysmat_rows(s, im, L)
    A = P.sysmat_rows(s, im, L, W[1], Wt, Wa)
    torch.cuda.synchronize()
    return dict(T=T, eta=eta, L=L, W=W, G=G, A=A)


@pytest.fixture(scope="module", params=["RING2D", "RING2D_NARROW"])
def both(request, P, orc):
    return request.param, _oracle(orc, request.param), _gpu(P, request.param)


def test_response_table(both):
    name, o, g = both
    assert_close(g["T"].cpu().numpy(), o["T"], 1e-5, 1e-7, f"{name} table")
    # FP64 prefix sums: last slot is the counting rate eta of Eq. 6
    e = g["eta"].cpu().numpy()
    assert_close(e[..., -1], o["eta"], 1e-6, 1e-12, "eta")
    pref = np.concatenate([np.zeros(o["T"].shape[:4] + (1,)),
                           np.cumsum(o["T"].sum(-1), axis=-1)], axis=-1)
    assert_close(e, pref, 1e-6, 1e-12, "eta prefix")


def test_spread_all_norms(both):
    name, o, g = both
    ok = o["margin"] >= MARGIN
    assert ok.mean() > 0.99
    for n in (0, 1, 2):
        got = g["W"][n].cpu().numpy()[ok]
        ref = o["W"][n][ok]
        scale = np.abs(ref).reshape(len(ref), -1).max(1)[:, None, None]
        assert_close(got, ref, 1e-5, SPREAD_ATOL_REL * scale + 1e-30, f"{name} spread norm {n}")


def test_geometric_rows(both):
    name, o, g = both
    ptr, col, val = [a.cpu().numpy() for a in g["G"][:3]]
    err, n = compare_chord_rows((ptr, col, val), o["G"], o["nv"])
    assert n > 1000


def test_set_rows_equal_list_rows(both, P):
    name, o, g = both
    w = I.workload(name)
    rp, col, val = P.sysmat_rows_set(w["scanner"], w["image"], w["lors"])
    torch.cuda.synchronize()
    assert torch.equal(rp, g["G"][0]) and torch.equal(col, g["G"][1])
    assert torch.equal(val, g["G"][2])


def test_psf_rows_and_projectors(both, orc):
    # A row receives the spreads of every LOR whose window lands on it; a LOR
    # with a rounding decision within MARGIN of its boundary has several
    # correct spreads, so the rows it reaches (through a nonempty geometric
    # row) are left out and counted.
    name, o, g = both
    s = o["w"]["scanner"]
    A = orc.rows_psf_dense(s, o["L"], o["G"], o["W"][1], o["Wt"], o["Wa"], o["nv"])
    amb = o["margin"] < MARGIN
    E = (2 * o["Wt"] + 1) * (2 * o["Wa"] + 1)
    reach = orc.rows_psf_dense(s, o["L"], o["G"], np.broadcast_to(
        amb[:, None, None].astype(np.float64), (len(o["L"]), E, E)).copy(), o["Wt"], o["Wa"],
        o["nv"])
    keep = ~(reach != 0).any(1)
    print(f"{name}: {amb.sum()} tie LORs, {(~keep).sum()} of {len(keep)} PSF rows left out")
    assert keep.mean() > 0.9
    ptr, col, val, _ = g["A"]
    ptr, col, val = ptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    Ag = np.zeros_like(A)
    rows = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    Ag[rows, col] = val
    wsum = o["W"][1].reshape(len(o["L"]), -1).sum(1)   # weight landing scale per row
    floor = 1e-6 * np.maximum(wsum, wsum.max() * 1e-3)[:, None]
    assert_close(Ag[keep], A[keep], 1e-4, floor[keep], f"{name} PSF rows")
    # sparsity: entries above the floor agree
    assert np.array_equal(Ag[keep] > 2 * floor[keep], A[keep] > 2 * floor[keep])
    # columns ascending within rows
    assert all(np.all(np.diff(col[ptr[i]:ptr[i + 1]]) > 0) for i in range(len(ptr) - 1))


def test_projectors_and_mlem(P, orc):
    w = I.workload("RING2D")
    o = _oracle(orc, "RING2D")
    g = _gpu(P, "RING2D")
    s = w["scanner"]
    A = orc.rows_psf_dense(s, o["L"], o["G"], o["W"][1], 3, 0, o["nv"])
    ptr, col, val, _ = g["A"]
    M = P.Matrix(ptr, col, val, o["nv"])
    x = I.phantom_discs(w["image"], 0).reshape(-1)
    xt = torch.from_numpy(x).cuda()
    y = M.forward(xt)
    yo = A @ x.astype(np.float64)
    assert_close(y.cpu().numpy(), yo, 1e-4, 1e-6 * yo.max(), "forward")
    r = torch.from_numpy(I.random_lor_values(len(o["L"]), 100)).cuda()
    b = M.back(r)
    bo = A.T @ r.cpu().numpy().astype(np.float64)
    assert_close(b.cpu().numpy(), bo, 1e-4, 1e-6 * bo.max(), "back")
    # adjointness on the GPU (FP64 final reductions)
    for k in range(4):
        xk = torch.from_numpy(I.random_image(w["image"], 200 + k).reshape(-1)).cuda()
        yk = torch.from_numpy(I.random_lor_values(len(o["L"]), 300 + k)).cuda()
        lhs = torch.dot(M.forward(xk).double(), yk.double()).item()
        rhs = torch.dot(xk.double(), M.back(yk).double()).item()
        assert lhs == pytest.approx(rhs, rel=1e-5)
    # 10 MLEM iterations through the library's projector and EM kernels
    from paper_1607_06170_gb300.torch_api import mlem

    yt = torch.from_numpy(yo.astype(np.float32)).cuda()
    xg = mlem(M, yt, iters=10).cpu().numpy().astype(np.float64)
    xo = orc.mlem(lambda v: A @ v, lambda q: A.T @ q, yo, o["nv"], 10)
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert rel < 1e-4, rel


def test_back_sens_stored_rows(P):
    """Stored-row plans: one pass gives A^T y and A^T 1."""
    w = I.workload("RING2D")
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    L = torch.from_numpy(I.workload_lors(w)).cuda()
    Wg = P.bin_spread(s, t, T, eta, L, Wt, Wa)
    ptr, col, val, _ = P.sysmat_rows(s, im, L, Wg, Wt, Wa)
    M = P.Matrix(ptr, col, val, im["nx"] * im["ny"] * im["nz"])
    r = torch.from_numpy(I.random_lor_values(M.n_rows, 909)).cuda()
    x, sens = M.back_sens(r)
    torch.testing.assert_close(x, M.back(r), rtol=1e-5, atol=1e-6 * x.abs().max().item())
    ones = torch.ones(M.n_rows, device="cuda")
    torch.testing.assert_close(sens, M.back(ones), rtol=1e-5, atol=1e-6 * sens.abs().max().item())
