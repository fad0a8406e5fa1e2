"""GPU parity on a small 3D ring (12 blocks x 4 x 4 crystals x 2 block rings,
22176 LORs): table, class spreads, chord rows and the factored PSF projector
A = S G against the FP64 oracle (which uses one spread per LOR, no classes)."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import SPREAD_ATOL_REL, assert_close, compare_chord_rows

pytestmark = pytest.mark.gpu
NAME = "RING3D_SMALL"


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
    T, eta = orc.table_build(s, t)
    L = I.workload_lors(w)
    W = orc.spread(s, t, T, L, Wt, Wa)
    G = orc.rows_geom(s, im, L)
    return dict(w=w, T=T, eta=eta, L=L, W=W, G=G, nv=im["nx"] * im["ny"] * im["nz"],
                margin=orc.tie_margin(s, t, T, L))


@pytest.fixture(scope="module")
def gpu(P, ref):
    w = ref["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    L = P.lor_set_list(s, ls)
    C = P.lor_set_classes(s, ls)
    WC = P.bin_spread(s, t, T, eta, C, Wt, Wa)
    G = P.sysmat_rows(s, im, L)
    M = P.Matrix(G[0], G[1], G[2], ref["nv"]).set_spread(s, ls, Wt, Wa, WC)
    torch.cuda.synchronize()
    return dict(T=T, eta=eta, L=L, C=C, WC=WC, G=G, M=M)


def test_table(gpu, ref):
    assert_close(gpu["T"].cpu().numpy(), ref["T"], 1e-5, 1e-7, "table")
    assert_close(gpu["eta"].cpu().numpy()[..., -1], ref["eta"], 1e-6, 1e-12, "eta")


def test_lor_set_order(gpu, ref):
    np.testing.assert_array_equal(gpu["L"].cpu().numpy(), ref["L"])
    w = ref["w"]
    s, Dm = w["scanner"], w["lors"]["max_ring_diff"]
    nt = I.n_transaxial(s)
    tp = I.transaxial_pairs(s, w["lors"]["fan_half"])
    tp = tp[tp[:, 0] < s["nt_block"]]
    want = []
    for a, b in tp:
        for d in range(-Dm, Dm + 1):
            ra = max(0, -d)
            want.append((ra * nt + a, (ra + d) * nt + b))
    np.testing.assert_array_equal(gpu["C"].cpu().numpy(), np.array(want, dtype=np.int32))


def test_class_spreads(gpu, ref, orc):
    w = ref["w"]
    Wt, Wa = w["window"]
    C = gpu["C"].cpu().numpy()
    Wo = orc.spread(w["scanner"], w["table"], ref["T"], C, Wt, Wa)
    m = orc.tie_margin(w["scanner"], w["table"], ref["T"], C)
    ok = m >= 1e-5
    assert ok.mean() > 0.99
    scale = np.abs(Wo).reshape(len(C), -1).max(1)[:, None, None]
    assert_close(gpu["WC"].cpu().numpy()[ok], Wo[ok], 1e-5, SPREAD_ATOL_REL * scale[ok] + 1e-30,
                 "class spread")


def test_class_spreads_mirrors(P, gpu, ref, orc):
    """psf_bin_spread_classes: one class of each orbit under the axial and
    transaxial reflections goes through the spread kernel (equal to
    psf_bin_spread there), the others are its images; every class is checked
    against the oracle's own spread of its representative LOR."""
    w = ref["w"]
    s, t, ls = w["scanner"], w["table"], w["lors"]
    Wt, Wa = w["window"]
    Wm = P.bin_spread_classes(s, t, gpu["T"], gpu["eta"], ls, gpu["C"], Wt, Wa).cpu().numpy()
    W = gpu["WC"].cpu().numpy()
    C = gpu["C"].cpu().numpy()
    same = (Wm == W).reshape(len(C), -1).all(1)
    assert same.mean() > 0.25  # the computed classes (168 of 588 here)
    Wo = orc.spread(s, t, ref["T"], C, Wt, Wa)
    ok = orc.tie_margin(s, t, ref["T"], C) >= 1e-5
    assert ok.mean() > 0.99
    scale = np.abs(Wo).reshape(len(C), -1).max(1)[:, None, None]
    assert_close(Wm[ok], Wo[ok], 1e-5, SPREAD_ATOL_REL * scale[ok] + 1e-30,
                 "class spreads through the mirrors")


def test_geometric_rows(gpu, ref):
    ptr, col, val = [a.cpu().numpy() for a in gpu["G"][:3]]
    compare_chord_rows((ptr, col, val), ref["G"], ref["nv"])


def test_set_rows_equal_list_rows(P, gpu, ref):
    # the per-transaxial-pair generator must give the very same CSR
    w = ref["w"]
    rp, col, val = P.sysmat_rows_set(w["scanner"], w["image"], w["lors"])
    torch.cuda.synchronize()
    assert torch.equal(rp, gpu["G"][0])
    assert torch.equal(col, gpu["G"][1])
    assert torch.equal(val, gpu["G"][2])


def test_factored_projector(gpu, ref, orc):
    w = ref["w"]
    s = w["scanner"]
    Wt, Wa = w["window"]
    assert (ref["margin"] >= 1e-5).all()
    M = gpu["M"]
    x = I.random_image(w["image"], 500).reshape(-1)
    y = M.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.spread_apply(s, ref["L"], ref["W"], Wt, Wa, orc.csr_fwd(ref["G"], x))
    assert_close(y, yo, 2e-5, 1e-6 * yo.max(), "factored forward")
    r = I.random_lor_values(len(ref["L"]), 501)
    b = M.back(torch.from_numpy(r).cuda()).cpu().numpy()
    bo = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], ref["W"], Wt, Wa, r), ref["nv"])
    assert_close(b, bo, 2e-5, 1e-6 * bo.max(), "factored back")
    for k in range(3):
        xk = torch.from_numpy(I.random_image(w["image"], 600 + k).reshape(-1)).cuda()
        yk = torch.from_numpy(I.random_lor_values(len(ref["L"]), 700 + k)).cuda()
        lhs = torch.dot(M.forward(xk).double(), yk.double()).item()
        rhs = torch.dot(xk.double(), M.back(yk).double()).item()
        assert lhs == pytest.approx(rhs, rel=1e-5)


@pytest.mark.parametrize("Wt,Wa", [(2, 1), (1, 3)])
def test_class_spreads_other_windows(P, gpu, ref, orc, Wt, Wa):
    """Windows without a compile-time kernel go through the generic one."""
    w = ref["w"]
    C = gpu["C"].cpu().numpy()
    WC = P.bin_spread(w["scanner"], w["table"], gpu["T"], gpu["eta"], gpu["C"], Wt, Wa)
    Wo = orc.spread(w["scanner"], w["table"], ref["T"], C, Wt, Wa)
    ok = orc.tie_margin(w["scanner"], w["table"], ref["T"], C) >= 1e-5
    scale = np.abs(Wo).reshape(len(C), -1).max(1)[:, None, None]
    assert_close(WC.cpu().numpy()[ok], Wo[ok], 1e-5, SPREAD_ATOL_REL * scale[ok] + 1e-30,
                 "class spread")


def test_sensitivity(gpu, ref, orc):
    """psf_sensitivity (window sums for S^T 1) equals A^T 1 of the oracle and
    the GPU back-projection of ones."""
    w = ref["w"]
    Wt, Wa = w["window"]
    M = gpu["M"]
    sens = M.sensitivity().cpu().numpy()
    back1 = M.back(torch.ones(M.n_rows, device="cuda")).cpu().numpy()
    ones = np.ones(len(ref["L"]))
    so = orc.csr_back(ref["G"], orc.spread_adjoint(w["scanner"], ref["L"], ref["W"], Wt, Wa, ones),
                      ref["nv"])
    assert_close(sens, so, 2e-5, 1e-6 * so.max(), "sensitivity vs oracle")
    assert_close(sens, back1, 1e-5, 1e-6 * back1.max(), "sensitivity vs back(1)")


def test_back_sens_pair(gpu):
    """psf_back_sens gives psf_back and psf_sensitivity in one pass."""
    M = gpu["M"]
    r = torch.from_numpy(I.random_lor_values(M.n_rows, 808)).cuda()
    x, sens = M.back_sens(r)
    torch.testing.assert_close(x, M.back(r), rtol=1e-5, atol=1e-6 * x.abs().max().item())
    s1 = M.sensitivity()
    torch.testing.assert_close(sens, s1, rtol=1e-5, atol=1e-6 * s1.abs().max().item())


def _pair_patch_ran(P, M, r):
    P.timing_enable(True)
    out = M.back_sens(r)
    ran = P.timing_read()
    P.timing_enable(False)
    return out, ran


def test_back_sens_pair_shared_memory(P, gpu, ref, orc):
    """With the image declared, psf_back_sens accumulates each transaxial
    pair's rows in shared memory (pair form -3): A^T r and A^T 1 against the
    oracle's G^T (S^T r) and G^T (S^T 1), and against the global-atomic pair
    kernel of the same plan without the image."""
    w = ref["w"]
    s, ls, im = w["scanner"], w["lors"], w["image"]
    Wt, Wa = w["window"]
    G = gpu["G"]
    M = P.Matrix(G[0], G[1], G[2], ref["nv"]).set_spread(s, ls, Wt, Wa, gpu["WC"]).set_image(im)
    r = torch.from_numpy(I.random_lor_values(M.n_rows, 811)).cuda()
    (x, sens), ran = _pair_patch_ran(P, M, r)
    assert "csr_back_patch_kernel" in ran and "csr_back_pair_kernel" not in ran
    x0, s0 = gpu["M"].back_sens(r)
    torch.testing.assert_close(x, x0, rtol=1e-5, atol=1e-6 * x0.abs().max().item())
    torch.testing.assert_close(sens, s0, rtol=1e-5, atol=1e-6 * s0.abs().max().item())
    rn = r.cpu().numpy().astype(np.float64)
    ones = np.ones(len(ref["L"]))
    for got, q in ((x, rn), (sens, ones)):
        want = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], ref["W"], Wt, Wa, q),
                            ref["nv"])
        assert_close(got.cpu().numpy(), want, 2e-5, 1e-6 * np.abs(want).max(), "pair patch")


def test_back_sens_pair_shared_memory_foreign_columns(P, gpu, ref):
    """Rows whose voxels are not the pair's cells (the columns of every row
    replaced by a seeded permutation of the grid) take the global atomics:
    the shared-memory pair form still equals the plain pair kernel."""
    w = ref["w"]
    s, ls, im = w["scanner"], w["lors"], w["image"]
    Wt, Wa = w["window"]
    G = gpu["G"]
    perm = torch.from_numpy(I.rng(812).permutation(ref["nv"]).astype(np.int32)).cuda()
    col = perm[G[1].long()].contiguous()
    Ma = P.Matrix(G[0], col, G[2], ref["nv"]).set_spread(s, ls, Wt, Wa, gpu["WC"]).set_image(im)
    Mb = P.Matrix(G[0], col, G[2], ref["nv"]).set_spread(s, ls, Wt, Wa, gpu["WC"])
    r = torch.from_numpy(I.random_lor_values(Ma.n_rows, 813)).cuda()
    (x, sens), ran = _pair_patch_ran(P, Ma, r)
    assert "csr_back_patch_kernel" in ran
    x0, s0 = Mb.back_sens(r)
    torch.testing.assert_close(x, x0, rtol=1e-5, atol=1e-6 * x0.abs().max().item())
    torch.testing.assert_close(sens, s0, rtol=1e-5, atol=1e-6 * s0.abs().max().item())


def test_set_image_rejects_other_grids(P, gpu, ref):
    w = ref["w"]
    im = dict(w["image"], nz=w["image"]["nz"] + 1)
    with pytest.raises(P.PSFError):
        gpu["M"].set_image(im)


def test_factored_projector_tall_scanner(P, orc):
    """A set of 72 crystal rings (ring strips beyond one half-warp: the factored
    stencil takes whole warps per difference group) against the oracle."""
    w = I.workload("RING3D_TALL")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    To, _ = orc.table_build(s, t)
    L = I.workload_lors(w)
    Wo = orc.spread(s, t, To, L, Wt, Wa)
    Go = orc.rows_geom(s, im, L)
    T, eta = P.response_build(s, t)
    WC = P.bin_spread(s, t, T, eta, P.lor_set_classes(s, ls), Wt, Wa)
    G = P.sysmat_rows_set(s, im, ls)
    M = P.Matrix(G[0], G[1], G[2], nv).set_spread(s, ls, Wt, Wa, WC)
    x = I.random_image(im, 640).reshape(-1)
    y = M.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.spread_apply(s, L, Wo, Wt, Wa, orc.csr_fwd(Go, x))
    assert_close(y, yo, 2e-5, 1e-6 * yo.max(), "factored forward, 72 rings")
    r = I.random_lor_values(len(L), 641)
    b = M.back(torch.from_numpy(r).cuda()).cpu().numpy()
    bo = orc.csr_back(Go, orc.spread_adjoint(s, L, Wo, Wt, Wa, r), nv)
    assert_close(b, bo, 2e-5, 1e-6 * bo.max(), "factored back, 72 rings")
    # the same through the plain stencil form
    M.set_stencil_form(1)
    torch.testing.assert_close(M.forward(torch.from_numpy(x).cuda()).cpu(), torch.from_numpy(y),
                               rtol=1e-5, atol=1e-6 * float(abs(y).max()))


@pytest.mark.parametrize("form", [1, 2, 3, 4, 5])
def test_every_stencil_form(P, gpu, ref, orc, form):
    """Each stencil form of the factored projector (1 plain, 2 register-blocked,
    3 and 4 cp.async-staged, 5 the bulk-copy pipeline) against the oracle, in
    both directions; the form's own kernel must be the one that ran."""
    w = ref["w"]
    s, ls = w["scanner"], w["lors"]
    Wt, Wa = w["window"]
    G = gpu["G"]
    M = P.Matrix(G[0], G[1], G[2], ref["nv"]).set_spread(s, ls, Wt, Wa, gpu["WC"])
    M.set_stencil_form(form)
    x = I.random_image(w["image"], 650).reshape(-1)
    r = I.random_lor_values(len(ref["L"]), 651)
    P.timing_enable(True)
    y = M.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    b = M.back(torch.from_numpy(r).cuda()).cpu().numpy()
    ran = P.timing_read()
    P.timing_enable(False)
    name = {1: "stencil_kernel", 2: "stencil2_kernel", 3: "stencil3_kernel",
            4: "stencil4_kernel", 5: "stencil5_kernel"}[form]
    assert f"{name}<forward>" in ran and f"{name}<adjoint>" in ran, sorted(ran)
    yo = orc.spread_apply(s, ref["L"], ref["W"], Wt, Wa, orc.csr_fwd(ref["G"], x))
    assert_close(y, yo, 2e-5, 1e-6 * yo.max(), f"form {form} forward")
    bo = orc.csr_back(ref["G"], orc.spread_adjoint(s, ref["L"], ref["W"], Wt, Wa, r), ref["nv"])
    assert_close(b, bo, 2e-5, 1e-6 * bo.max(), f"form {form} back")


def test_stencil5_follows_new_spreads(P, gpu, ref):
    """Form 5 keeps a re-laid-out copy of the class spreads: a later
    psf_matrix_set_spread (here with halved spreads) must be picked up."""
    w = ref["w"]
    s, ls = w["scanner"], w["lors"]
    Wt, Wa = w["window"]
    G = gpu["G"]
    M = P.Matrix(G[0], G[1], G[2], ref["nv"]).set_spread(s, ls, Wt, Wa, gpu["WC"])
    M.set_stencil_form(5)
    x = torch.from_numpy(I.random_image(w["image"], 652).reshape(-1)).cuda()
    y1 = M.forward(x).clone()
    half = gpu["WC"] * 0.5
    M.set_spread(s, ls, Wt, Wa, half)
    M.set_stencil_form(5)
    y2 = M.forward(x)
    torch.testing.assert_close(y2, 0.5 * y1, rtol=1e-6, atol=1e-7 * y1.abs().max().item())
