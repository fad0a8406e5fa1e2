"""GPU parity at the full 3D workload (44.7M LORs, 160 x 160 x 104 voxels) in
the launch configuration bench.py times: class spreads from
psf_bin_spread_classes (orbit classes through the spread kernel, the others as
their mirror images) and a projector plan tuned by psf_matrix_autotune.
Checked on outputs the oracle can compute one by one -- the whole response
table, sampled class spreads (computed and mirrored), sampled chord rows,
sampled forward-projected LORs (each gathered from the oracle's per-LOR
spreads of up to 2 x 2401 neighbouring LORs) -- and, over every class, LOR
and voxel, against the direct spread kernel and the plain projector forms."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import SPREAD_ATOL_REL, TABLE_ATOL, assert_close, compare_chord_rows

pytestmark = pytest.mark.gpu
NAME = "RING3D"
MARGIN = 1e-5  # classes with a rounding decision closer than this have several correct spreads


@pytest.fixture(scope="module")
def setup(orc):
    from paper_1607_06170_gb300 import build, psf as P

    build.build()
    w = I.workload(NAME)
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    C = P.lor_set_classes(s, ls)
    WC = P.bin_spread(s, t, T, eta, C, Wt, Wa)  # every class through the spread kernel
    WM = P.bin_spread_classes(s, t, T, eta, ls, C, Wt, Wa)  # as bench.py: orbits + images
    G = P.sysmat_rows_set(s, im, ls)
    nv = im["nx"] * im["ny"] * im["nz"]
    M = P.Matrix(G[0], G[1], G[2], nv).set_spread(s, ls, Wt, Wa, WM).set_image(im)
    tuned = M.autotune()
    torch.cuda.synchronize()
    To, eo = orc.table_build(s, t)
    tp = I.transaxial_pairs(s, ls["fan_half"]).astype(np.int64)
    rp = I.ring_pairs(s, ls["max_ring_diff"]).astype(np.int64)
    return dict(w=w, P=P, T=T, eta=eta, C=C, WC=WC, WM=WM, G=G, M=M, tuned=tuned, To=To, eo=eo,
                tp=tp, rp=rp, nv=nv)


def class_orbits(s, ls, C):
    """For each class (rows of C, in class order): the smallest class index of
    its orbit under the axial reflection (ring difference d -> -d) and the
    transaxial reflection through block 0's centre plane (crystal x -> (Nb - 1
    - x) mod Nt, ends swapped with d -> -d when the reflected first crystal
    comes after the second, then rotated by whole blocks until the first
    crystal is in block 0)."""
    nt, nb = I.n_transaxial(s), s["nt_block"]
    a, b = C[:, 0] % nt, C[:, 1] % nt
    d = C[:, 1] // nt - C[:, 0] // nt
    index = {(int(x), int(y), int(z)): k for k, (x, y, z) in enumerate(zip(a, b, d))}

    def refl_t(x, y, z):
        x2, y2 = (nb - 1 - x) % nt, (nb - 1 - y) % nt
        if x2 > y2:
            x2, y2, z = y2, x2, -z
        k = x2 // nb
        return x2 - k * nb, y2 - k * nb, z

    out = np.empty(len(C), dtype=np.int64)
    for k, key in enumerate(zip(a.tolist(), b.tolist(), d.tolist())):
        x, y, z = key
        orbit = [key, (x, y, -z), refl_t(x, y, z), refl_t(x, y, -z)]
        out[k] = min(index[o] for o in orbit)
    return out


def lor_of(d, rows):
    nt = I.n_transaxial(d["w"]["scanner"])
    nrp = len(d["rp"])
    t = d["tp"][rows // nrp]
    r = d["rp"][rows % nrp]
    return np.stack([r[:, 0] * nt + t[:, 0], r[:, 1] * nt + t[:, 1]], 1).astype(np.int32)


def test_table_full(setup):
    d = setup
    assert_close(d["T"].cpu().numpy(), d["To"], 1e-5, TABLE_ATOL, "table")
    assert_close(d["eta"].cpu().numpy()[..., -1], d["eo"], 1e-5, 1e-12, "eta")


def test_sampled_class_spreads(setup, orc):
    d = setup
    w = d["w"]
    Wt, Wa = w["window"]
    C = d["C"].cpu().numpy()
    pick = np.random.default_rng(31).choice(len(C), 48, replace=False)
    Wo = orc.spread(w["scanner"], w["table"], d["To"], C[pick], Wt, Wa)
    ok = orc.tie_margin(w["scanner"], w["table"], d["To"], C[pick]) >= MARGIN
    print(f"sampled classes: {(~ok).sum()} of {len(pick)} left out by the tie margin")
    assert ok.sum() >= 40
    got = d["WC"][torch.from_numpy(pick).cuda()].cpu().numpy()
    scale = np.abs(Wo).reshape(len(pick), -1).max(1)[:, None, None]
    assert_close(got[ok], Wo[ok], 1e-5, SPREAD_ATOL_REL * scale[ok] + 1e-30, "class spreads")


def test_mirrored_classes_equal_direct(setup, orc):
    """psf_bin_spread_classes against psf_bin_spread on all 84,227 classes:
    the orbit classes are the same kernel's output (bit-equal), the images
    equal the direct spread except where a sub-LOR decision of the class or of
    its image sits within the working precision of a boundary; every class
    outside tolerance must be one the oracle's tie margin flags."""
    d = setup
    w = d["w"]
    s, ls = w["scanner"], w["lors"]
    C = d["C"].cpu().numpy()
    can = class_orbits(s, ls, C)
    computed = can == np.arange(len(C))
    print(f"{computed.sum()} orbit classes computed, {(~computed).sum()} images")
    assert computed.sum() == 21744 and len(C) == 84227
    WM, WC = d["WM"], d["WC"]
    cidx = torch.from_numpy(np.flatnonzero(computed)).cuda()
    assert torch.equal(WM[cidx], WC[cidx])
    scale = WC.abs().amax(dim=(1, 2), keepdim=True)
    tol = 1e-5 * WC.abs() + SPREAD_ATOL_REL * scale + 1e-30
    bad = ((WM - WC).abs() > tol).any(2).any(1).cpu().numpy()
    assert not (bad & computed).any()
    nbad = int(bad.sum())
    print(f"mirrored classes outside tolerance: {nbad} of {len(C)}")
    assert nbad <= 0.2 * len(C)
    if nbad:
        m = orc.tie_margin(s, w["table"], d["To"], C[bad])
        assert (m < MARGIN).all(), C[bad][m >= MARGIN][:5]


def test_image_classes_against_oracle(setup, orc):
    """Sampled image classes (written by the mirror kernel, never by the
    spread kernel) against the oracle's own spread of the class LOR; half of
    them with the first crystal at the centre of block 0 (Nb = 13 is odd, so
    the transaxial reflection maps that crystal onto itself)."""
    d = setup
    w = d["w"]
    s, ls = w["scanner"], w["lors"]
    Wt, Wa = w["window"]
    nt, nb = I.n_transaxial(s), s["nt_block"]
    C = d["C"].cpu().numpy()
    can = class_orbits(s, ls, C)
    img = np.flatnonzero(can != np.arange(len(C)))
    centre = img[(C[img, 0] % nt) == (nb - 1) // 2]
    other = img[(C[img, 0] % nt) != (nb - 1) // 2]
    assert len(centre) > 32
    g = np.random.default_rng(34)
    pick = np.concatenate([g.choice(centre, 32, replace=False), g.choice(other, 32, replace=False)])
    Wo = orc.spread(s, w["table"], d["To"], C[pick], Wt, Wa)
    ok = orc.tie_margin(s, w["table"], d["To"], C[pick]) >= MARGIN
    print(f"image classes: {(~ok).sum()} of {len(pick)} left out by the tie margin "
          f"({(~ok[:32]).sum()} of the 32 centre-crystal classes)")
    assert ok[:32].sum() >= 24 and ok[32:].sum() >= 24
    got = d["WM"][torch.from_numpy(pick).cuda()].cpu().numpy()
    scale = np.abs(Wo).reshape(len(pick), -1).max(1)[:, None, None]
    assert_close(got[ok], Wo[ok], 1e-5, SPREAD_ATOL_REL * scale[ok] + 1e-30, "image classes")


def test_sampled_rows(setup, orc):
    d = setup
    w = d["w"]
    ptr = d["G"][0]
    n = ptr.numel() - 1
    rows = np.sort(np.random.default_rng(32).choice(n, 3000, replace=False))
    L = lor_of(d, rows)
    ref = orc.rows_geom(w["scanner"], w["image"], L)
    pr = ptr.cpu().numpy()
    col, val = d["G"][1], d["G"][2]
    starts, ends = pr[rows], pr[rows + 1]
    idx = torch.from_numpy(np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)])).cuda()
    gcol = col[idx].cpu().numpy()
    gval = val[idx].cpu().numpy()
    gptr = np.concatenate([[0], np.cumsum(ends - starts)])
    compare_chord_rows((gptr, gcol, gval), ref, d["nv"])


def test_set_rows_equal_list_rows_full(setup):
    """Every row of the structured-set generator (the one bench.py times) is
    bit-identical to the per-LOR tracer's row of the same LOR: 44.7M rows,
    about 4e9 nonzeros."""
    d = setup
    P, w, G = d["P"], d["w"], d["G"]
    L = P.lor_set_list(w["scanner"], w["lors"])
    ptr, col, val, _ = P.sysmat_rows(w["scanner"], w["image"], L)
    del L
    assert torch.equal(ptr, G[0])
    assert torch.equal(col, G[1])
    assert torch.equal(val, G[2])


def _neighbours(d, m_row):
    """Geometric LORs whose +-3 x +-3 window lands on LOR m_row, with the
    window entries (e1, e2) of each term."""
    w = d["w"]
    s = w["scanner"]
    nt, nr = I.n_transaxial(s), I.n_rings(s)
    F, Dm = w["lors"]["fan_half"], w["lors"]["max_ring_diff"]
    Wt, Wa = w["window"]
    W2a = 2 * Wa + 1
    (X, Y), = lor_of(d, np.array([m_row]))
    tX, rX, tY, rY = X % nt, X // nt, Y % nt, Y // nt
    terms = []
    for e1 in range((2 * Wt + 1) * W2a):
        dt1, da1 = e1 // W2a - Wt, e1 % W2a - Wa
        for e2 in range((2 * Wt + 1) * W2a):
            dt2, da2 = e2 // W2a - Wt, e2 % W2a - Wa
            for t1, r1, t2, r2 in ((tX, rX, tY, rY), (tY, rY, tX, rX)):
                g1t, g2t = (t1 - dt1) % nt, (t2 - dt2) % nt
                g1r, g2r = r1 - da1, r2 - da2
                if not (0 <= g1r < nr and 0 <= g2r < nr) or g1t >= g2t:
                    continue
                dd = g2t - g1t
                if dd < nt // 2 - F or dd > nt // 2 + F or abs(g2r - g1r) > Dm:
                    continue
                terms.append((g1r * nt + g1t, g2r * nt + g2t, e1, e2))
    return terms


def test_sampled_forward_outputs(setup, orc):
    # Each sampled output gathers up to 2 x 2401 neighbouring LORs, each with
    # 4096 sub-LORs; somewhere among them a rounding decision sits within the
    # FP32 working precision of a node or lattice boundary, where both sides
    # of the boundary are correct.  The oracle counts, per neighbour, the
    # sub-LORs with a decision within 1e-5 of a boundary, and the comparison
    # allows each such sub-LOR 8x its average share of that neighbour's term.
    d = setup
    w = d["w"]
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    nsub = (t["n_sub_t"] * t["n_sub_a"]) ** 2
    x = I.phantom_cylinder(im, 1).reshape(-1)
    y = d["M"].forward(torch.from_numpy(x).cuda()).cpu().numpy()
    g = np.random.default_rng(33)
    rows = [int(r) for r in g.choice(y.size, 40, replace=False)]
    checked = 0
    for m_row in rows:
        terms = _neighbours(d, m_row)
        if not terms:
            continue
        lors = np.unique(np.array([(a, b) for a, b, _, _ in terms], dtype=np.int32), axis=0)
        _, namb = orc.tie_count(s, t, d["To"], lors, 1e-5)
        Wg = orc.spread(s, t, d["To"], lors, Wt, Wa)
        Gg = orc.rows_geom(s, im, lors)
        p = orc.csr_fwd(Gg, x.astype(np.float64))
        if not p.any():
            continue
        pos = {(int(a), int(b)): k for k, (a, b) in enumerate(lors)}
        ref, amb = 0.0, 0.0
        for a, b, e1, e2 in terms:
            k = pos[(a, b)]
            term = Wg[k, e1, e2] * p[k]
            ref += term
            amb += 8.0 * namb[k] / nsub * abs(term)
        assert abs(y[m_row] - ref) <= 2e-5 * abs(ref) + amb + 1e-12, (m_row, y[m_row], ref, amb)
        checked += 1
        if checked == 3:
            break
    assert checked == 3


def test_adjoint_identity_full(setup):
    d = setup
    im = d["w"]["image"]
    M = d["M"]
    n = d["G"][0].numel() - 1
    for k in range(2):
        xk = torch.from_numpy(I.random_image(im, 900 + k).reshape(-1)).cuda()
        yk = torch.from_numpy(I.random_lor_values(n, 910 + k)).cuda()
        lhs = torch.dot(M.forward(xk).double(), yk.double()).item()
        rhs = torch.dot(xk.double(), M.back(yk).double()).item()
        assert lhs == pytest.approx(rhs, rel=1e-5)


def test_sensitivity_full(setup):
    """At full size: psf_sensitivity against the back-projection of ones."""
    M = setup["M"]
    sens = M.sensitivity()
    back1 = M.back(torch.ones(M.n_rows, device="cuda"))
    torch.testing.assert_close(sens, back1, rtol=1e-5, atol=1e-6 * back1.abs().max().item())


def test_tuned_launches_equal_plain_forms(setup):
    """The autotuned launches bench.py times (work-queue forward, pair
    back-projection with the sensitivity, staged stencils) against the plain
    forms (grid-stride CSR kernels, one-output-per-thread stencil) of the same
    rows and spreads, element by element over all LORs and voxels."""
    d = setup
    P, M, G, w = d["P"], d["M"], d["G"], d["w"]
    s, ls, im = w["scanner"], w["lors"], w["image"]
    Wt, Wa = w["window"]
    (fc, ft), (bc, bt) = d["tuned"]
    print(f"tuned launches: forward chunk {fc} x {ft} threads, back chunk {bc} x {bt}")
    Mp = P.Matrix(G[0], G[1], G[2], d["nv"]).set_spread(s, ls, Wt, Wa, d["WM"])
    Mp.set_launch(0).set_stencil_form(1)
    x = torch.from_numpy(I.phantom_cylinder(im, 1).reshape(-1)).cuda()
    y = torch.from_numpy(I.random_lor_values(M.n_rows, 920)).cuda()
    yt, yp = M.forward(x), Mp.forward(x)
    torch.testing.assert_close(yt, yp, rtol=1e-5, atol=1e-6 * yp.abs().max().item())
    bt_, st_ = M.back_sens(y)
    bp_, sp_ = Mp.back(y), Mp.back(torch.ones_like(y))
    torch.testing.assert_close(bt_, bp_, rtol=1e-5, atol=1e-6 * bp_.abs().max().item())
    torch.testing.assert_close(st_, sp_, rtol=1e-5, atol=1e-6 * sp_.abs().max().item())
    torch.testing.assert_close(M.back(y), bp_, rtol=1e-5, atol=1e-6 * bp_.abs().max().item())
    torch.testing.assert_close(M.sensitivity(), sp_, rtol=1e-5, atol=1e-6 * sp_.abs().max().item())


def test_pair_shared_memory_full_size(setup):
    """The pair back-projection with each transaxial pair's voxels in shared
    memory (the plan's image declared) against the global-atomic pair kernel,
    over every voxel of the bench's rows (pairs with more cells than the
    shared array holds send the rest to the global atomics)."""
    d = setup
    P, G, w = d["P"], d["G"], d["w"]
    s, ls, im = w["scanner"], w["lors"], w["image"]
    Wt, Wa = w["window"]
    r = torch.from_numpy(I.random_lor_values(G[0].numel() - 1, 940)).cuda()
    Ma = P.Matrix(G[0], G[1], G[2], d["nv"]).set_spread(s, ls, Wt, Wa, d["WM"]).set_image(im)
    Mb = P.Matrix(G[0], G[1], G[2], d["nv"]).set_spread(s, ls, Wt, Wa, d["WM"])
    P.timing_enable(True)
    xa, sa = Ma.back_sens(r)
    ran = P.timing_read()
    P.timing_enable(False)
    assert "csr_back_patch_kernel" in ran
    xb, sb = Mb.back_sens(r)
    torch.testing.assert_close(xa, xb, rtol=1e-5, atol=1e-6 * xb.abs().max().item())
    torch.testing.assert_close(sa, sb, rtol=1e-5, atol=1e-6 * sb.abs().max().item())
    del Ma, Mb


def test_stencil5_full_size(setup):
    """The bulk-copy pipeline form of S and S^T at the full size (including
    the pairs near crystal 0 whose partners wrap and are staged transposed)
    against the plain one-output-per-thread stencil, over every LOR."""
    d = setup
    P, G, w = d["P"], d["G"], d["w"]
    s, ls = w["scanner"], w["lors"]
    Wt, Wa = w["window"]
    n = G[0].numel() - 1
    pvec = torch.from_numpy(I.random_lor_values(n, 930)).cuda()
    Mp = P.Matrix(G[0], G[1], G[2], d["nv"]).set_spread(s, ls, Wt, Wa, d["WM"])
    x = torch.from_numpy(I.phantom_cylinder(w["image"], 1).reshape(-1)).cuda()
    res = {}
    for form in (1, 5):
        Mp.set_stencil_form(form)
        P.timing_enable(True)
        res[form] = (Mp.forward(x), Mp.back(pvec))
        ran = P.timing_read()
        P.timing_enable(False)
        if form == 5:
            assert "stencil5_kernel<forward>" in ran and "stencil5_kernel<adjoint>" in ran
    for k in range(2):
        a, b = res[5][k], res[1][k]
        torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6 * b.abs().max().item())
