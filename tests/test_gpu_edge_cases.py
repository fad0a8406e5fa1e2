"""Edge cases of the library on the GPU: empty inputs, invalid arguments,
degenerate and invalid LORs, rows of very uneven length."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import assert_close, compare_chord_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1607_06170_gb300 import build, psf

    build.build()
    return psf


@pytest.fixture(scope="module")
def ring2d(P):
    w = I.workload("RING2D")
    T, eta = P.response_build(w["scanner"], w["table"])
    return dict(w=w, T=T, eta=eta, nv=w["image"]["nx"] * w["image"]["ny"])


def test_empty_inputs(P, ring2d):
    w = ring2d["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    L0 = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    W0 = P.bin_spread(s, t, ring2d["T"], ring2d["eta"], L0, Wt, Wa)
    assert W0.shape == (0, 2 * Wt + 1, 2 * Wt + 1)
    rp, col, val, _ = P.sysmat_rows(s, im, L0)
    assert rp.cpu().tolist() == [0] and col.numel() == 0
    M = P.Matrix(rp, col, val, ring2d["nv"])
    x = torch.rand(ring2d["nv"], device="cuda")
    assert M.forward(x).numel() == 0
    assert torch.count_nonzero(M.back(torch.zeros(0, device="cuda"))) == 0
    assert torch.count_nonzero(M.sensitivity()) == 0
    rows = P.event_rows(s, ls, L0)
    assert rows.numel() == 0
    assert torch.count_nonzero(P.histogram(rows, 10, 1.0)) == 0


def test_invalid_arguments_raise(P, ring2d):
    from paper_1607_06170_gb300.psf import PSFError

    w = ring2d["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    L = torch.from_numpy(I.workload_lors(w)[1000:1008]).cuda()  # chords across the image
    with pytest.raises(PSFError):  # quadrant (half_t + 1)(half_a + 1) above 16
        P.bin_spread(s, t, ring2d["T"], ring2d["eta"], L, 15, 1)
    with pytest.raises(PSFError):  # geometric rows are FP32 only
        P.sysmat_rows(s, im, L, dtype="bf16")
    with pytest.raises(PSFError):  # the voxel-driven generator is planar
        w3 = I.workload("RING3D_SMALL")
        T3, e3 = P.response_build(w3["scanner"], w3["table"])
        P.voxel_homog(w3["scanner"], w3["table"], T3, e3, w3["image"], w3["lors"], 8, 1)
    with pytest.raises(PSFError):  # sinogram indexing needs an even ring
        P.sino_bins(dict(s, n_blocks=9, nt_block=7), dict(fan_half=20, max_ring_diff=0))
    # capacity below the row count: PSF_ECAPACITY and the required size
    lib = P.lib()
    rp = torch.empty(L.shape[0] + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(4, dtype=torch.int32, device="cuda")
    val = torch.empty(4, dtype=torch.float32, device="cuda")
    nnz = C.c_int64()
    rc = lib.psf_sysmat_rows(C.byref(P.scanner(s)), C.byref(P.image(im)), P._ptr(L), L.shape[0],
                             None, 0, 0, 0, P._ptr(rp), P._ptr(col), P._ptr(val), None, 4,
                             C.byref(nnz), P._stream())
    torch.cuda.synchronize()
    assert rc == -2 and nnz.value > 4  # PSF_ECAPACITY


def test_invalid_and_degenerate_lors(P, ring2d, orc):
    """Invalid crystal ids and pairs of one crystal give empty rows and zero
    spreads; a pair inside one block (its chord runs along the block face) has
    no spread and, outside the image, no chords; valid LORs next to them are
    unaffected."""
    w = ring2d["w"]
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    good = I.workload_lors(w)[[0, 500, 1500]]
    bad = np.array([[-1, 5], [3, 3], [2, 900], [0, 3]], dtype=np.int32)  # [0, 3]: one block
    L = np.concatenate([good, bad]).astype(np.int32)
    Lt = torch.from_numpy(L).cuda()
    W = P.bin_spread(s, t, ring2d["T"], ring2d["eta"], Lt, Wt, Wa).cpu().numpy()
    assert np.all(W[3:] == 0.0)
    To, _ = orc.table_build(s, t)
    Wo = orc.spread(s, t, To, good, Wt, Wa)
    assert_close(W[:3], Wo, 1e-5, 1e-6 * np.abs(Wo).max(), "spreads beside invalid LORs")
    rp, col, val, _ = P.sysmat_rows(s, im, Lt)
    rp = rp.cpu().numpy()
    assert np.all(np.diff(rp)[3:] == 0)
    compare_chord_rows((rp[:4], col.cpu().numpy()[: rp[3]], val.cpu().numpy()[: rp[3]]),
                       orc.rows_geom(s, im, good), ring2d["nv"])


def test_uneven_rows_every_launch(P, ring2d):
    """The planar ring's rows run from empty (LORs that miss the image) to
    about 90 voxels; every projector launch gives the same projections."""
    w = ring2d["w"]
    s, im = w["scanner"], w["image"]
    Lt = torch.from_numpy(I.workload_lors(w)).cuda()
    rp, col, val, _ = P.sysmat_rows(s, im, Lt)
    lens = torch.diff(rp).cpu().numpy()
    assert lens.min() == 0 and lens.max() > 60
    M = P.Matrix(rp, col, val, ring2d["nv"])
    x = torch.from_numpy(I.phantom_discs(im, 0).reshape(-1)).cuda()
    y = torch.from_numpy(I.random_lor_values(M.n_rows, 5)).cuda()
    M.set_launch(0)
    f0, b0 = M.forward(x), M.back(y)
    for chunk, threads in [(1, 128), (7, 256), (128, 512), (-1, 256), (-2, 256)]:
        M.set_launch(chunk, threads)
        torch.testing.assert_close(M.forward(x), f0, rtol=1e-6, atol=1e-6 * f0.abs().max().item())
        torch.testing.assert_close(M.back(y), b0, rtol=1e-5, atol=1e-6 * b0.abs().max().item())
    M.check()


def test_bulk_staged_long_and_empty_rows(P):
    """Bulk-staged projectors on rows longer than a staged chunk (4096
    entries: chunks where no row starts), runs of empty rows, a row that
    starts exactly on a chunk boundary and a ragged tail; misaligned arrays
    are refused."""
    rng = np.random.default_rng(7)
    lens = np.array([5000, 0, 0, 3, 8192 - 5003, 9001, 0, 1, 17, 0, 4100, 2, 0, 0], dtype=np.int64)
    assert lens.sum() % 4 != 0
    ptr = np.concatenate([[0], np.cumsum(lens)])
    assert 8192 in ptr  # a row starting on a chunk boundary
    nv = 3000
    col = rng.integers(0, nv, ptr[-1]).astype(np.int32)
    val = rng.random(ptr[-1]).astype(np.float32)
    ptr_t, col_t, val_t = (torch.from_numpy(a).cuda() for a in (ptr, col, val))
    M = P.Matrix(ptr_t, col_t, val_t, nv)
    x = torch.from_numpy(rng.random(nv).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.random(len(lens)).astype(np.float32)).cuda()
    M.set_launch(0)
    f0, b0 = M.forward(x).clone(), M.back(y).clone()
    M.set_launch(-2)
    torch.testing.assert_close(M.forward(x), f0, rtol=1e-5, atol=1e-6 * f0.abs().max().item())
    torch.testing.assert_close(M.back(y), b0, rtol=1e-5, atol=1e-6 * b0.abs().max().item())
    bs, _ = M.back_sens(y)
    torch.testing.assert_close(bs, b0, rtol=1e-5, atol=1e-6 * b0.abs().max().item())
    M.check()
    ref = np.array([val[ptr[i]:ptr[i + 1]].astype(np.float64) @ x.cpu().numpy()[col[ptr[i]:ptr[i + 1]]]
                    for i in range(len(lens))])
    assert_close(M.forward(x).cpu().numpy(), ref, 1e-5, 1e-6 * np.abs(ref).max(), "bulk forward")
    # column and value arrays off a 16-byte boundary: the bulk form is refused
    col2 = torch.cat([torch.zeros(1, dtype=torch.int32, device="cuda"), col_t])[1:]
    M2 = P.Matrix(ptr_t, col2, val_t, nv)
    with pytest.raises(Exception):
        M2.set_launch(-2)


def test_bounded_wait_reports_timeout(P, ring2d):
    """The bulk-staged kernels' waits for their copies are bounded: with the
    limit forced to give up at once, every launch records PSF_ETIMEOUT in the
    plan's status word (psf_matrix_check raises it; the copies in flight are
    still drained before a CTA exits), and with the default limit the same
    plan projects normally again."""
    from paper_1607_06170_gb300.psf import PSFError

    w = ring2d["w"]
    s, im = w["scanner"], w["image"]
    Lt = torch.from_numpy(I.workload_lors(w)).cuda()
    rp, col, val, _ = P.sysmat_rows(s, im, Lt)
    M = P.Matrix(rp, col, val, ring2d["nv"])
    x = torch.from_numpy(I.phantom_discs(im, 0).reshape(-1)).cuda()
    M.set_launch(0)
    f0 = M.forward(x).clone()
    M.set_launch(-2)
    M.check()
    try:
        P.set_wait_limit(-1)
        M.forward(x)
        with pytest.raises(PSFError, match="bounded device wait"):
            M.check()
        M.back_sens(f0)
        with pytest.raises(PSFError, match="bounded device wait"):
            M.check()
    finally:
        P.set_wait_limit(P.WAIT_LIMIT_DEFAULT)
    M.check()  # cleared by the read
    torch.testing.assert_close(M.forward(x), f0, rtol=1e-6, atol=1e-6 * f0.abs().max().item())
    M.check()


def test_typed_rows_planar_ring_and_narrow_gap(P):
    """The 16-bit set rows on the planar rings (one slab per row, the narrow-gap
    ring with short chords at the block corners): same structure as the FP32
    rows, values within BF16 rounding of them."""
    for name in ("RING2D", "RING2D_NARROW"):
        w = I.workload(name)
        s, im, ls = w["scanner"], w["image"], w["lors"]
        ptr, col, val = P.sysmat_rows_set(s, im, ls)
        ptr2, col2, val2, sc = P.sysmat_rows_set_typed(s, im, ls, "bf16")
        assert torch.equal(ptr, ptr2) and torch.equal(col, col2)
        rows = torch.repeat_interleave(torch.arange(ptr.numel() - 1, device="cuda"),
                                       ptr[1:] - ptr[:-1])
        err = (val2.float() * sc[rows] - val).abs()
        assert bool((err <= (2.0 ** -8 + 2.0 ** -22) * val).all()), name


def test_stencil_form5_whole_warp_groups(P):
    """On a scanner of 72 rings (18 ring strips: each group of 4 ring
    differences takes a whole warp) the pipelined stencil form runs with
    whole-warp groups and equals the fourth form in both directions."""
    w = I.workload("RING3D_TALL")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    T, eta = P.response_build(s, t)
    WC = P.bin_spread(s, t, T, eta, P.lor_set_classes(s, ls), Wt, Wa)
    G = P.sysmat_rows_set(s, im, ls)
    M = P.Matrix(G[0], G[1], G[2], nv).set_spread(s, ls, Wt, Wa, WC)
    x = torch.from_numpy(I.random_image(im, 660).reshape(-1)).cuda()
    r = torch.from_numpy(I.random_lor_values(M.n_rows, 661)).cuda()
    out = {}
    for form in (4, 5):
        M.set_stencil_form(form)
        P.timing_enable(True)
        out[form] = (M.forward(x).clone(), M.back(r).clone())
        ran = P.timing_read()
        P.timing_enable(False)
        assert f"stencil{form}_kernel<forward>" in ran, sorted(ran)
    for k in range(2):
        b = out[4][k]
        torch.testing.assert_close(out[5][k], b, rtol=1e-5, atol=1e-6 * b.abs().max().item())


def test_traced_plan_arguments(P):
    """A traced-row plan refuses launch tuning and a size it cannot index,
    and its projections of zeros are zero."""
    from paper_1607_06170_gb300.psf import PSFError

    w = I.workload("RING3D_SMALL")
    s, im, ls = w["scanner"], w["image"], w["lors"]
    M = P.Matrix.traced(s, im, ls)
    with pytest.raises(PSFError):
        M.autotune()
    with pytest.raises(PSFError):
        M.set_launch(64, 256)
    nv = im["nx"] * im["ny"] * im["nz"]
    assert torch.count_nonzero(M.forward(torch.zeros(nv, device="cuda"))) == 0
    assert torch.count_nonzero(M.back(torch.zeros(M.n_rows, device="cuda"))) == 0
    M.check()
    big = dict(im, nx=4096, ny=4096, nz=4096)  # 2^36 voxels: beyond int32 voxel ids
    with pytest.raises(PSFError):
        P.Matrix.traced(s, big, ls)
