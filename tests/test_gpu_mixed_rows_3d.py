"""Mixed-precision geometric rows of the 3D structured set (BF16 and FP16
values with a per-row FP32 scale, FP32 accumulation) -- the HBM-bound rows of
the factored projector A = S G.  Checked against the FP32 rows of the same set
(identical columns and row pointers, each value within its format's rounding)
and, through 10 MLEM iterations of the factored projector on the small 3D ring,
against the FP64 oracle's image (relative L2 within 1e-3)."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# the format's unit roundoff relative to the value (8 and 11 significand bits:
# half an ulp is at most 2^-8 and 2^-11 of the value), and half the format's
# smallest spacing (FP16 subnormals) relative to the row scale; FP32 rounding
# of the scale product and of the quotient adds a few 2^-24
REL = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}
ABS = {"bf16": 2.0 ** -134, "f16": 2.0 ** -25}
IMAGE_TOL = {"f32": 1e-4, "bf16": 1e-3, "f16": 1e-3}


@pytest.fixture(scope="module")
def P():
    from paper_1607_06170_gb300 import build, psf

    build.build()
    return psf


@pytest.mark.parametrize("name", ["RING3D_SMALL", "RING2D", "RING3D"])
@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_typed_rows_against_fp32_rows(P, name, dtype):
    w = I.workload(name)
    s, im, ls = w["scanner"], w["image"], w["lors"]
    ptr, col, val = P.sysmat_rows_set(s, im, ls)
    ptr2, col2, val2, scale = P.sysmat_rows_set_typed(s, im, ls, dtype)
    torch.cuda.synchronize()
    assert torch.equal(ptr, ptr2) and torch.equal(col, col2)
    assert val2.dtype == {"bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    n = ptr.numel() - 1
    step = 1 << 21  # rows per chunk (the full 3D set has ~4e9 values)
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        a, b = int(ptr[r0]), int(ptr[r1])
        rows = torch.repeat_interleave(torch.arange(r0, r1, device="cuda"),
                                       ptr[r0 + 1:r1 + 1] - ptr[r0:r1])
        sc = scale[rows]
        f32 = val[a:b]
        v = val2[a:b].float()
        err = (v * sc - f32).abs()
        tol = (REL[dtype] + 4 * 2.0 ** -24) * f32.abs() + ABS[dtype] * sc
        assert bool((err <= tol).all()), (r0, float((err / tol).max()))
        # every stored value lies in (0, 1]: the scale bounds the row's chords
        assert bool((v > 0).all()) and bool((v <= 1).all())
        assert bool((f32 <= sc * (1 + 2.0 ** -22)).all())


def test_fp32_form_is_the_set_generator(P):
    w = I.workload("RING3D_SMALL")
    s, im, ls = w["scanner"], w["image"], w["lors"]
    a = P.sysmat_rows_set(s, im, ls)
    b = P.sysmat_rows_set_typed(s, im, ls, "f32")
    assert b[3] is None
    for x, y in zip(a, b[:3]):
        assert torch.equal(x, y)


def test_typed_rows_reject_bad_arguments(P):
    import ctypes as C

    w = I.workload("RING3D_SMALL")
    s, i, l = P.scanner(w["scanner"]), P.image(w["image"]), P.lor_set(w["lors"])
    n, _ = P.lor_set_size(w["scanner"], w["lors"])
    ptr = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(8, dtype=torch.int32, device="cuda")
    val = torch.zeros(8, dtype=torch.bfloat16, device="cuda")
    sc = torch.zeros(n, dtype=torch.float32, device="cuda")
    nnz = C.c_int64()
    L = P.lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cp = lambda t: C.c_void_p(t.data_ptr())
    # unknown dtype, F32 with a scale, 16-bit fill without a scale
    assert L.psf_sysmat_rows_set_typed(C.byref(s), C.byref(i), C.byref(l), 7, cp(ptr), None,
                                       None, None, 0, C.byref(nnz), st) == -1
    assert L.psf_sysmat_rows_set_typed(C.byref(s), C.byref(i), C.byref(l), 0, cp(ptr), cp(col),
                                       cp(val), cp(sc), 8, C.byref(nnz), st) == -1
    assert L.psf_sysmat_rows_set_typed(C.byref(s), C.byref(i), C.byref(l), 1, cp(ptr), cp(col),
                                       cp(val), None, 8, C.byref(nnz), st) == -1
    # too small: capacity error with the required count
    assert L.psf_sysmat_rows_set_typed(C.byref(s), C.byref(i), C.byref(l), 1, cp(ptr), cp(col),
                                       cp(val), cp(sc), 8, C.byref(nnz), st) == -2
    assert nnz.value > 8


@pytest.fixture(scope="module")
def small3d(orc):
    w = I.workload("RING3D_SMALL")
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    L = I.workload_lors(w)
    To, _ = orc.table_build(s, t)
    Wo = orc.spread(s, t, To, L, Wt, Wa)
    Go = orc.rows_geom(s, im, L)
    fwd = lambda v: orc.spread_apply(s, L, Wo, Wt, Wa, orc.csr_fwd(Go, v))
    back = lambda q: orc.csr_back(Go, orc.spread_adjoint(s, L, Wo, Wt, Wa, q), nv)
    xt = I.phantom_cylinder(im, w["index"]).reshape(-1).astype(np.float64)
    y = fwd(xt)
    xo = orc.mlem(fwd, back, y, nv, 10)
    return dict(w=w, nv=nv, y=y, xo=xo, margin=orc.tie_margin(s, t, To, L))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_factored_mlem_with_typed_rows(P, small3d, dtype):
    from paper_1607_06170_gb300.torch_api import mlem

    c = small3d
    w = c["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    assert (c["margin"] >= 1e-5).all()
    T, eta = P.response_build(s, t)
    WC = P.bin_spread_classes(s, t, T, eta, ls, P.lor_set_classes(s, ls), Wt, Wa)
    ptr, col, val, scale = P.sysmat_rows_set_typed(s, im, ls, dtype)
    M = P.Matrix(ptr, col, val, c["nv"], row_scale=scale).set_spread(s, ls, Wt, Wa, WC)
    M.autotune()
    y = torch.from_numpy(c["y"].astype(np.float32)).cuda()
    x = mlem(M, y, iters=10).cpu().numpy().astype(np.float64)
    err = float(np.linalg.norm(x - c["xo"]) / np.linalg.norm(c["xo"]))
    print(f"\n{dtype} G rows: image after 10 MLEM iterations, rel L2 vs the FP64 oracle {err:.2e}")
    assert err < IMAGE_TOL[dtype], err
