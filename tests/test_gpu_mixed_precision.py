"""Mixed-precision PSF rows (BF16 and FP16 values with a per-row FP32 scale,
FP32 accumulation) on the planar ring with the 8-ellipse phantom: the error
of every stage against the FP64 oracle (table, spread, rows, projection,
image after 10 MLEM iterations), with the image within 1e-3 relative L2.
The FP32 form is held to the FP32 tolerances."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NAME = "RING2D_ELLIPSES"
IMAGE_TOL = {"f32": 1e-4, "bf16": 1e-3, "f16": 1e-3}
# worst elementwise error of a stored value relative to its row's largest
# value: half an ulp at the format's mantissa width (FP32 rows are exact up to
# the FP32 rounding of the arithmetic, 1e-4 as everywhere else)
ROW_TOL = {"f32": 1e-4, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case(orc):
    from paper_1607_06170_gb300 import build, psf as P

    build.build()
    w = I.workload(NAME)
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    L = I.workload_lors(w)
    To, eo = orc.table_build(s, t)
    Wo = orc.spread(s, t, To, L, Wt, Wa)
    Go = orc.rows_geom(s, im, L)
    Ao = orc.rows_psf_dense(s, L, Go, Wo, Wt, Wa, nv)
    xt = I.phantom_ellipses(im, w["index"]).reshape(-1).astype(np.float64)
    y = Ao @ xt
    xo = orc.mlem(lambda v: Ao @ v, lambda q: Ao.T @ q, y, nv, 10)
    T, eta = P.response_build(s, t)
    Lg = torch.from_numpy(L).cuda()
    Wg = P.bin_spread(s, t, T, eta, Lg, Wt, Wa)
    torch.cuda.synchronize()
    return dict(P=P, w=w, nv=nv, L=Lg, To=To, Wo=Wo, Ao=Ao, xt=xt, y=y, xo=xo, T=T, W=Wg)


def test_stage_errors(case):
    c = case
    assert _rel(c["T"].cpu().numpy(), c["To"]) < 1e-6
    assert _rel(c["W"].cpu().numpy(), c["Wo"]) < 1e-5


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_rows_projection_and_mlem(case, dtype):
    from paper_1607_06170_gb300.torch_api import mlem

    c, P = case, case["P"]
    w = c["w"]
    s, im = w["scanner"], w["image"]
    Wt, Wa = w["window"]
    ptr, col, val, scale = P.sysmat_rows(s, im, c["L"], c["W"], Wt, Wa, dtype=dtype)
    # rows: dense copy, values times the row scale
    p_, c_, v_ = ptr.cpu().numpy(), col.cpu().numpy(), val.float().cpu().numpy()
    rows = np.repeat(np.arange(len(p_) - 1), np.diff(p_))
    A = np.zeros_like(c["Ao"])
    sc = np.ones(len(p_) - 1) if scale is None else scale.cpu().numpy().astype(np.float64)
    A[rows, c_] = v_ * sc[rows]
    rowmax = np.abs(c["Ao"]).max(1, keepdims=True)
    err_rows = float((np.abs(A - c["Ao"]) / np.maximum(rowmax, 1e-30)).max())
    assert err_rows <= ROW_TOL[dtype] * 1.01, err_rows
    M = P.Matrix(ptr, col, val, c["nv"], row_scale=scale)
    xt = torch.from_numpy(c["xt"].astype(np.float32)).cuda()
    err_proj = _rel(M.forward(xt).cpu().numpy(), c["y"])
    yt = torch.from_numpy(c["y"].astype(np.float32)).cuda()
    err_img = _rel(mlem(M, yt, iters=10).cpu().numpy(), c["xo"])
    print(f"\n{dtype}: rows max err / row max {err_rows:.2e}, projection rel L2 "
          f"{err_proj:.2e}, image after 10 MLEM iterations rel L2 {err_img:.2e}")
    assert err_proj < 4 * ROW_TOL[dtype]
    assert err_img < IMAGE_TOL[dtype], err_img
