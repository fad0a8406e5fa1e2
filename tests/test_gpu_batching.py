"""Batching of rows of uneven length: the planar ring's PSF rows (row
lengths spread over an order of magnitude) through the persistent
work-queue projectors (each warp takes the next chunk of rows from a
counter), the launch picked by the plan's autotuner, and 10 MLEM iterations
captured in one CUDA graph."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["f32", "f16"])
def plan(request):
    from paper_1607_06170_gb300 import build, psf as P

    build.build()
    w = I.workload("RING2D_ELLIPSES")
    s, t, im = w["scanner"], w["table"], w["image"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    L = torch.from_numpy(I.workload_lors(w)).cuda()
    W = P.bin_spread(s, t, T, eta, L, Wt, Wa)
    ptr, col, val, scale = P.sysmat_rows(s, im, L, W, Wt, Wa, dtype=request.param)
    nv = im["nx"] * im["ny"] * im["nz"]
    M = P.Matrix(ptr, col, val, nv, row_scale=scale)
    x = torch.from_numpy(I.phantom_ellipses(im, w["index"]).reshape(-1)).cuda()
    torch.cuda.synchronize()
    return dict(P=P, M=M, ptr=ptr, x=x, nv=nv)


def test_rows_are_uneven(plan):
    n = np.diff(plan["ptr"].cpu().numpy())
    n = n[n > 0]
    assert n.max() >= 10 * n.min()


def test_work_queue_launches_match(plan):
    M, x = plan["M"], plan["x"]
    y0 = M.forward(x).clone()
    r = torch.from_numpy(I.random_lor_values(M.n_rows, 5)).cuda()
    b0 = M.back(r).clone()
    for chunk in (1, 8, 32):
        for threads in (128, 512):
            M.set_launch(chunk, threads)
            assert torch.equal(M.forward(x), y0), (chunk, threads)  # same per-row sum order
            torch.testing.assert_close(M.back(r), b0, rtol=1e-6, atol=1e-6 * b0.abs().max().item())
    if M.dtype_name == "f32":
        M.set_launch(-1)  # streaming forward tiles
        torch.testing.assert_close(M.forward(x), y0, rtol=1e-6, atol=1e-6 * y0.abs().max().item())
        M.set_launch(-2)  # bulk-staged chunks, every direction
        torch.testing.assert_close(M.forward(x), y0, rtol=1e-6, atol=1e-6 * y0.abs().max().item())
        torch.testing.assert_close(M.back(r), b0, rtol=1e-6, atol=1e-6 * b0.abs().max().item())
        bs, ss = M.back_sens(r)
        M.set_launch(0)
        s0 = M.sensitivity()
        torch.testing.assert_close(bs, b0, rtol=1e-6, atol=1e-6 * b0.abs().max().item())
        torch.testing.assert_close(ss, s0, rtol=1e-6, atol=1e-6 * s0.abs().max().item())
        M.check()
    else:
        with pytest.raises(Exception):  # FP32 rows only
            M.set_launch(-2)
    M.set_launch(0)
    with pytest.raises(Exception):
        M.set_launch(4, 100)


def test_autotune_and_graph_mlem(plan):
    from paper_1607_06170_gb300.torch_api import mlem

    M, x = plan["M"], plan["x"]
    for chunk, threads in M.autotune():
        assert chunk >= -2 and (chunk <= 0 or threads % 32 == 0)
    y = M.forward(x).clone()
    xe = mlem(M, y, iters=10)
    xg = mlem(M, y, iters=10, graph=True)
    torch.cuda.synchronize()
    rel = (torch.linalg.norm(xg - xe) / torch.linalg.norm(xe)).item()
    assert rel < 1e-5, rel


def test_mlem_resume_from_saved_image(plan, tmp_path):
    """Checkpoint / resume: the MLEM state is the image; 6 iterations equal 3,
    a save and reload of the image (torch.save), then 3 more from it."""
    from paper_1607_06170_gb300.torch_api import mlem

    M, x = plan["M"], plan["x"]
    y = M.forward(x).clone()
    sens = M.sensitivity()
    x6 = mlem(M, y, iters=6, sens=sens)
    x3 = mlem(M, y, iters=3, sens=sens)
    torch.save(x3.cpu(), tmp_path / "mlem_state.pt")
    x3r = torch.load(tmp_path / "mlem_state.pt").cuda()
    x6r = mlem(M, y, iters=3, x0=x3r, sens=sens)
    torch.cuda.synchronize()
    rel = (torch.linalg.norm(x6r - x6) / torch.linalg.norm(x6)).item()
    assert rel < 1e-5, rel
