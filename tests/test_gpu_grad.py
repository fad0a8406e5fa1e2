"""Differentiation through the PSF projector: `PSFProject` (a torch autograd
Function whose backward is the hand-written back-projector psf_back).

* RING3D scanner with 128 x 128 x 104 voxels of 1 mm (44.7M LORs, factored
  A = S G) and Poisson counts of mean 20 per LOR: the dot-product identity on
  32 random (x, y) pairs, and the autograd gradient of the Poisson
  log-likelihood L(x) = sum y log(Ax) - Ax against central finite differences
  (step 1e-3) on 64 random voxels.  The finite differences take A's column
  e_v from the forward projector and evaluate L(x +- h e_v) in FP64, so they
  check the backward (A^T) against the forward (A) column by column.
* RING3D_SMALL (every LOR also computed by the oracle): the GPU gradient
  against the FP64 oracle's A^T(y/Ax) - A^T 1."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import assert_close

pytestmark = pytest.mark.gpu


def _loglik64(y, yh):
    """FP64 Poisson log-likelihood (log y! dropped), 0 log 0 = 0."""
    pos = yh > 0
    return (y[pos] * torch.log(yh[pos])).sum() - yh.sum()


@pytest.fixture(scope="module")
def big():
    from paper_1607_06170_gb300 import build, psf as P
    from paper_1607_06170_gb300.torch_api import project

    build.build()
    w = I.workload("RING3D_GRAD")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    T, eta = P.response_build(s, t)
    WC = P.bin_spread(s, t, T, eta, P.lor_set_classes(s, ls), Wt, Wa)
    G = P.sysmat_rows_set(s, im, ls)
    nv = im["nx"] * im["ny"] * im["nz"]
    M = P.Matrix(G[0], G[1], G[2], nv).set_spread(s, ls, Wt, Wa, WC)
    xt = torch.from_numpy(I.phantom_cylinder(im, w["index"]).reshape(-1)).cuda()
    yt = M.forward(xt)
    scale = 20.0 / yt.double().mean().item()
    y = torch.from_numpy(I.poisson_counts((yt.double() * scale).cpu().numpy(),
                                          w["index"])).cuda()
    torch.cuda.synchronize()
    return dict(w=w, M=M, nv=nv, y=y, project=project, sens=M.back(torch.ones_like(y)))


def test_dot_product_32_pairs(big):
    M, nv, w = big["M"], big["nv"], big["w"]
    for k in range(32):
        x = torch.from_numpy(I.random_image(w["image"], 1000 + k).reshape(-1)).cuda()
        r = torch.from_numpy(I.random_lor_values(M.n_rows, 2000 + k)).cuda()
        lhs = torch.dot(M.forward(x).double(), r.double()).item()
        rhs = torch.dot(x.double(), M.back(r).double()).item()
        assert lhs == pytest.approx(rhs, rel=1e-5), k


def test_autograd_gradient_vs_finite_differences(big):
    M, y, sens = big["M"], big["y"].double(), big["sens"]
    x = torch.ones(big["nv"], dtype=torch.float32, device="cuda")
    x[sens <= 1e-12 * sens.max()] = 0.0
    xg = x.clone().requires_grad_(True)
    yh = big["project"](xg, M)
    L = _loglik64(y, yh.double())
    L.backward()
    g = xg.grad.double()
    # analytic form of the same gradient, through the library calls directly
    yh0 = M.forward(x)
    ratio = torch.where(yh0 > 0, y.float() / yh0, torch.zeros_like(yh0))
    g_direct = (M.back(ratio) - sens).double()
    assert torch.allclose(g, g_direct, rtol=1e-4, atol=1e-5 * g_direct.abs().max().item())
    # central differences on 64 voxels the scanner sees
    live = torch.nonzero(sens > 1e-3 * sens.max()).flatten().cpu().numpy()
    pick = np.random.default_rng(64).choice(live, 64, replace=False)
    h = 1e-3
    yh64 = yh0.double()
    for v in pick:
        e = torch.zeros_like(x)
        e[int(v)] = 1.0
        a = M.forward(e).double()  # column v of A
        fd = (_loglik64(y, yh64 + h * a) - _loglik64(y, yh64 - h * a)).item() / (2 * h)
        scale = (y * a / torch.clamp(yh64, min=1e-30)).sum().item() + a.sum().item()
        assert abs(fd - g[int(v)].item()) <= 1e-4 * scale, (int(v), fd, g[int(v)].item())


def test_gradient_vs_oracle_small(orc):
    from paper_1607_06170_gb300 import psf as P
    from paper_1607_06170_gb300.torch_api import project

    w = I.workload("RING3D_SMALL")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    nv = im["nx"] * im["ny"] * im["nz"]
    # oracle: one spread per LOR, A = S G as two steps
    To, _ = orc.table_build(s, t)
    L = I.workload_lors(w)
    Wo = orc.spread(s, t, To, L, Wt, Wa)
    Go = orc.rows_geom(s, im, L)

    def fwd(v):
        return orc.spread_apply(s, L, Wo, Wt, Wa, orc.csr_fwd(Go, v))

    def back(r):
        return orc.csr_back(Go, orc.spread_adjoint(s, L, Wo, Wt, Wa, r), nv)

    xt = I.phantom_cylinder(im, 3).reshape(-1).astype(np.float64)
    ym = fwd(xt)
    y = I.poisson_counts(ym * (20.0 / ym.mean()), 3).astype(np.float64)
    x = I.random_image(im, 77).reshape(-1).astype(np.float64) + 0.5
    g_o = orc.poisson_grad(fwd, back, y, x)
    # GPU
    T, eta = P.response_build(s, t)
    WC = P.bin_spread(s, t, T, eta, P.lor_set_classes(s, ls), Wt, Wa)
    G = P.sysmat_rows_set(s, im, ls)
    M = P.Matrix(G[0], G[1], G[2], nv).set_spread(s, ls, Wt, Wa, WC)
    xg = torch.from_numpy(x.astype(np.float32)).cuda().requires_grad_(True)
    yt = torch.from_numpy(y).cuda()
    _loglik64(yt, project(xg, M).double()).backward()
    g = xg.grad.double().cpu().numpy()
    scale = orc.csr_back(Go, orc.spread_adjoint(s, L, Wo, Wt, Wa, y / np.maximum(fwd(x), 1e-30)),
                         nv) + back(np.ones_like(y))
    assert_close(g, g_o, 1e-4, 2e-4 * scale, "log-likelihood gradient")
