"""Voxel-driven homogenization (psf_voxel_homog, Sec. 2.3 Eq. 11-12) on the
GPU against the FP64 oracle on the planar ring, and its relation to the
LOR-driven matrix A = S G."""
import numpy as np
import pytest
import torch

from paper_1607_06170_gb300 import inputs as I
from parity import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(orc):
    from paper_1607_06170_gb300 import build, psf as P

    build.build()
    w = I.workload("RING2D")
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    T, eta = P.response_build(s, t)
    To, _ = orc.table_build(s, t)
    return dict(P=P, w=w, T=T, eta=eta, To=To, L=I.workload_lors(w))


@pytest.mark.parametrize("k", [60, 240])
def test_voxel_homog_vs_oracle(setup, orc, k):
    P, w = setup["P"], setup["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt = w["window"][0]
    A = P.voxel_homog(s, t, setup["T"], setup["eta"], im, ls, k, Wt).cpu().numpy()
    Ao, margin = orc.voxel_homog(s, t, setup["To"], im, setup["L"], k, Wt)
    assert margin.min() > 1e-5  # no response decision within reach of FP32 rounding
    scale = np.abs(Ao).max(0, keepdims=True)
    assert_close(A, Ao, 1e-5, 1e-6 * scale + 1e-30, f"voxel-driven A (k = {k})")


def test_against_lor_driven(setup, orc):
    """Both generators spread each line of response over neighbouring pairs;
    projected on the disc phantom they agree in shape (correlation > 0.9)
    though they weigh lines differently (chord length against equal angles)."""
    P, w = setup["P"], setup["w"]
    s, t, im, ls = w["scanner"], w["table"], w["image"], w["lors"]
    Wt, Wa = w["window"]
    A = P.voxel_homog(s, t, setup["T"], setup["eta"], im, ls, 960, Wt).cpu().numpy()
    L = setup["L"]
    W = orc.spread(s, t, setup["To"], L, Wt, Wa)
    G = orc.rows_geom(s, im, L)
    x = I.phantom_discs(im, 0).reshape(-1).astype(np.float64)
    y_lor = orc.spread_apply(s, L, W, Wt, Wa, orc.csr_fwd(G, x))
    y_vox = A.astype(np.float64) @ x
    c = np.corrcoef(y_lor, y_vox)[0, 1]
    print(f"\nvoxel-driven (k = 960) vs LOR-driven projection of the disc phantom: corr {c:.4f}")
    assert c > 0.9
