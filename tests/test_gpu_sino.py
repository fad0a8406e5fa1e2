"""Sinogram indexing on the GPU (psf_sino_bins) against the oracle on the
paper's scanner (Sec. 4, Table 1: 192 angles x 199 bins)."""
import numpy as np
import pytest

from paper_1607_06170_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_sino_bins(orc):
    from paper_1607_06170_gb300 import build, psf as P

    build.build()
    w = I.workload("EPLUS260")
    s, ls = w["scanner"], w["lors"]
    view, bins = P.sino_bins(s, ls)
    got = np.stack([view.cpu().numpy(), bins.cpu().numpy()], 1)
    want = orc.sino_index(s, I.transaxial_pairs(s, ls["fan_half"]), ls["fan_half"])
    np.testing.assert_array_equal(got, want)
    n, _ = P.lor_set_size(s, ls)
    assert n == len(got) * len(I.ring_pairs(s, ls["max_ring_diff"]))
    assert P.len_ring_pairs(s, ls) == len(I.ring_pairs(s, ls["max_ring_diff"]))
