"""Pins of the oracle's sinogram indexing (Sec. 4, Table 1: 192 angles x 199
bins for 384 crystals per ring) on the paper's scanner: the index reading
maps the set's transaxial pairs one to one onto views x bins, orders the
bins of a view by the geometric signed distance of the LOR from the axis,
and the views by the LOR's normal angle."""
import math

import numpy as np

from paper_1607_06170_gb300 import inputs as I


def test_sino_index_is_one_to_one(orc):
    w = I.workload("EPLUS260")
    s, F = w["scanner"], w["lors"]["fan_half"]
    tp = I.transaxial_pairs(s, F)
    vb = orc.sino_index(s, tp, F)
    assert len(tp) == w["sino"]["views"] * w["sino"]["bins"]
    assert vb[:, 0].min() == 0 and vb[:, 0].max() == w["sino"]["views"] - 1
    assert vb[:, 1].min() == 0 and vb[:, 1].max() == w["sino"]["bins"] - 1
    flat = vb[:, 0] * w["sino"]["bins"] + vb[:, 1]
    assert len(np.unique(flat)) == len(tp)


def test_sino_index_follows_the_geometry(orc):
    w = I.workload("EPLUS260")
    s, F = w["scanner"], w["lors"]["fan_half"]
    nt = I.n_transaxial(s)
    tp = I.transaxial_pairs(s, F)
    vb = orc.sino_index(s, tp, F)
    geo = np.array([orc.lor_normal(s, a, b) for a, b in tp])
    step = 2 * math.pi / nt  # one view spans two crystal steps of the normal angle
    nb = s["nt_block"]
    for v in range(0, w["sino"]["views"], 7):
        sel = np.nonzero(vb[:, 0] == v)[0][np.argsort(vb[vb[:, 0] == v, 1])]
        # crystal c sits near angle 2 pi (c - (Nb - 1)/2) / N, so the normal of (a, b)
        # is near pi (a + b - (Nb - 1)) / N modulo pi: within a view step of the
        # view's nominal angle (flat blocks shift crystals by a fraction of a step)
        phi = geo[sel, 0]
        nominal = (2 * v + 0.5 - (nb - 1)) * math.pi / nt
        dphi = np.angle(np.exp(2j * (phi - nominal))) / 2  # difference modulo pi
        assert np.all(np.abs(dphi) < step), (v, np.abs(dphi).max() / step)
        # signed distance along the view's nominal normal falls with the bin
        # (ideal ring: -R sin(pi (bin - F) / N))
        dist = geo[sel, 1] * np.sign(np.cos(phi - nominal))
        assert np.all(np.diff(dist) < 0), v
