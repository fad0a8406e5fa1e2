"""Pins of the oracle's single-photon response (Sec. 2.1.1, Eq. 1; Sec. 2.1.3, Eq. 6-7).

The oracle clips every crystal box against the ray; these tests check it
against things fixed independently of that code: the closed form of a
contiguous array, a Monte Carlo of exponential free paths that finds crystals
by point membership, normalisation identities, and the paper's own setup.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1607_06170_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def flat(wt=2.0, wa=2.0, depth=10.0, gt=0.0, ga=0.0, mu=0.087):
    return I.scanner(8, 8, 1, 1, wt, wa, depth, gt, ga, 50.0, 0.0, mu)


def closed_form_contiguous(alpha, u, lam, D, mu, K):
    """T_k for a contiguous array (no gaps), derived from the depths z_k at
    which the ray crosses into crystal k: z_0 = 0, z_k = (s + (k-1) lam)/tan a,
    s = (1-u) lam, and T_k = exp(-mu z_k/cos a) - exp(-mu min(z_{k+1}, D)/cos a)."""
    T = np.zeros(K)
    if alpha == 0.0:
        T[0] = 1.0 - math.exp(-mu * D)
        return T
    s = (1.0 - u) * lam
    z = [0.0] + [(s + (k - 1) * lam) / math.tan(alpha) for k in range(1, K + 1)]
    for k in range(K):
        if z[k] >= D:
            break
        T[k] = math.exp(-mu * z[k] / math.cos(alpha)) - math.exp(
            -mu * min(z[k + 1], D) / math.cos(alpha))
    return T


def test_eta_matches_closed_form_values(orc):
    # Sum over an unbounded array: 1 - exp(-mu D / cos a).
    s = flat()
    for deg, want in [(0, 0.5810485), (30, 0.6338051), (60, 0.8244796)]:
        _, eta = orc.trace_response(s, math.radians(deg), 0.0, 0.5, 0.5, 40, 1)
        assert eta == pytest.approx(want, abs=5e-8)
        assert eta == pytest.approx(1 - math.exp(-0.87 / math.cos(math.radians(deg))), rel=1e-14)


@pytest.mark.parametrize("deg", [0.0, 3.0, 11.25, 30.0, 47.0, 78.75])
@pytest.mark.parametrize("u", [0.0625, 0.3125, 0.5, 0.9375])
def test_contiguous_closed_form(orc, deg, u):
    s = flat()
    T, eta = orc.trace_response(s, math.radians(deg), 0.0, u, 0.5, 40, 1)
    want = closed_form_contiguous(math.radians(deg), u, 2.0, 10.0, 0.087, 40)
    np.testing.assert_allclose(T[:, 0], want, rtol=1e-12, atol=1e-15)
    assert eta == pytest.approx(want.sum(), rel=1e-12)


def test_axial_motion_alone_is_the_same_closed_form(orc):
    # alpha_t = 0, polar angle theta: the ray moves only axially, tan(theta) per depth.
    s = flat(wt=1.9, wa=2.5)
    th = math.radians(35.0)
    T, _ = orc.trace_response(s, 0.0, th, 0.5, 0.25, 1, 30)
    want = closed_form_contiguous(th, 0.25, 2.5, 10.0, 0.087, 30)
    np.testing.assert_allclose(T[0, :], want, rtol=1e-12, atol=1e-15)


def _mc_response(s, alpha, theta, u, v, Mx, My, n, seed):
    """Monte Carlo of first interactions with exponential free paths.

    Material length along the ray is integrated on a fine grid by testing
    whether each sample point lies inside a crystal (modular arithmetic on the
    pitch), independent of the box clipping of the oracle."""
    g = np.random.default_rng(seed)
    pt, pa = s["xtal_w_t"] + s["gap_t"], s["xtal_w_a"] + s["gap_a"]
    tx, ty = math.tan(alpha), math.tan(theta) / math.cos(alpha)
    ds = math.sqrt(1 + tx * tx + ty * ty)
    N = 400_000
    z = (np.arange(N) + 0.5) * (s["depth"] / N)
    x = u * s["xtal_w_t"] + z * tx
    y = v * s["xtal_w_a"] + z * ty
    inside = (np.mod(x, pt) < s["xtal_w_t"]) & (np.mod(y, pa) < s["xtal_w_a"])
    dl = ds * s["depth"] / N
    cum = np.cumsum(inside * dl)
    ell = g.exponential(1.0 / s["mu"], size=n)
    k = np.searchsorted(cum, ell)
    hit = k < N
    kx = np.floor(x[k[hit]] / pt).astype(int)
    ky = np.floor(y[k[hit]] / pa).astype(int)
    H = np.zeros((Mx, My))
    np.add.at(H, (np.minimum(kx, Mx - 1), np.minimum(ky, My - 1)), 1.0)
    return H / n


@pytest.mark.parametrize("case", [
    (25.0, 0.0, 0.3, 0.5), (55.0, 10.0, 0.8, 0.2), (10.0, 30.0, 0.1, 0.9), (0.0, 20.0, 0.5, 0.7),
])
def test_monte_carlo_gapped_3d(orc, case):
    deg_t, deg_a, u, v = case
    s = flat(wt=1.9, wa=1.9, gt=0.3, ga=0.3)
    T, eta = orc.trace_response(s, math.radians(deg_t), math.radians(deg_a), u, v, 12, 12)
    n = 400_000
    H = _mc_response(s, math.radians(deg_t), math.radians(deg_a), u, v, 12, 12, n, seed=7)
    sd = np.sqrt(np.maximum(T * (1 - T), 1.0 / n) / n)
    assert np.all(np.abs(H - T) <= 5 * sd + 2e-4), np.max(np.abs(H - T) / sd)
    assert H.sum() == pytest.approx(eta, abs=5 * math.sqrt(eta * (1 - eta) / n) + 2e-4)


def test_normalisation_eq7(orc):
    # rho0 = T / eta sums to one; rho = eta rho0 sums to eta <= 1 (Eq. 6-7).
    w = I.workload("RING3D_SMALL")
    T, eta = orc.table_build(w["scanner"], w["table"])
    sums = T.sum(axis=(-1, -2))
    np.testing.assert_allclose(sums, eta, rtol=1e-12)
    assert np.all(eta <= 1.0) and np.all(eta > 0)
    rho0 = T / eta[..., None, None]
    np.testing.assert_allclose(rho0.sum(axis=(-1, -2)), 1.0, rtol=1e-12)


def test_table_nodes_and_spir_grid(orc):
    # The SPIR grid of Sec. 2.1.1 (0..60 degrees in 5-degree steps) is K = 13
    # nodes with amax = 65; entries are the trace at the node angles.
    g = json.load(open(os.path.join(GOLDEN, "spir_grid.json")))
    K, amax = g["n_nodes"], g["amax_deg"]
    assert [k * amax / K for k in range(K)] == g["angles_deg"]
    s = flat()
    t = I.table(K, 1, g["sub_positions"], 1, 40, 1, amax, 90.0)
    T, eta = orc.table_build(s, t)
    for k, deg in enumerate(g["angles_deg"]):
        for p in range(g["sub_positions"]):
            Tr, er = orc.trace_response(s, math.radians(deg), 0.0, (p + 0.5) / 8, 0.5, 40, 1)
            np.testing.assert_allclose(T[k, 0, p, 0, :, :], Tr, rtol=0, atol=0)
            assert eta[k, 0, p, 0] == er
    # nearest-node lookup
    assert orc.node(math.radians(2.49), amax, K) == 0
    assert orc.node(math.radians(2.51), amax, K) == 1
    assert orc.node(math.radians(89.0), amax, K) == K - 1


def test_peak_moves_with_entry_position(orc):
    # Sec. 2.1.1, Fig. 3 discussion: at 30 degrees with x = 8, the peak crystal
    # depends on the entry segment (the first segment peaks in the struck
    # crystal, the last one in the next).  The analytic model has no Compton
    # scatter, so the switch segment itself is not pinned.
    g = json.load(open(os.path.join(GOLDEN, "spir_grid.json")))
    s = flat()
    peaks = []
    for p in range(g["sub_positions"]):
        T, _ = orc.trace_response(s, math.radians(g["fig3_alpha_deg"]), 0.0, (p + 0.5) / 8,
                                  0.5, 16, 1)
        peaks.append(int(np.argmax(T[:, 0])))
    assert peaks[0] == 0 and peaks[-1] == 1
    assert peaks == sorted(peaks)


def test_single_ring_axial_subpositions_collapse(orc):
    # In a single-ring (2D) scanner the axial entry row does not change the
    # response, which is why the 4 x 4 entry grid reduces to 4 positions.
    s = flat()
    t = I.table(8, 1, 4, 4, 32, 1, 90.0, 90.0)
    T, eta = orc.table_build(s, t)
    for iv in range(1, 4):
        np.testing.assert_array_equal(T[:, :, :, iv], T[:, :, :, 0])
        np.testing.assert_array_equal(eta[:, :, :, iv], eta[:, :, :, 0])
