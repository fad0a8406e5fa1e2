"""Pins of the two-block gap path (Sec. 2.1.2, Eq. 2, 4, 5) and of the
homogenization spread (Sec. 2.2 Eq. 10, Sec. 2.3 Eq. 11-12) in the oracle."""
import math

import numpy as np
import pytest

from paper_1607_06170_gb300 import inputs as I


def _block0_frame(R):
    phi1 = 2 * math.pi / R
    n1 = np.array([math.cos(phi1), math.sin(phi1)])
    t1 = np.array([-math.sin(phi1), math.cos(phi1)])
    return n1, t1


@pytest.mark.parametrize("name", ["RING2D", "RING2D_NARROW", "RING3D"])
def test_sigma_is_corner_gap(orc, name):
    s = I.workload(name)["scanner"]
    W = s["nt_block"] * s["xtal_w_t"] + (s["nt_block"] - 1) * s["gap_t"]
    # B = intersection of the face lines x = r and p.n1 = r; sigma = |B| along the face - W/2
    R, r = s["n_blocks"], s["radius"]
    n1, _ = _block0_frame(R)
    By = (r - r * n1[0]) / n1[1]
    assert orc.sigma(s) == pytest.approx(By - W / 2, rel=1e-12)


@pytest.mark.parametrize("name", ["RING2D", "RING2D_NARROW", "RING3D"])
def test_eq4_against_line_intersection(orc, name):
    # Extend the photon's path beyond P0 until it meets block1's face line;
    # AP1 measured from block1's corner A must equal Eq. 4, and P0P1 the run.
    s = I.workload(name)["scanner"]
    R, r = s["n_blocks"], s["radius"]
    W = s["nt_block"] * s["xtal_w_t"] + (s["nt_block"] - 1) * s["gap_t"]
    n1, t1 = _block0_frame(R)
    A = r * n1 - 0.5 * W * t1
    for alpha in np.radians([2 * 180 / R + 1.0, 50.0, 61.0, 74.0]):
        for nu in [0.1, 1.0, 3.7, W - 0.2]:
            P0 = np.array([r, 0.5 * W - nu])
            d = np.array([math.cos(alpha), math.sin(alpha)])
            t = (r - P0 @ n1) / (d @ n1)
            P1 = P0 + t * d
            ap1 = (P1 - A) @ (-t1)          # distance from A away from block1
            assert abs((P1 - A) @ n1) < 1e-9  # P1 lies on block1's face line
            beta, AP1, run = orc.gap_eq(s, alpha, nu)
            assert beta == pytest.approx(alpha - 2 * math.pi / R, abs=1e-15)
            assert AP1 == pytest.approx(ap1, rel=1e-11)
            assert run == pytest.approx(t, rel=1e-11)


def _flat_ring(Nb=8, R=100000, wt=2.0, gt=0.0, na=1, nbr=1):
    # corner gap sigma = gt/2, so A and C are one intra-block gap apart and
    # block1 continues block0's crystal lattice
    W = Nb * wt + (Nb - 1) * gt
    r = 0.5 * (W + gt) / math.tan(math.pi / R)
    return I.scanner(R, Nb, na, nbr, wt, wt, 10.0, gt, gt, r, gt, 0.087)


@pytest.mark.parametrize("gt", [0.0, 0.3])
@pytest.mark.parametrize("deg", [33.0, 52.0, 71.0])
def test_gap_path_reduces_to_one_flat_array(orc, gt, deg):
    # R -> inf with the lattice continued across the corner: block1 continues
    # block0's array, so Eq. 2-5 must reproduce the long-array response: the
    # virtual entry lands on the real entry position and block1's crystal j
    # sits at offset Nb-i+j.
    s = _flat_ring(gt=gt)
    assert abs(orc.sigma(s) - 0.5 * gt) < 1e-6
    K, P, M = 8, 4, 40
    t = I.table(K, 1, P, 1, M, 1, 90.0, 90.0)
    T, _ = orc.table_build(s, t)
    a = math.radians(deg)
    k = orc.node(a, 90.0, K)
    assert orc.node(a - 2 * math.pi / s["n_blocks"], 90.0, K) == k
    for i in [3, 7]:
        for p in range(P):
            ent, eta = orc.composed(s, t, T, i, p, 0, [math.cos(a), math.sin(a), 0.0])
            got = np.zeros(M)
            for dt, da, v in ent:
                assert da == 0
                got[dt] += v
            want = T[k, 0, p, 0, :, 0]
            # two-block model: offsets past block1 (a third block) are not reached
            n2 = 2 * s["nt_block"] - i
            np.testing.assert_allclose(got[:n2], want[:n2], rtol=1e-12, atol=0)
            assert not got[n2:].any()


def test_gap_path_reduces_3d(orc):
    s = _flat_ring(Nb=6, wt=1.9, gt=0.3, na=6, nbr=2)
    t = I.table(8, 4, 4, 4, 24, 12, 80.0, 40.0)
    T, _ = orc.table_build(s, t)
    at, th = math.radians(52.0), math.radians(21.0)
    kt, ka = orc.node(at, 80.0, 8), orc.node(th, 40.0, 4)
    d = [math.cos(th) * math.cos(at), math.cos(th) * math.sin(at), math.sin(th)]
    xid = 5 * (s["n_blocks"] * s["nt_block"]) + 2   # ring 5, crystal 2 of block 0
    for p in range(4):
        for q in range(4):
            ent, _ = orc.composed(s, t, T, xid, p, q, d)
            got = np.zeros((24, 12))
            for dt, da, v in ent:
                got[dt, da] += v
            n2 = 2 * s["nt_block"] - 2
            np.testing.assert_allclose(got[:n2], T[kt, ka, p, q, :n2, :], rtol=1e-12, atol=0)


def test_neighbour_block_dominates_at_large_angle(orc):
    # Sec. 2.1.2 (Fig. 5 discussion): 16-crystal blocks, photon entering the
    # last crystal (15) at its last segment (7 of 8) next to a narrow gap: at
    # large incidence angles most detections fall in the neighbouring block.
    R, Nb = 24, 16
    r = (0.5 * Nb * 2.0 + 0.5) / math.tan(math.pi / R)
    s = I.scanner(R, Nb, 1, 1, 2.0, 2.0, 10.0, 0.0, 0.0, r, 0.0, 0.087)
    assert orc.sigma(s) == pytest.approx(0.5)
    t = I.table(36, 1, 8, 1, 40, 1, 90.0, 90.0)
    T, _ = orc.table_build(s, t)
    share = []
    for deg in [20.0, 40.0, 55.0, 65.0]:
        a = math.radians(deg)
        ent, eta = orc.composed(s, t, T, 15, 7, 0, [math.cos(a), math.sin(a), 0.0])
        b0 = sum(v for dt, _, v in ent if dt <= 0)
        b1 = sum(v for dt, _, v in ent if dt > 0)
        share.append(b1 / (b0 + b1))
    assert share[0] < 0.5 < share[-1]
    assert share == sorted(share)


def test_no_penetration_below_block_angle(orc):
    s = I.workload("RING2D_NARROW")["scanner"]
    t = I.workload("RING2D_NARROW")["table"]
    T, _ = orc.table_build(s, t)
    a = math.radians(40.0)   # below 2 pi / R = 45 degrees: beta <= 0
    ent, _ = orc.composed(s, t, T, 7, 3, 0, [math.cos(a), math.sin(a), 0.0])
    assert all(dt <= 0 for dt, _, _ in ent)


# ---------------------------------------------------------------- spread
def _outer_window(ent1, ent2, Wt, Wa):
    E = (2 * Wt + 1) * (2 * Wa + 1)
    w = np.zeros((E, E))
    for dt1, da1, v1 in ent1:
        if abs(dt1) > Wt or abs(da1) > Wa:
            continue
        for dt2, da2, v2 in ent2:
            if abs(dt2) > Wt or abs(da2) > Wa:
                continue
            w[(dt1 + Wt) * (2 * Wa + 1) + da1 + Wa, (dt2 + Wt) * (2 * Wa + 1) + da2 + Wa] += v1 * v2
    return w


def _subpairs(orc, s, t, T, id1, id2):
    P, Q = t["n_sub_t"], t["n_sub_a"]
    for p1 in range(P):
        for q1 in range(Q):
            for p2 in range(P):
                for q2 in range(Q):
                    E1 = orc.face_point(s, id1, ((p1 + .5) / P - .5) * s["xtal_w_t"],
                                        ((q1 + .5) / Q - .5) * s["xtal_w_a"])
                    E2 = orc.face_point(s, id2, ((p2 + .5) / P - .5) * s["xtal_w_t"],
                                        ((q2 + .5) / Q - .5) * s["xtal_w_a"])
                    r1 = orc.composed(s, t, T, id1, p1, q1, E1 - E2)
                    r2 = orc.composed(s, t, T, id2, p2, q2, E2 - E1)
                    yield r1, r2


@pytest.mark.parametrize("name", ["RING2D", "RING3D_SMALL"])
def test_spread_is_mean_of_rank_one_products(orc, name):
    # Eq. 10: each sub-LOR contributes rho1 (x) rho2; Eq. 12 sums them.
    w = I.workload(name)
    s, t = w["scanner"], w["table"]
    Wt, Wa = w["window"]
    T, _ = orc.table_build(s, t)
    lors = I.workload_lors(w)
    pick = lors[np.random.default_rng(1).choice(len(lors), 6, replace=False)]
    W = orc.spread(s, t, T, pick, Wt, Wa, orc.NORM_NONE)
    for k, (a, b) in enumerate(pick):
        acc = None
        n = 0
        for (e1, _), (e2, _) in _subpairs(orc, s, t, T, a, b):
            o = _outer_window(e1, e2, Wt, Wa)
            acc = o if acc is None else acc + o
            n += 1
        np.testing.assert_allclose(W[k], acc / n, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("name", ["RING2D", "RING3D_SMALL"])
def test_spread_sum_rules(orc, name):
    w = I.workload(name)
    s, t = w["scanner"], w["table"]
    Wt, Wa = w["window"]
    T, _ = orc.table_build(s, t)
    lors = I.workload_lors(w)
    pick = lors[np.random.default_rng(2).choice(len(lors), 5, replace=False)]
    we = orc.spread(s, t, T, pick, Wt, Wa, orc.NORM_EFF)
    wu = orc.spread(s, t, T, pick, Wt, Wa, orc.NORM_UNIT)
    wn = orc.spread(s, t, T, pick, Wt, Wa, orc.NORM_NONE)
    for k, (a, b) in enumerate(pick):
        full = np.mean([r1[1] * r2[1] for r1, r2 in _subpairs(orc, s, t, T, a, b)])
        if full == 0.0:
            assert not we[k].any()
            continue
        assert we[k].sum() == pytest.approx(full, rel=1e-12)
        assert wu[k].sum() == pytest.approx(1.0, rel=1e-12)
        assert wn[k].sum() <= full * (1 + 1e-12)
        np.testing.assert_allclose(we[k] * wn[k].sum(), wn[k] * full, rtol=1e-12, atol=1e-300)


def test_same_block_pairs_have_no_spread(orc):
    w = I.workload("RING2D")
    T, _ = orc.table_build(w["scanner"], w["table"])
    W = orc.spread(w["scanner"], w["table"], T, [[0, 5], [9, 14]], 3, 0)
    assert not W.any()


@pytest.mark.parametrize("name", ["RING2D", "RING3D_SMALL"])
def test_spread_rotation_symmetry(orc, name):
    w = I.workload(name)
    s, t = w["scanner"], w["table"]
    Wt, Wa = w["window"]
    Nb, Nt = s["nt_block"], I.n_transaxial(s)
    T, _ = orc.table_build(s, t)
    lors = I.workload_lors(w)
    lors = lors[(lors[:, 1] % Nt) < Nt - 2 * Nb]
    pick = lors[np.random.default_rng(3).choice(len(lors), 12, replace=False)]
    rot = pick.copy()
    rot[:, 0] += Nb
    rot[:, 1] += Nb
    W0 = orc.spread(s, t, T, pick, Wt, Wa)
    W1 = orc.spread(s, t, T, rot, Wt, Wa)
    np.testing.assert_allclose(W1, W0, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("name", ["RING2D", "RING3D_SMALL"])
def test_spread_mirror_symmetry(orc, name):
    # Mirror through block 0's centre plane: block b -> -b, crystal i -> Nb-1-i,
    # so every transaxial offset changes sign.
    w = I.workload(name)
    s, t = w["scanner"], w["table"]
    Wt, Wa = w["window"]
    Nb, R, Nt = s["nt_block"], s["n_blocks"], I.n_transaxial(s)
    T, _ = orc.table_build(s, t)

    def mir(x):
        ring, c = divmod(int(x), Nt)
        b, i = divmod(c, Nb)
        return ring * Nt + ((-b) % R) * Nb + (Nb - 1 - i)

    lors = I.workload_lors(w)
    pick = lors[np.random.default_rng(4).choice(len(lors), 12, replace=False)]
    mirrored, swapped = [], []
    for a, b in pick:
        ma, mb = mir(a), mir(b)
        if ma % Nt < mb % Nt:
            mirrored.append((ma, mb))
            swapped.append(False)
        else:
            mirrored.append((mb, ma))
            swapped.append(True)
    W0 = orc.spread(s, t, T, pick, Wt, Wa)
    W1 = orc.spread(s, t, T, mirrored, Wt, Wa)
    E = (2 * Wt + 1) * (2 * Wa + 1)
    W2a = 2 * Wa + 1
    flip = np.array([(2 * Wt - e // W2a) * W2a + e % W2a for e in range(E)])
    for k in range(len(pick)):
        want = W0[k][np.ix_(flip, flip)]
        if swapped[k]:
            want = want.T
        np.testing.assert_allclose(W1[k], want, rtol=1e-11, atol=1e-15)


def test_spread_axial_translation(orc):
    w = I.workload("RING3D_SMALL")
    s, t = w["scanner"], w["table"]
    Nt = I.n_transaxial(s)
    T, _ = orc.table_build(s, t)
    base = [[0 * Nt + 1, 2 * Nt + 20], [1 * Nt + 5, 1 * Nt + 27], [3 * Nt + 9, 0 * Nt + 30]]
    moved = [[a + 2 * Nt, b + 2 * Nt] for a, b in base]
    np.testing.assert_allclose(orc.spread(s, t, T, moved, 3, 2), orc.spread(s, t, T, base, 3, 2),
                               rtol=1e-11, atol=1e-15)


def test_spread_axial_mirror(orc):
    """Reflection through the scanner's axial centre plane: ring r -> NR-1-r
    for both crystals (the ring lattice has one pitch, so it maps onto
    itself); every axial offset changes sign and the ring difference with
    it, the transaxial offsets are unchanged."""
    w = I.workload("RING3D_SMALL")
    s, t = w["scanner"], w["table"]
    Wt, Wa = w["window"]
    Nt = I.n_transaxial(s)
    NR = s["n_block_rings"] * s["na_block"]
    T, _ = orc.table_build(s, t)
    lors = I.workload_lors(w)
    pick = lors[np.random.default_rng(5).choice(len(lors), 16, replace=False)]
    assert any(a // Nt != b // Nt for a, b in pick)  # oblique LORs among them
    mirrored = [((NR - 1 - a // Nt) * Nt + a % Nt, (NR - 1 - b // Nt) * Nt + b % Nt)
                for a, b in pick]
    W0 = orc.spread(s, t, T, pick, Wt, Wa)
    W1 = orc.spread(s, t, T, mirrored, Wt, Wa)
    assert (W0.sum(axis=(1, 2)) > 0).sum() >= 12
    W2a = 2 * Wa + 1
    E = (2 * Wt + 1) * W2a
    flip = np.array([(e // W2a) * W2a + (2 * Wa - e % W2a) for e in range(E)])
    for k in range(len(pick)):
        np.testing.assert_allclose(W1[k], W0[k][np.ix_(flip, flip)], rtol=1e-11, atol=1e-15)
