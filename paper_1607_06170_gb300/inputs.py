"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds descriptions and random draws only -- scanner, table and
image descriptions, LOR lists and phantoms -- and none of the method's
arithmetic.  Every draw uses ``numpy.random.default_rng(160706170 + k)`` with
``k`` the index of the workload below, so both sides see identical numbers.

Workloads (named by what they are):

* ``RING2D``   one ring of 8 blocks x 8 crystals (2 x 2 x 10 mm LYSO,
  mu = 0.087/mm) at radius 50 mm; all 2016 crystal-pair LORs; 4 transaxial
  sub-positions (the 4 axial rows of the 4 x 4 entry grid collapse in a
  single-ring scanner); 8 incidence-angle nodes; spread +-3 crystals;
  64 x 64 image of 1 mm pixels; 5 discs + 4 point sources.
* ``RING2D_NARROW``  the same blocks at the radius that leaves a 0.5 mm gap on
  each side of a block corner (test-only, exercises penetration through a
  narrow gap); 24 x 24 image.
* ``RING3D``   24 blocks x 13 x 13 crystals x 4 block rings (312 crystals per
  ring, 52 rings), 1.9 mm crystals on a 2.2 mm pitch, radius 130 mm; 8 x 8
  sub-positions; 32 transaxial x 8 polar angle nodes; LORs with ring
  difference <= 15 and transaxial fan +-104; spread +-3 x +-3;
  160 x 160 x 104 voxels of 0.8 mm; uniform cylinder phantom.
* ``RING3D_SMALL``  a 12-block, 4 x 4-crystal, 2-block-ring scanner with the
  same crystal pitch, for parity tests that the oracle finishes in seconds.
* ``RING2D_ELLIPSES``  the RING2D geometry with an 8-ellipse phantom
  (contrast 1-8), used for the mixed-precision MLEM comparison.
* ``RING3D_GRAD``  the RING3D scanner with 128 x 128 x 104 voxels of 1 mm and
  Poisson counts of mean 20 per LOR, for the differentiation checks.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 160706170


def rng(k: int) -> np.random.Generator:
    return np.random.default_rng(SEED + k)


# ----------------------------------------------------------------- scanners
def scanner(n_blocks, nt_block, na_block, n_block_rings, xtal_w_t, xtal_w_a, depth, gap_t,
            gap_a, radius, block_gap_a, mu) -> dict:
    return dict(n_blocks=n_blocks, nt_block=nt_block, na_block=na_block,
                n_block_rings=n_block_rings, xtal_w_t=xtal_w_t, xtal_w_a=xtal_w_a, depth=depth,
                gap_t=gap_t, gap_a=gap_a, radius=radius, block_gap_a=block_gap_a, mu=mu)


def table(n_ang_t, n_ang_a, n_sub_t, n_sub_a, max_off_t, max_off_a, ang_max_t_deg,
          ang_max_a_deg) -> dict:
    return dict(n_ang_t=n_ang_t, n_ang_a=n_ang_a, n_sub_t=n_sub_t, n_sub_a=n_sub_a,
                max_off_t=max_off_t, max_off_a=max_off_a, ang_max_t_deg=ang_max_t_deg,
                ang_max_a_deg=ang_max_a_deg)


def image(nx, ny, nz, dx, dy, dz) -> dict:
    """Grid centred on the scanner axis; (ox, oy, oz) is the corner of voxel 0."""
    return dict(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
                ox=-0.5 * nx * dx, oy=-0.5 * ny * dy, oz=-0.5 * nz * dz)


def n_crystals(s: dict) -> int:
    return s["n_blocks"] * s["nt_block"] * s["na_block"] * s["n_block_rings"]


def n_transaxial(s: dict) -> int:
    return s["n_blocks"] * s["nt_block"]


def n_rings(s: dict) -> int:
    return s["na_block"] * s["n_block_rings"]


_RING2D_SCANNER = scanner(8, 8, 1, 1, 2.0, 2.0, 10.0, 0.0, 0.0, 50.0, 0.0, 0.087)
# radius for a 0.5 mm gap AB = BC at every block corner: (8 + 0.5) / tan(pi/8)
_NARROW_R = 8.5 / math.tan(math.pi / 8)

WORKLOADS = {
    "RING2D": dict(
        index=0,
        scanner=_RING2D_SCANNER,
        table=table(8, 1, 4, 1, 32, 1, 90.0, 90.0),
        image=image(64, 64, 1, 1.0, 1.0, 1.0),
        window=(3, 0),
        lors=dict(fan_half=31, max_ring_diff=0),
    ),
    "RING2D_NARROW": dict(
        index=10,
        scanner=scanner(8, 8, 1, 1, 2.0, 2.0, 10.0, 0.0, 0.0, _NARROW_R, 0.0, 0.087),
        table=table(8, 1, 4, 1, 32, 1, 90.0, 90.0),
        image=image(24, 24, 1, 1.0, 1.0, 1.0),
        window=(3, 0),
        lors=dict(fan_half=31, max_ring_diff=0),
    ),
    "RING3D": dict(
        index=1,
        scanner=scanner(24, 13, 13, 4, 1.9, 1.9, 10.0, 0.3, 0.3, 130.0, 0.3, 0.087),
        table=table(32, 8, 8, 8, 16, 6, 72.0, 16.0),
        image=image(160, 160, 104, 0.8, 0.8, 0.8),
        window=(3, 3),
        lors=dict(fan_half=104, max_ring_diff=15),
    ),
    "RING3D_SMALL": dict(
        index=11,
        scanner=scanner(12, 4, 4, 2, 1.9, 1.9, 10.0, 0.3, 0.3, 30.0, 0.3, 0.087),
        table=table(13, 4, 4, 4, 16, 8, 65.0, 36.0),
        image=image(24, 24, 16, 1.5, 1.5, 1.1),
        window=(3, 2),
        lors=dict(fan_half=10, max_ring_diff=3),
    ),
    # RING3D_SMALL's blocks stacked 18 high (72 crystal rings): a set whose
    # ring-pair plane needs whole-warp groups in the factored stencil
    "RING3D_TALL": dict(
        index=13,
        scanner=scanner(12, 4, 4, 18, 1.9, 1.9, 10.0, 0.3, 0.3, 30.0, 0.3, 0.087),
        table=table(13, 4, 4, 4, 16, 8, 65.0, 36.0),
        image=image(24, 24, 144, 1.5, 1.5, 1.1),
        window=(3, 2),
        lors=dict(fan_half=2, max_ring_diff=1),
    ),
    "RING2D_ELLIPSES": dict(
        index=2,
        scanner=_RING2D_SCANNER,
        table=table(8, 1, 4, 1, 32, 1, 90.0, 90.0),
        image=image(64, 64, 1, 1.0, 1.0, 1.0),
        window=(3, 0),
        lors=dict(fan_half=31, max_ring_diff=0),
    ),
    # list-mode OSEM: the 3D ring with 8 block rings (104 crystal rings), three
    # uniform spheres of equal concentration, subsets of events
    "RING3D_LM": dict(
        index=4,
        scanner=scanner(24, 13, 13, 8, 1.9, 1.9, 10.0, 0.3, 0.3, 130.0, 0.3, 0.087),
        table=table(32, 8, 8, 8, 16, 6, 72.0, 16.0),
        image=image(200, 200, 208, 0.8, 0.8, 0.8),
        window=(3, 3),
        lors=dict(fan_half=104, max_ring_diff=15),
        listmode=dict(events=10_000_000, subset_events=1_000_000, radii_mm=(5.0, 10.0, 20.0),
                      n_keep=5),
    ),
    "RING3D_SMALL_LM": dict(
        index=12,
        scanner=scanner(12, 4, 4, 2, 1.9, 1.9, 10.0, 0.3, 0.3, 30.0, 0.3, 0.087),
        table=table(13, 4, 4, 4, 16, 8, 65.0, 36.0),
        image=image(24, 24, 16, 1.5, 1.5, 1.1),
        window=(3, 2),
        lors=dict(fan_half=10, max_ring_diff=3),
        listmode=dict(events=20_000, subset_events=5_000, radii_mm=(2.0, 3.0, 4.0), n_keep=5),
    ),
    # the paper's scanner (Sec. 4): 2 rings of 24 modules of 16 x 16 crystals of 2 x 2 x 10 mm
    # on a 2 mm pitch (384 crystals per crystal ring, 32 rings); the radius is not given (125 mm
    # reading); the histogram organisation of Table 1: 192 angles x 199 bins per ring pair,
    # direct and cross planes (ring difference <= 1, 63 slices of 1 mm), 380 x 380 x 63 image
    "EPLUS260": dict(
        index=5,
        scanner=scanner(24, 16, 16, 2, 2.0, 2.0, 10.0, 0.0, 0.0, 125.0, 0.0, 0.087),
        table=table(32, 2, 8, 8, 16, 4, 60.0, 4.0),
        image=image(380, 380, 63, 0.5, 0.5, 1.0),
        window=(3, 1),
        lors=dict(fan_half=99, max_ring_diff=1),
        sino=dict(views=192, bins=199),
    ),
    "RING3D_GRAD": dict(
        index=3,
        scanner=scanner(24, 13, 13, 4, 1.9, 1.9, 10.0, 0.3, 0.3, 130.0, 0.3, 0.087),
        table=table(32, 8, 8, 8, 16, 6, 72.0, 16.0),
        image=image(128, 128, 104, 1.0, 1.0, 1.0),
        window=(3, 3),
        lors=dict(fan_half=104, max_ring_diff=15),
    ),
}


def workload(name: str) -> dict:
    return WORKLOADS[name]


# --------------------------------------------------------------- LOR lists
def transaxial_pairs(s: dict, fan_half: int) -> np.ndarray:
    """Crystal pairs (a, b), a < b, with b - a within fan_half of half the ring.

    Listed lexicographically.  fan_half = Nt/2 - 1 lists every pair.
    """
    nt = n_transaxial(s)
    out = []
    for a in range(nt):
        lo = max(a + 1, a + nt // 2 - fan_half)
        hi = min(nt - 1, a + nt // 2 + fan_half)
        if hi >= lo:
            b = np.arange(lo, hi + 1)
            out.append(np.stack([np.full_like(b, a), b], 1))
    return np.concatenate(out).astype(np.int32)


def ring_pairs(s: dict, max_ring_diff: int) -> np.ndarray:
    """Ordered crystal-ring pairs (ra, rb) with |ra - rb| <= max_ring_diff, lexicographic."""
    nr = n_rings(s)
    ra, rb = np.meshgrid(np.arange(nr), np.arange(nr), indexing="ij")
    keep = np.abs(ra - rb) <= max_ring_diff
    return np.stack([ra[keep], rb[keep]], 1).astype(np.int32)


def lor_list(s: dict, fan_half: int, max_ring_diff: int) -> np.ndarray:
    """LORs as crystal-id pairs (id = ring * Nt + transaxial index).

    Row order: transaxial pair (a, b) major, ring pair (ra, rb) minor; the
    first crystal of each LOR is the one with the smaller transaxial index.
    """
    nt = n_transaxial(s)
    tp = transaxial_pairs(s, fan_half).astype(np.int64)
    rp = ring_pairs(s, max_ring_diff).astype(np.int64)
    a = (rp[None, :, 0] * nt + tp[:, None, 0]).reshape(-1)
    b = (rp[None, :, 1] * nt + tp[:, None, 1]).reshape(-1)
    return np.stack([a, b], 1).astype(np.int32)


def _crystal_hits(s: dict, p, d):
    """Crystal reached by rays from points p along directions d (torch [M, 3]
    float64): the front-face plane of the block the ray leaves the ring
    polygon through, the crystal under the hit point (transaxial pitch, rings
    on a uniform axial pitch centred on z = 0).  Returns (transaxial index,
    ring, ok) with ok False where the hit point falls off the crystal faces
    (block corners, gaps, beyond the rings)."""
    import torch

    R, nb = s["n_blocks"], s["nt_block"]
    nr = n_rings(s)
    pt = s["xtal_w_t"] + s["gap_t"]
    pa = s["xtal_w_a"] + s["gap_a"]
    # the exit through the circumscribed circle picks the block up to one
    # neighbour; the nearest of those three face planes is the polygon's exit
    rc = s["radius"] / math.cos(math.pi / R)
    dxy, pxy = d[:, :2], p[:, :2]
    aa = (dxy * dxy).sum(1)
    bb = (pxy * dxy).sum(1)
    cc = (pxy * pxy).sum(1) - rc * rc
    tc = (-bb + torch.sqrt(torch.clamp(bb * bb - aa * cc, min=0.0))) / aa
    e = pxy + tc[:, None] * dxy
    b0 = torch.round(torch.atan2(e[:, 1], e[:, 0]) / (2 * math.pi / R)).long()
    cand = (b0[:, None] + torch.tensor([-1, 0, 1], device=p.device)[None, :]) % R   # [M, 3]
    phi = (2 * math.pi / R) * cand.double()
    dn = dxy[:, :1] * torch.cos(phi) + dxy[:, 1:] * torch.sin(phi)
    pn = pxy[:, :1] * torch.cos(phi) + pxy[:, 1:] * torch.sin(phi)
    t = torch.where(dn > 1e-12, (s["radius"] - pn) / torch.where(dn > 1e-12, dn, 1.0),
                    torch.full_like(dn, math.inf))
    tm, j = torch.min(t, 1)
    blk = cand.gather(1, j[:, None])[:, 0]
    h = p + torch.where(torch.isfinite(tm), tm, 0.0)[:, None] * d
    pb = (2 * math.pi / R) * blk.double()
    st = -h[:, 0] * torch.sin(pb) + h[:, 1] * torch.cos(pb)
    u = st / pt + 0.5 * (nb - 1)                                    # crystal centres at integers
    i = torch.round(u).long()
    ok = torch.isfinite(tm) & ((u - i).abs() * pt <= 0.5 * s["xtal_w_t"]) & (i >= 0) & (i < nb)
    v = h[:, 2] / pa + 0.5 * (nr - 1)
    r = torch.round(v).long()
    ok &= ((v - r).abs() * pa <= 0.5 * s["xtal_w_a"]) & (r >= 0) & (r < nr)
    return blk * nb + i, r, ok


def listmode_events(w: dict, n: int, k: int, device="cpu"):
    """Coincidence events as crystal-id pairs (torch int32 [n, 2] on `device`,
    id = ring * Nt + transaxial index; the first crystal is the one with the
    smaller transaxial index) from three uniform spheres of equal
    concentration (radii w["listmode"]["radii_mm"], seeded centres inside the
    image), emitted back to back in isotropic directions.  A pair is redrawn
    when a photon misses the crystal faces or the pair is outside the LOR set
    (fan, ring difference).  Directions are drawn uniformly in the band of
    axial direction cosines that can reach an accepted pair (a redraw of the
    rest).  Seeded per device type (torch generators)."""
    import torch

    s, im, ls = w["scanner"], w["image"], w["lors"]
    gen = torch.Generator(device=device).manual_seed(SEED + k)
    radii = torch.tensor(w["listmode"]["radii_mm"], dtype=torch.float64, device=device)
    nt, nr = n_transaxial(s), n_rings(s)
    F, Dm = ls["fan_half"], ls["max_ring_diff"]
    half_xy = 0.5 * min(im["nx"] * im["dx"], im["ny"] * im["dy"])
    half_z = 0.5 * min(im["nz"] * im["dz"], nr * (s["xtal_w_a"] + s["gap_a"]))
    g = rng(k)  # sphere centres from the numpy stream (identical on every device)
    cen = []
    for rs in w["listmode"]["radii_mm"]:
        rho = g.uniform(0.0, max(0.0, 0.8 * half_xy - rs))
        ang = g.uniform(0.0, 2 * np.pi)
        zz = max(0.0, 0.8 * half_z - rs)
        cen.append((rho * np.cos(ang), rho * np.sin(ang), g.uniform(-zz, zz)))
    centres = torch.tensor(cen, dtype=torch.float64, device=device)
    prob = radii ** 3 / (radii ** 3).sum()
    # largest axial slope of an accepted pair: Dm + 1 ring pitches over the shortest chord
    pa = s["xtal_w_a"] + s["gap_a"]
    chord = 2 * s["radius"] * math.sin(math.pi * (nt // 2 - F) / nt)
    slope = 1.25 * (Dm + 1) * pa / chord
    cmax = min(1.0, slope / math.sqrt(1 + slope * slope))
    out, have = [], 0
    f64 = dict(dtype=torch.float64, device=device, generator=gen)
    while have < n:
        m = max(6 * (n - have), 4096)
        sph = torch.multinomial(prob, m, replacement=True, generator=gen)
        dirs = torch.randn((m, 3), **f64)
        dirs /= dirs.norm(dim=1, keepdim=True)
        rad = radii[sph] * torch.rand(m, **f64) ** (1.0 / 3.0)
        p = centres[sph] + rad[:, None] * dirs
        cz = (2 * torch.rand(m, **f64) - 1) * cmax
        az = 2 * math.pi * torch.rand(m, **f64)
        sz = torch.sqrt(1.0 - cz * cz)
        d = torch.stack([sz * torch.cos(az), sz * torch.sin(az), cz], 1)
        c1, r1, ok1 = _crystal_hits(s, p, d)
        c2, r2, ok2 = _crystal_hits(s, p, -d)
        swap = c1 > c2
        a, b = torch.where(swap, c2, c1), torch.where(swap, c1, c2)
        ra, rb = torch.where(swap, r2, r1), torch.where(swap, r1, r2)
        dd = b - a
        ok = ok1 & ok2 & (a != b) & (dd >= nt // 2 - F) & (dd <= nt // 2 + F) & (
            (rb - ra).abs() <= Dm)
        ev = torch.stack([ra * nt + a, rb * nt + b], 1)[ok][: n - have]
        out.append(ev)
        have += ev.shape[0]
    return torch.cat(out).to(torch.int32)


def workload_lors(w: dict) -> np.ndarray:
    return lor_list(w["scanner"], w["lors"]["fan_half"], w["lors"]["max_ring_diff"])


def n_lors(w: dict) -> int:
    s = w["scanner"]
    return len(transaxial_pairs(s, w["lors"]["fan_half"])) * len(
        ring_pairs(s, w["lors"]["max_ring_diff"]))


# ---------------------------------------------------------------- phantoms
def _centres(im: dict):
    x = im["ox"] + (np.arange(im["nx"]) + 0.5) * im["dx"]
    y = im["oy"] + (np.arange(im["ny"]) + 0.5) * im["dy"]
    z = im["oz"] + (np.arange(im["nz"]) + 0.5) * im["dz"]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def _voxel_of(im: dict, x: float, y: float) -> tuple:
    ix = int(math.floor((x - im["ox"]) / im["dx"]))
    iy = int(math.floor((y - im["oy"]) / im["dy"]))
    return ix, iy


def phantom_discs(im: dict, k: int) -> np.ndarray:
    """5 uniform discs (radius U(2,8) mm, activity U(1,10)) + 4 point sources.

    Disc centres are uniform in the disc of radius 0.9*R_fov - r, voxelised by
    pixel-centre inclusion (overlaps add).  Point sources are single pixels of
    value 10: three uniform inside 0.9*R_fov, one at exactly 0.9*R_fov at a
    seeded angle.  R_fov is the image half-width.  Returns float32 [nz,ny,nx].
    """
    g = rng(k)
    X, Y, _ = _centres(im)
    rfov = 0.5 * im["nx"] * im["dx"]
    x = np.zeros(X.shape)
    for _ in range(5):
        r = g.uniform(2.0, 8.0)
        act = g.uniform(1.0, 10.0)
        rr = (0.9 * rfov - r) * math.sqrt(g.uniform())
        th = g.uniform(0.0, 2 * math.pi)
        cx, cy = rr * math.cos(th), rr * math.sin(th)
        x += act * (((X - cx) ** 2 + (Y - cy) ** 2) <= r * r)
    pts = []
    for _ in range(3):
        rr = 0.9 * rfov * math.sqrt(g.uniform())
        th = g.uniform(0.0, 2 * math.pi)
        pts.append((rr * math.cos(th), rr * math.sin(th)))
    th = g.uniform(0.0, 2 * math.pi)
    pts.append((0.9 * rfov * math.cos(th), 0.9 * rfov * math.sin(th)))
    for px, py in pts:
        ix, iy = _voxel_of(im, px, py)
        ix = min(max(ix, 0), im["nx"] - 1)
        iy = min(max(iy, 0), im["ny"] - 1)
        x[:, iy, ix] = 10.0
    return x.astype(np.float32)


def phantom_ellipses(im: dict, k: int) -> np.ndarray:
    """Background disc (radius 0.9*R_fov, activity 1) + 8 seeded ellipses.

    Semi-axes U(2,10) mm, seeded rotation, centres inside the background,
    added activity U(0,7) so the contrast spans 1-8.  float32 [nz,ny,nx].
    """
    g = rng(k)
    X, Y, _ = _centres(im)
    rfov = 0.5 * im["nx"] * im["dx"]
    rb = 0.9 * rfov
    x = 1.0 * ((X ** 2 + Y ** 2) <= rb * rb)
    for _ in range(8):
        a, b = g.uniform(2.0, 10.0), g.uniform(2.0, 10.0)
        rot = g.uniform(0.0, math.pi)
        rr = (rb - max(a, b)) * math.sqrt(g.uniform())
        th = g.uniform(0.0, 2 * math.pi)
        cx, cy = rr * math.cos(th), rr * math.sin(th)
        act = g.uniform(0.0, 7.0)
        u = (X - cx) * math.cos(rot) + (Y - cy) * math.sin(rot)
        v = -(X - cx) * math.sin(rot) + (Y - cy) * math.cos(rot)
        x += act * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
    return x.astype(np.float32)


def phantom_cylinder(im: dict, k: int) -> np.ndarray:
    """Uniform cylinder of radius 0.9*R_fov over the full axial extent, plus
    seeded multiplicative texture U(0.9, 1.1) so no two voxels are equal."""
    g = rng(k)
    X, Y, _ = _centres(im)
    rfov = 0.5 * im["nx"] * im["dx"]
    inside = (X ** 2 + Y ** 2) <= (0.9 * rfov) ** 2
    tex = g.uniform(0.9, 1.1, size=X.shape)
    return (inside * tex).astype(np.float32)


def random_image(im: dict, k: int, lo=0.0, hi=1.0) -> np.ndarray:
    return rng(k).uniform(lo, hi, size=(im["nz"], im["ny"], im["nx"])).astype(np.float32)


def random_lor_values(n: int, k: int, lo=0.0, hi=1.0) -> np.ndarray:
    return rng(k).uniform(lo, hi, size=n).astype(np.float32)


def poisson_counts(mean: np.ndarray, k: int) -> np.ndarray:
    return rng(k).poisson(np.asarray(mean, dtype=np.float64)).astype(np.float32)
