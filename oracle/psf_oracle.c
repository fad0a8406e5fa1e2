/*
 * psf_oracle.c -- plain FP64 CPU oracle for the P-SPIR PSF system matrix
 * (Sun et al., "Fast and accurate generation method of PSF-based system
 * matrix for PET reconstruction", Chinese Physics C, 2016).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check of the package entry and
 * the CPU-baseline leg of the benchmark do.  It shares no code, header, table
 * or constant with the CUDA library; both sides receive the same plain
 * numbers (scanner, table and image descriptions, LOR lists, images) from the
 * seeded input module.
 *
 * Everything is double precision and written to be checked against the paper
 * by eye, not to be fast: brute-force box clipping instead of incremental
 * tracing, dense accumulators, no symmetry reuse.  OpenMP only splits
 * independent LORs across threads.
 *
 * Readings of passages where the paper is silent or garbled are stated at the
 * function that takes them.  Parity status per function:
 *   orc_trace_response  pinned (closed form, Monte Carlo, normalisation sums)
 *   orc_table_build     pinned (via orc_trace_response + node grid checks)
 *   orc_composed        pinned (sigma=0, R->inf reduction to one flat array)
 *   orc_spread          pinned (rank-1 case, sum rules, ring symmetries)
 *   orc_siddon          pinned (axis-aligned chords, brute slab-clip tracer)
 *   orc_rows_psf        pinned (definition A = S G checked on scatter identity)
 *   orc_csr_fwd / back  pinned (dot-product identity, MLEM count identity)
 *   orc_spread_topn     pinned (N = whole window is the identity, sum rule,
 *                       ranking against a brute-force order, tie rules)
 *   orc_sino_index      pinned (one to one onto views x bins; bins ordered by
 *                       the geometric offset within a view, views by angle)
 *   orc_voxel_homog     pinned (column sums against the composed efficiencies,
 *                       quarter-turn symmetry, centre pixel)
 *   agreement of the analytic response with GATE: parity unpinned (the
 *   paper's response curves, Figs. 2-5, are not in the text).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------------- */
/* Geometry (Sec. 3 scanner description; Fig. 6 for the block layout)     */
/* ---------------------------------------------------------------------- */

typedef struct {
    int R;          /* blocks per ring (R of Eq. 2)                         */
    int Nb;         /* transaxial crystals per block                        */
    int Na;         /* axial crystals per block                             */
    int NBR;        /* block rings                                          */
    double wt, wa;  /* crystal face width, transaxial (lambda of Eq. 5) / axial */
    double depth;   /* crystal depth                                        */
    double gt, ga;  /* air gap between neighbouring crystals inside a block */
    double radius;  /* scanner axis to the block front-face centre          */
    double bga;     /* axial air gap between block rings                    */
    double mu;      /* linear attenuation coefficient (1/mm)                */
} orc_scanner;

typedef struct {
    int Kt, Ka;           /* angle nodes: transaxial / polar                */
    int Pt, Pa;           /* sub-positions per crystal face (x of Sec. 2.1.1) */
    int Mt, Ma;           /* stored crystal offsets along travel            */
    double amax_t_deg;    /* node spacing = amax / K                        */
    double amax_a_deg;
} orc_table;

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double ox, oy, oz;    /* corner of voxel (0,0,0)                        */
} orc_image;

static int orc_nt(const orc_scanner *s) { return s->R * s->Nb; }
static int orc_nrings(const orc_scanner *s) { return s->NBR * s->Na; }
static double orc_pt(const orc_scanner *s) { return s->wt + s->gt; }
static double orc_pa(const orc_scanner *s) { return s->wa + s->ga; }
static double orc_block_width(const orc_scanner *s)
{
    return s->Nb * s->wt + (s->Nb - 1) * s->gt;
}

/* Gap sigma = AB = BC of Fig. 6: B is where the front-face lines of two
 * neighbouring blocks meet, C the corner of block0 and A the corner of
 * block1.  The face line of a block lies at distance `radius` from the axis,
 * so B sits r*tan(pi/R) from the block centre along the face. */
double orc_sigma(const orc_scanner *s)
{
    return s->radius * tan(ORC_PI / s->R) - 0.5 * orc_block_width(s);
}

/* Axial centre of crystal ring k; rings are centred on z = 0. */
static double orc_ring_z(const orc_scanner *s, int k)
{
    int br = k / s->Na, ia = k % s->Na;
    double H = s->Na * s->wa + (s->Na - 1) * s->ga;
    double Z = s->NBR * H + (s->NBR - 1) * s->bga;
    return br * (H + s->bga) + ia * orc_pa(s) + 0.5 * s->wa - 0.5 * Z;
}

/* Crystal id = ring * Nt + block * Nb + i.  Block b is centred at angle
 * 2 pi b / R; crystal i of a block sits at tangential offset
 * (i - (Nb-1)/2) * pitch, the index growing counter-clockwise. */
typedef struct {
    int ring, block, i, ct;
    double n[2], t[2];        /* outward normal, counter-clockwise tangent */
    double s_centre;          /* tangential coordinate of the crystal centre */
    double z_centre;
} orc_xtal;

static orc_xtal orc_decode(const orc_scanner *s, int id)
{
    orc_xtal x;
    int Nt = orc_nt(s);
    x.ring = id / Nt;
    x.ct = id % Nt;
    x.block = x.ct / s->Nb;
    x.i = x.ct % s->Nb;
    double phi = 2.0 * ORC_PI * x.block / s->R;
    x.n[0] = cos(phi);
    x.n[1] = sin(phi);
    x.t[0] = -sin(phi);
    x.t[1] = cos(phi);
    x.s_centre = (x.i - 0.5 * (s->Nb - 1)) * orc_pt(s);
    x.z_centre = orc_ring_z(s, x.ring);
    return x;
}

/* Point on the front face of crystal `id`, displaced by (off_t, off_a) from
 * the face centre along the tangent and the axis. */
void orc_face_point(const orc_scanner *s, int id, double off_t, double off_a,
                    double P[3])
{
    orc_xtal x = orc_decode(s, id);
    double st = x.s_centre + off_t;
    P[0] = s->radius * x.n[0] + st * x.t[0];
    P[1] = s->radius * x.n[1] + st * x.t[1];
    P[2] = x.z_centre + off_a;
}

/* ---------------------------------------------------------------------- */
/* Single-photon response (Sec. 2.1.1, Eq. 1; normalisation Sec. 2.1.3)   */
/* ---------------------------------------------------------------------- */

/*
 * Response of one ray entering a flat crystal array (Sec. 2.1.1).  The paper
 * counts M_i/M (Eq. 1) in a GATE simulation; here the count ratio is replaced
 * by its analytic expectation without scatter: the probability that the first
 * interaction happens in crystal i is exp(-mu * L_before) * (1 - exp(-mu L_i)),
 * with L_i the path length inside crystal i and L_before the path length in
 * crystal material met earlier along the ray (gaps are air).
 *
 * Frame of the array: x lateral along the transaxial travel direction, y
 * axial along the axial travel direction, z depth from the front face.
 * Crystal (kx, ky) occupies [kx*pt, kx*pt+wt] x [ky*pa, ky*pa+wa] x [0, D].
 * The ray enters crystal (0,0) at (u*wt, v*wa, 0): u, v are measured from the
 * crystal edge the ray moves away from.  Its direction has transaxial angle
 * alpha_t to the face normal (in the transaxial plane) and polar angle theta
 * to the transaxial plane, i.e. per unit depth it moves tan(alpha_t)
 * laterally and tan(theta)/cos(alpha_t) axially.
 *
 * T[kx*My + ky] receives the first-interaction probability of crystal (kx,ky)
 * for kx < Mx, ky < My.  *eta receives the total over all crystals the ray
 * meets (the counting rate eta of Eq. 6 for unit activity and time), so that
 * rho = eta * rho0 (Eq. 7) with rho0 = T / eta summing to one.
 *
 * Each crystal box is clipped against the ray independently (slab method),
 * and the attenuation before a crystal is the sum over the boxes the ray
 * entered earlier.
 */
void orc_trace_response(const orc_scanner *s, double alpha_t, double theta,
                        double u, double v, int Mx, int My, double *T,
                        double *eta)
{
    const double pt = orc_pt(s), pa = orc_pa(s), D = s->depth;
    const double tx = tan(alpha_t), ty = tan(theta) / cos(alpha_t);
    const double x0 = u * s->wt, y0 = v * s->wa;
    const double ds = sqrt(1.0 + tx * tx + ty * ty);
    int kxmax = (int)floor((x0 + D * tx) / pt) + 1;
    int kymax = (int)floor((y0 + D * ty) / pa) + 1;
    int nbox = (kxmax + 1) * (kymax + 1);
    double *zin = (double *)malloc(sizeof(double) * nbox);
    double *len = (double *)malloc(sizeof(double) * nbox);
    int *kxs = (int *)malloc(sizeof(int) * nbox);
    int *kys = (int *)malloc(sizeof(int) * nbox);
    int nb = 0;
    for (int kx = 0; kx <= kxmax; ++kx) {
        for (int ky = 0; ky <= kymax; ++ky) {
            double lo = 0.0, hi = D;
            double ax = kx * pt, bx = ax + s->wt;
            double ay = ky * pa, by = ay + s->wa;
            if (tx > 0.0) {
                double z0 = (ax - x0) / tx, z1 = (bx - x0) / tx;
                if (z0 > lo) lo = z0;
                if (z1 < hi) hi = z1;
            } else if (!(x0 >= ax && x0 <= bx)) {
                continue;
            }
            if (ty > 0.0) {
                double z0 = (ay - y0) / ty, z1 = (by - y0) / ty;
                if (z0 > lo) lo = z0;
                if (z1 < hi) hi = z1;
            } else if (!(y0 >= ay && y0 <= by)) {
                continue;
            }
            if (hi > lo) {
                zin[nb] = lo;
                len[nb] = (hi - lo) * ds;
                kxs[nb] = kx;
                kys[nb] = ky;
                ++nb;
            }
        }
    }
    for (int k = 0; k < Mx * My; ++k) T[k] = 0.0;
    double total = 0.0;
    for (int a = 0; a < nb; ++a) {
        double before = 0.0;
        for (int b = 0; b < nb; ++b)
            if (zin[b] < zin[a]) before += len[b];
        double p = exp(-s->mu * before) * (1.0 - exp(-s->mu * len[a]));
        total += p;
        if (kxs[a] < Mx && kys[a] < My) T[kxs[a] * My + kys[a]] = p;
    }
    *eta = total;
    free(zin);
    free(len);
    free(kxs);
    free(kys);
}

/* Table layout: T[((((kt*Ka + ka)*Pt + iu)*Pa + iv)*Mt + dx)*Ma + dz],
 * eta[((kt*Ka + ka)*Pt + iu)*Pa + iv]. */
static size_t orc_tidx(const orc_table *tb, int kt, int ka, int iu, int iv)
{
    return (((size_t)kt * tb->Ka + ka) * tb->Pt + iu) * tb->Pa + iv;
}

/*
 * The P-SPIR table (Sec. 2.1.1): one response per incidence angle and entry
 * sub-position.  Reading of the angle grid: the SPIR model samples the
 * incidence angle on a uniform grid starting at 0 (0..60 degrees in 5-degree
 * steps); here node k sits at k * amax / K degrees, k = 0..K-1.  Each crystal
 * bar is divided into P equal parts (x = 8 in the paper); sub-position p is
 * evaluated at its centre (p + 1/2) / P.
 */
void orc_table_build(const orc_scanner *s, const orc_table *tb, double *T,
                     double *eta)
{
    const double dt = tb->amax_t_deg / tb->Kt * ORC_PI / 180.0;
    const double da = tb->amax_a_deg / tb->Ka * ORC_PI / 180.0;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int kt = 0; kt < tb->Kt; ++kt)
        for (int ka = 0; ka < tb->Ka; ++ka)
            for (int iu = 0; iu < tb->Pt; ++iu)
                for (int iv = 0; iv < tb->Pa; ++iv) {
                    size_t e = orc_tidx(tb, kt, ka, iu, iv);
                    orc_trace_response(s, kt * dt, ka * da,
                                       (iu + 0.5) / tb->Pt, (iv + 0.5) / tb->Pa,
                                       tb->Mt, tb->Ma,
                                       T + e * tb->Mt * tb->Ma, eta + e);
                }
}

/* Nearest node of the grid (reading of the table lookup; no interpolation). */
int orc_node(double ang, double amax_deg, int K)
{
    double step = amax_deg / K * ORC_PI / 180.0;
    int k = (int)floor(ang / step + 0.5);
    return k > K - 1 ? K - 1 : k;
}

/* ---------------------------------------------------------------------- */
/* Response seen from the ring, with two-block penetration (Sec. 2.1.2)   */
/* ---------------------------------------------------------------------- */

typedef struct {
    int dt;       /* transaxial offset in ring crystal index (wraps mod Nt) */
    int da;       /* crystal-ring offset                                    */
    double val;   /* first-interaction probability                          */
} orc_entry;

/*
 * Gap construction of Fig. 6 for a photon entering block0 at distance nu from
 * its edge C (nu = CP0) with incidence angle alpha toward block1:
 *   beta = alpha - 2 pi / R                                        (Eq. 2)
 *   AP1  = sigma + sin(pi/2 - alpha) / sin(pi/2 + beta) * (sigma + nu)  (Eq. 4)
 * (the law of sines in triangle B P0 P1, whose angle at B is 2 pi / R).
 * *run receives the side P0 P1 of the same triangle, the transaxial distance
 * the photon covers between P0 and the extended face line BD of block1.
 */
void orc_gap_eq(const orc_scanner *s, double alpha, double nu, double *beta,
                double *AP1, double *run)
{
    double sigma = orc_sigma(s);
    *beta = alpha - 2.0 * ORC_PI / s->R;
    *AP1 = sigma + sin(0.5 * ORC_PI - alpha) / sin(0.5 * ORC_PI + *beta) * (sigma + nu);
    *run = (sigma + nu) * sin(2.0 * ORC_PI / s->R) / sin(0.5 * ORC_PI + *beta);
}

/*
 * Response of the crystals around crystal `id` to a photon that enters its
 * front face at sub-position (ipt, ipa) -- indices counted from the -tangent
 * and -axial edges -- travelling along `dir` (any length, pointing out of the
 * ring).  Offsets are in ring crystal index and crystal ring.
 *
 * Block0 (the struck block) takes the table entries of its own crystals;
 * entries that would lie beyond its lateral edge are dropped.  If the
 * incidence angle exceeds the angle between neighbouring block normals, the
 * neighbouring block in the travel direction (block1) is reached through the
 * gap by the construction of Fig. 6:
 *   beta = alpha - 2 pi / R                                   (Eq. 2)
 *   AP1  = sigma + sin(pi/2 - alpha) / sin(pi/2 + beta) * (sigma + nu)  (Eq. 4)
 *   n    = AP1 / lambda                                       (Eq. 5)
 * with nu = CP0 the distance from the entry point to the block edge.  The
 * photon is taken to enter a virtual crystal of block1's array, extended
 * beyond its corner A, at distance AP1 from A; block1's real crystal j (j = 0
 * next to A) then sits floor(n) + 1 + j crystals further along the travel
 * direction, and its response is read from the same table at (beta, the
 * entry position within the virtual crystal).
 * Readings: with intra-block gaps the virtual crystals repeat with the block
 * pitch, and an entry point that falls into a virtual gap enters the next
 * virtual crystal toward A at its trailing edge.  In 3D the transaxial
 * construction is done in the transaxial projection (the polar angle is
 * unchanged by the rotation between blocks), and the axial entry position is
 * the ray's axial coordinate at P1 on a uniform ring lattice.
 *
 * Returns the number of entries written to out; *eta_out receives their sum.
 */
int orc_composed(const orc_scanner *s, const orc_table *tb, const double *T,
                 int id, int ipt, int ipa, const double dir[3],
                 orc_entry *out, int cap, double *eta_out)
{
    orc_xtal x = orc_decode(s, id);
    double vn = dir[0] * x.n[0] + dir[1] * x.n[1];
    double vt = dir[0] * x.t[0] + dir[1] * x.t[1];
    double vz = dir[2];
    int ne = 0;
    *eta_out = 0.0;
    if (!(vn > 0.0)) return 0;
    double alpha = atan2(fabs(vt), vn);
    double theta = atan2(fabs(vz), sqrt(vn * vn + vt * vt));
    int sgt = vt >= 0.0 ? 1 : -1;
    int sga = vz >= 0.0 ? 1 : -1;
    int iu = sgt > 0 ? ipt : tb->Pt - 1 - ipt;
    int iv = sga > 0 ? ipa : tb->Pa - 1 - ipa;
    int kt = orc_node(alpha, tb->amax_t_deg, tb->Kt);
    int ka = orc_node(theta, tb->amax_a_deg, tb->Ka);
    const double *Tb = T + orc_tidx(tb, kt, ka, iu, iv) * tb->Mt * tb->Ma;
    double sum = 0.0;

    /* block0: crystals i + sgt*dx inside the block */
    for (int dx = 0; dx < tb->Mt; ++dx) {
        int ii = x.i + sgt * dx;
        if (ii < 0 || ii >= s->Nb) break;
        for (int dz = 0; dz < tb->Ma; ++dz) {
            double val = Tb[dx * tb->Ma + dz];
            if (val == 0.0) continue;
            if (ne < cap) {
                out[ne].dt = sgt * dx;
                out[ne].da = sga * dz;
                out[ne].val = val;
            }
            ++ne;
            sum += val;
        }
    }

    /* block1 through the gap (Eq. 2, 4, 5) */
    double beta, AP1, run;
    orc_gap_eq(s, alpha, 0.5 * orc_block_width(s) -
                   sgt * (x.s_centre + ((ipt + 0.5) / tb->Pt - 0.5) * s->wt),
               &beta, &AP1, &run);
    if (beta > 0.0) {
        double ze = x.z_centre + ((ipa + 0.5) / tb->Pa - 0.5) * s->wa;
        double pt = orc_pt(s);
        double q = AP1 - s->gt;
        if (q < 0.0) q = 0.0;
        int m = (int)floor(q / pt);
        double f = q - m * pt;
        double u1 = f < s->wt ? (s->wt - f) / s->wt : 0.0;
        int iu1 = (int)floor(u1 * tb->Pt);
        if (iu1 > tb->Pt - 1) iu1 = tb->Pt - 1;
        double z1 = ze + sga * run * tan(theta);
        double pa = orc_pa(s);
        double zlo0 = orc_ring_z(s, 0) - 0.5 * s->wa;
        int k1 = (int)floor((z1 - zlo0) / pa);
        double fa = (z1 - zlo0) - k1 * pa;
        double v1;
        if (fa <= s->wa) {
            v1 = sga > 0 ? fa / s->wa : (s->wa - fa) / s->wa;
        } else {
            if (sga > 0) k1 += 1;
            v1 = 0.0;
        }
        int iv1 = (int)floor(v1 * tb->Pa);
        if (iv1 > tb->Pa - 1) iv1 = tb->Pa - 1;
        int kt1 = orc_node(beta, tb->amax_t_deg, tb->Kt);
        const double *T1 = T + orc_tidx(tb, kt1, ka, iu1, iv1) * tb->Mt * tb->Ma;
        for (int j = 0; j < s->Nb; ++j) {
            int dx = m + 1 + j;
            if (dx >= tb->Mt) break;
            int dt = sgt > 0 ? (s->Nb - x.i + j) : -(x.i + 1 + j);
            for (int dz = 0; dz < tb->Ma; ++dz) {
                double val = T1[dx * tb->Ma + dz];
                if (val == 0.0) continue;
                if (ne < cap) {
                    out[ne].dt = dt;
                    out[ne].da = (k1 - x.ring) + sga * dz;
                    out[ne].val = val;
                }
                ++ne;
                sum += val;
            }
        }
    }
    *eta_out = sum;
    return ne;
}

/* ---------------------------------------------------------------------- */
/* Homogenization spread of a LOR (Sec. 2.2 Eq. 10, Sec. 2.3 Eq. 11-12)   */
/* ---------------------------------------------------------------------- */

enum { ORC_NORM_NONE = 0, ORC_NORM_EFF = 1, ORC_NORM_UNIT = 2 };

/*
 * Spread of each listed LOR (crystal ids lors[2k], lors[2k+1]) over the
 * crystal pairs within +-Wt transaxially and +-Wa axially of its two ends.
 *
 * Reading of the homogenization model: the equally weighted LORs through the
 * emission point are taken as the sub-LORs that join the sub-position centres
 * of the two crystal faces (Pt*Pa positions per face, every pairing equally
 * weighted).  Each sub-LOR gives the detected pair (c1+d1, c2+d2) the product
 * of the two single-photon responses (Eq. 10); summing over sub-LORs is the
 * sum of Eq. 12.  Pairs of crystals in the same block get no spread (their
 * chord runs along the block face and enters neither crystal).
 *
 * Output w[k][e1][e2], e = (dt + Wt)*(2Wa+1) + (da + Wa), end 1 = lors[2k].
 * Normalisation (the paper fixes none):
 *   NONE: the truncated window as summed;
 *   EFF : rescaled so the window total equals the untruncated total
 *         mean over sub-LORs of eta1*eta2 (the efficiency of Eq. 7 is kept,
 *         the truncation loss is returned);
 *   UNIT: rescaled to total one.
 */
void orc_spread(const orc_scanner *s, const orc_table *tb, const double *T,
                const int32_t *lors, int64_t n, int Wt, int Wa, int norm,
                double *w)
{
    const int E = (2 * Wt + 1) * (2 * Wa + 1);
    const int cap = 4 * (tb->Mt * tb->Ma) + 16;
#pragma omp parallel
    {
        orc_entry *r1 = (orc_entry *)malloc(sizeof(orc_entry) * cap);
        orc_entry *r2 = (orc_entry *)malloc(sizeof(orc_entry) * cap);
#pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < n; ++k) {
            double *acc = w + (size_t)k * E * E;
            for (int e = 0; e < E * E; ++e) acc[e] = 0.0;
            int id1 = lors[2 * k], id2 = lors[2 * k + 1];
            orc_xtal x1 = orc_decode(s, id1), x2 = orc_decode(s, id2);
            if (x1.block == x2.block) continue;
            double sfull = 0.0;
            for (int p1 = 0; p1 < tb->Pt; ++p1)
            for (int q1 = 0; q1 < tb->Pa; ++q1)
            for (int p2 = 0; p2 < tb->Pt; ++p2)
            for (int q2 = 0; q2 < tb->Pa; ++q2) {
                double E1[3], E2[3], d1[3], d2[3];
                orc_face_point(s, id1, ((p1 + 0.5) / tb->Pt - 0.5) * s->wt,
                               ((q1 + 0.5) / tb->Pa - 0.5) * s->wa, E1);
                orc_face_point(s, id2, ((p2 + 0.5) / tb->Pt - 0.5) * s->wt,
                               ((q2 + 0.5) / tb->Pa - 0.5) * s->wa, E2);
                for (int c = 0; c < 3; ++c) {
                    d1[c] = E1[c] - E2[c];
                    d2[c] = -d1[c];
                }
                double eta1, eta2;
                int n1 = orc_composed(s, tb, T, id1, p1, q1, d1, r1, cap, &eta1);
                int n2 = orc_composed(s, tb, T, id2, p2, q2, d2, r2, cap, &eta2);
                sfull += eta1 * eta2;
                for (int a = 0; a < n1; ++a) {
                    if (abs(r1[a].dt) > Wt || abs(r1[a].da) > Wa) continue;
                    int e1 = (r1[a].dt + Wt) * (2 * Wa + 1) + (r1[a].da + Wa);
                    for (int b = 0; b < n2; ++b) {
                        if (abs(r2[b].dt) > Wt || abs(r2[b].da) > Wa) continue;
                        int e2 = (r2[b].dt + Wt) * (2 * Wa + 1) + (r2[b].da + Wa);
                        acc[e1 * E + e2] += r1[a].val * r2[b].val;
                    }
                }
            }
            double nsub = (double)tb->Pt * tb->Pa * tb->Pt * tb->Pa;
            double swin = 0.0;
            for (int e = 0; e < E * E; ++e) {
                acc[e] /= nsub;
                swin += acc[e];
            }
            sfull /= nsub;
            double scale = 1.0;
            if (norm == ORC_NORM_EFF && swin > 0.0) scale = sfull / swin;
            if (norm == ORC_NORM_UNIT && swin > 0.0) scale = 1.0 / swin;
            for (int e = 0; e < E * E; ++e) acc[e] *= scale;
        }
        free(r1);
        free(r2);
    }
}

/*
 * Diagnostic for parity tests: the smallest distance, over every sub-LOR of
 * each listed LOR, between a rounding decision of orc_composed and its
 * boundary -- nearest angle node (in node spacings), and on the gap path the
 * virtual crystal / sub-position / ring decisions (in their own spacings).
 * A LOR whose margin is below the working precision of another implementation
 * has more than one correct spread.  Decisions that cannot change the result
 * (a gap path that reaches no crystal) are not counted.
 */
static double frac_margin(double x)
{
    return fabs(x - rint(x));
}

/* Smallest margin of the response decisions of one end: crystal x entered at
 * sub-position (ipt, ipa) travelling along d (out of the ring). */
static double end_margin(const orc_scanner *s, const orc_table *tb, const double *T,
                         orc_xtal x, int ipt, int ipa, const double d[3])
{
    double best = 1.0;
    double vn = d[0] * x.n[0] + d[1] * x.n[1];
    double vt = d[0] * x.t[0] + d[1] * x.t[1];
    if (!(vn > 0.0)) return best;
    double alpha = atan2(fabs(vt), vn);
    double theta = atan2(fabs(d[2]), sqrt(vn * vn + vt * vt));
    double st = tb->amax_t_deg / tb->Kt * ORC_PI / 180.0;
    double sa = tb->amax_a_deg / tb->Ka * ORC_PI / 180.0;
    /* nearest node: boundaries where angle/step + 1/2 is an integer */
    if (alpha / st < tb->Kt - 1) best = fmin(best, frac_margin(alpha / st + 0.5));
    if (theta / sa < tb->Ka - 1) best = fmin(best, frac_margin(theta / sa + 0.5));
    int sgt = vt >= 0.0 ? 1 : -1, sga = d[2] >= 0.0 ? 1 : -1;
    double beta, AP1, run;
    orc_gap_eq(s, alpha, 0.5 * orc_block_width(s) -
                   sgt * (x.s_centre + ((ipt + 0.5) / tb->Pt - 0.5) * s->wt),
               &beta, &AP1, &run);
    if (!(beta > 0.0)) return best;
    /* does the gap path reach any stored crystal? */
    double q = AP1 - s->gt;
    if (q < 0.0) q = 0.0;
    int m = (int)floor(q / orc_pt(s));
    int kt1 = orc_node(beta, tb->amax_t_deg, tb->Kt);
    int ka = orc_node(theta, tb->amax_a_deg, tb->Ka);
    double reach = 0.0;
    for (int iu = 0; iu < tb->Pt; ++iu)
        for (int iv = 0; iv < tb->Pa; ++iv)
            for (int dx = m; dx < tb->Mt && dx <= m + 2; ++dx)
                for (int dz = 0; dz < tb->Ma; ++dz)
                    reach += T[(orc_tidx(tb, kt1, ka, iu, iv) * tb->Mt + dx) * tb->Ma + dz];
    if (reach == 0.0) return best;
    if (beta / st < tb->Kt - 1) best = fmin(best, frac_margin(beta / st + 0.5));
    best = fmin(best, frac_margin(q / orc_pt(s)));
    double f = q - m * orc_pt(s);
    best = fmin(best, fabs(f - s->wt) / orc_pt(s));
    if (f < s->wt) best = fmin(best, frac_margin((s->wt - f) / s->wt * tb->Pt));
    if (tb->Pa > 1 || orc_nrings(s) > 1) {
        double z1 = x.z_centre + ((ipa + 0.5) / tb->Pa - 0.5) * s->wa +
                    sga * run * tan(theta);
        double zl = z1 - (orc_ring_z(s, 0) - 0.5 * s->wa);
        best = fmin(best, frac_margin(zl / orc_pa(s)));
        double fa = zl - floor(zl / orc_pa(s)) * orc_pa(s);
        best = fmin(best, fabs(fa - s->wa) / orc_pa(s));
        if (fa <= s->wa) best = fmin(best, frac_margin(fa / s->wa * tb->Pa));
    }
    return best;
}

/* Smallest margin of the decisions for one sub-LOR (both ends). */
static double subpair_margin(const orc_scanner *s, const orc_table *tb, const double *T,
                             int id1, int id2, int p1, int q1, int p2, int q2)
{
    orc_xtal x1 = orc_decode(s, id1), x2 = orc_decode(s, id2);
    double E1[3], E2[3], d1[3], d2[3];
    orc_face_point(s, id1, ((p1 + 0.5) / tb->Pt - 0.5) * s->wt,
                   ((q1 + 0.5) / tb->Pa - 0.5) * s->wa, E1);
    orc_face_point(s, id2, ((p2 + 0.5) / tb->Pt - 0.5) * s->wt,
                   ((q2 + 0.5) / tb->Pa - 0.5) * s->wa, E2);
    for (int c = 0; c < 3; ++c) {
        d1[c] = E1[c] - E2[c];
        d2[c] = -d1[c];
    }
    return fmin(end_margin(s, tb, T, x1, p1, q1, d1), end_margin(s, tb, T, x2, p2, q2, d2));
}

/* Per LOR: the smallest margin over its sub-LORs (margin) and the number of
 * its sub-LORs whose margin is below tau (count, may be NULL). */
void orc_tie_stats(const orc_scanner *s, const orc_table *tb, const double *T,
                   const int32_t *lors, int64_t n, double tau, double *margin, int64_t *count)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < n; ++k) {
        int id1 = lors[2 * k], id2 = lors[2 * k + 1];
        double best = 1.0;
        int64_t nb = 0;
        if (orc_decode(s, id1).block != orc_decode(s, id2).block) {
            for (int p1 = 0; p1 < tb->Pt; ++p1)
            for (int q1 = 0; q1 < tb->Pa; ++q1)
            for (int p2 = 0; p2 < tb->Pt; ++p2)
            for (int q2 = 0; q2 < tb->Pa; ++q2) {
                double mg = subpair_margin(s, tb, T, id1, id2, p1, q1, p2, q2);
                best = fmin(best, mg);
                nb += mg < tau;
            }
        }
        margin[k] = best;
        if (count) count[k] = nb;
    }
}

void orc_tie_margin(const orc_scanner *s, const orc_table *tb, const double *T,
                    const int32_t *lors, int64_t n, double *margin)
{
    orc_tie_stats(s, tb, T, lors, n, 0.0, margin, NULL);
}

/* ---------------------------------------------------------------------- */
/* Geometric rows: chord lengths of a segment through the voxel grid      */
/* ---------------------------------------------------------------------- */

/*
 * Reading of "a segment lying on a grid plane belongs to the voxel above": the
 * crystal positions of a ring are computed with rounded sines and cosines, so
 * a LOR that lies on a grid plane by symmetry comes out tilted by ~1e-15 mm.
 * A coordinate that changes by less than 1e-9 voxel over the whole segment is
 * taken as constant, and a constant coordinate within 1e-9 voxel of a plane
 * is taken to lie on it.  Returns 1 and the voxel index for such an axis.
 */
static int orc_parallel_axis(double a, double b, double o, double d, int *idx)
{
    if (!(fabs((b - a) / d) < 1e-9)) return 0;
    double u = (a - o) / d;
    if (fabs(u - rint(u)) < 1e-9) u = rint(u);
    *idx = (int)floor(u);
    return 1;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

typedef struct { int64_t idx; double len; } orc_vl;
static int cmp_vl(const void *a, const void *b)
{
    int64_t x = ((const orc_vl *)a)->idx, y = ((const orc_vl *)b)->idx;
    return (x > y) - (x < y);
}

/*
 * Chord lengths (mm) of the segment a->b through the voxels of `im`, by the
 * parametric method: every grid-plane crossing inside the grid is collected,
 * the parameters are sorted, and each interval between consecutive crossings
 * belongs to the voxel containing its midpoint.  Voxels are half-open
 * [lo, hi) on every axis, so a segment lying on a grid plane belongs to the
 * voxel above it.  Output sorted by voxel index (x fastest); returns the
 * count, or -1 if cap is too small.
 */
int orc_siddon(const orc_image *im, const double a[3], const double b[3],
               int64_t *idx, double *len, int cap)
{
    const int nn[3] = {im->nx, im->ny, im->nz};
    const double dd[3] = {im->dx, im->dy, im->dz};
    const double oo[3] = {im->ox, im->oy, im->oz};
    double d[3], L = 0.0;
    for (int c = 0; c < 3; ++c) {
        d[c] = b[c] - a[c];
        L += d[c] * d[c];
    }
    L = sqrt(L);
    double amin = 0.0, amax = 1.0;
    int par[3], fix[3];
    for (int c = 0; c < 3; ++c) {
        double lo = oo[c], hi = oo[c] + nn[c] * dd[c];
        par[c] = orc_parallel_axis(a[c], b[c], oo[c], dd[c], &fix[c]);
        if (!par[c]) {
            double t0 = (lo - a[c]) / d[c], t1 = (hi - a[c]) / d[c];
            if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
            if (t0 > amin) amin = t0;
            if (t1 < amax) amax = t1;
        } else if (fix[c] < 0 || fix[c] >= nn[c]) {
            return 0;
        }
    }
    if (!(amax > amin)) return 0;
    int np = 2 + nn[0] + nn[1] + nn[2] + 3;
    double *al = (double *)malloc(sizeof(double) * np);
    int k = 0;
    al[k++] = amin;
    al[k++] = amax;
    for (int c = 0; c < 3; ++c) {
        if (par[c]) continue;
        for (int i = 0; i <= nn[c]; ++i) {
            double t = (oo[c] + i * dd[c] - a[c]) / d[c];
            if (t > amin && t < amax) al[k++] = t;
        }
    }
    qsort(al, k, sizeof(double), cmp_double);
    orc_vl *tmp = (orc_vl *)malloc(sizeof(orc_vl) * (k + 1));
    int nv = 0;
    for (int j = 0; j + 1 < k; ++j) {
        if (!(al[j + 1] > al[j])) continue;
        double mid = 0.5 * (al[j] + al[j + 1]);
        int v[3], ok = 1;
        for (int c = 0; c < 3; ++c) {
            v[c] = par[c] ? fix[c] : (int)floor((a[c] + mid * d[c] - oo[c]) / dd[c]);
            if (v[c] < 0 || v[c] >= nn[c]) ok = 0;
        }
        if (!ok) continue;
        tmp[nv].idx = ((int64_t)v[2] * nn[1] + v[1]) * nn[0] + v[0];
        tmp[nv].len = (al[j + 1] - al[j]) * L;
        ++nv;
    }
    qsort(tmp, nv, sizeof(orc_vl), cmp_vl);
    int out = 0;
    for (int j = 0; j < nv; ++j) {
        if (out > 0 && idx && idx[out - 1] == tmp[j].idx) {
            len[out - 1] += tmp[j].len;
            continue;
        }
        if (out >= cap) { out = -1; break; }
        idx[out] = tmp[j].idx;
        len[out] = tmp[j].len;
        ++out;
    }
    free(al);
    free(tmp);
    return out;
}

/*
 * Second, independent tracer for small grids: clip the segment against every
 * voxel box separately (slab method, half-open boxes) and keep positive
 * chords.  Same output convention as orc_siddon.
 */
int orc_slabclip(const orc_image *im, const double a[3], const double b[3],
                 int64_t *idx, double *len, int cap)
{
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const int nn[3] = {im->nx, im->ny, im->nz};
    const double dd[3] = {im->dx, im->dy, im->dz};
    const double oo[3] = {im->ox, im->oy, im->oz};
    int out = 0;
    int par[3], fix[3];
    for (int c = 0; c < 3; ++c) par[c] = orc_parallel_axis(a[c], b[c], oo[c], dd[c], &fix[c]);
    for (int iz = 0; iz < nn[2]; ++iz)
    for (int iy = 0; iy < nn[1]; ++iy)
    for (int ix = 0; ix < nn[0]; ++ix) {
        int v[3] = {ix, iy, iz};
        double t0 = 0.0, t1 = 1.0;
        int ok = 1;
        for (int c = 0; c < 3 && ok; ++c) {
            double lo = oo[c] + v[c] * dd[c], hi = lo + dd[c];
            if (par[c]) {
                if (fix[c] != v[c]) ok = 0;
            } else if (d[c] != 0.0) {
                double s0 = (lo - a[c]) / d[c], s1 = (hi - a[c]) / d[c];
                if (s0 > s1) { double t = s0; s0 = s1; s1 = t; }
                if (s0 > t0) t0 = s0;
                if (s1 < t1) t1 = s1;
            } else if (!(a[c] >= lo && a[c] < hi)) {
                ok = 0;
            }
        }
        if (!ok || !(t1 > t0)) continue;
        if (out >= cap) return -1;
        idx[out] = ((int64_t)iz * nn[1] + iy) * nn[0] + ix;
        len[out] = (t1 - t0) * L;
        ++out;
    }
    return out;
}

/* Geometric LOR of a crystal pair: front-face centre to front-face centre. */
static void orc_lor_ends(const orc_scanner *s, int id1, int id2, double a[3],
                         double b[3])
{
    orc_face_point(s, id1, 0.0, 0.0, a);
    orc_face_point(s, id2, 0.0, 0.0, b);
}

/* Row lengths of the geometric matrix G for a LOR list (first pass). */
void orc_rows_geom_count(const orc_scanner *s, const orc_image *im,
                         const int32_t *lors, int64_t n, int64_t *counts)
{
    int cap = im->nx + im->ny + im->nz + 8;
#pragma omp parallel
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t k = 0; k < n; ++k) {
            double a[3], b[3];
            orc_lor_ends(s, lors[2 * k], lors[2 * k + 1], a, b);
            counts[k] = orc_siddon(im, a, b, idx, len, cap);
        }
        free(idx);
        free(len);
    }
}

/* Fill G in CSR given row_ptr from the counts. */
void orc_rows_geom_fill(const orc_scanner *s, const orc_image *im,
                        const int32_t *lors, int64_t n, const int64_t *row_ptr,
                        int64_t *col, double *val)
{
    int cap = im->nx + im->ny + im->nz + 8;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
        double a[3], b[3];
        orc_lor_ends(s, lors[2 * k], lors[2 * k + 1], a, b);
        orc_siddon(im, a, b, col + row_ptr[k], val + row_ptr[k], cap);
    }
}

/*
 * Measured crystal pair that window entry (e1, e2) of a LOR lands on.
 * Transaxial indices wrap around the ring; crystal rings outside the scanner
 * and pairs of one crystal with itself give -1.  Otherwise the two crystal
 * ids are written to X, Y.
 */
int orc_window_pair(const orc_scanner *s, int id1, int id2, int Wt, int Wa,
                    int e1, int e2, int *X, int *Y)
{
    int Nt = orc_nt(s), NR = orc_nrings(s);
    int W2a = 2 * Wa + 1;
    int dt1 = e1 / W2a - Wt, da1 = e1 % W2a - Wa;
    int dt2 = e2 / W2a - Wt, da2 = e2 % W2a - Wa;
    int r1 = id1 / Nt + da1, r2 = id2 / Nt + da2;
    if (r1 < 0 || r1 >= NR || r2 < 0 || r2 >= NR) return -1;
    int c1 = ((id1 % Nt + dt1) % Nt + Nt) % Nt;
    int c2 = ((id2 % Nt + dt2) % Nt + Nt) % Nt;
    *X = r1 * Nt + c1;
    *Y = r2 * Nt + c2;
    if (*X == *Y) return -1;
    return 0;
}

/*
 * PSF rows, dense: A[m][v] = sum over listed LORs g and window entries
 * (e1,e2) landing on the pair of LOR m of w_g[e1][e2] * G_g[v]
 * (Sec. 2.3: each geometric LOR's photons are detected on the neighbouring
 * crystal pairs with the proportions of Eq. 12).  `pair_row` maps an
 * unordered crystal pair (X*Ncrys + Y, both orders) to its row or -1.
 * Small problems only: A is n x nvox doubles.
 */
void orc_rows_psf_dense(const orc_scanner *s, int64_t n, const int32_t *lors,
                        const int64_t *g_ptr, const int64_t *g_col,
                        const double *g_val, const double *w, int Wt, int Wa,
                        const int64_t *pair_row, int64_t nvox, double *A)
{
    const int E = (2 * Wt + 1) * (2 * Wa + 1);
    const int64_t Nc = (int64_t)orc_nt(s) * orc_nrings(s);
    memset(A, 0, sizeof(double) * n * nvox);
    for (int64_t g = 0; g < n; ++g) {
        for (int e1 = 0; e1 < E; ++e1)
            for (int e2 = 0; e2 < E; ++e2) {
                double wv = w[(size_t)g * E * E + e1 * E + e2];
                if (wv == 0.0) continue;
                int X, Y;
                if (orc_window_pair(s, lors[2 * g], lors[2 * g + 1], Wt, Wa, e1, e2, &X, &Y))
                    continue;
                int64_t m = pair_row[(int64_t)X * Nc + Y];
                if (m < 0) continue;
                for (int64_t j = g_ptr[g]; j < g_ptr[g + 1]; ++j)
                    A[m * nvox + g_col[j]] += wv * g_val[j];
            }
    }
}

/* ---------------------------------------------------------------------- */
/* Projectors (used inside MLEM, Sec. 3)                                  */
/* ---------------------------------------------------------------------- */

void orc_csr_fwd(int64_t n, const int64_t *ptr, const int64_t *col,
                 const double *val, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n; ++m) {
        double acc = 0.0;
        for (int64_t j = ptr[m]; j < ptr[m + 1]; ++j) acc += val[j] * x[col[j]];
        y[m] = acc;
    }
}

void orc_csr_back(int64_t n, const int64_t *ptr, const int64_t *col,
                  const double *val, const double *y, int64_t nvox, double *x)
{
    memset(x, 0, sizeof(double) * nvox);
    for (int64_t m = 0; m < n; ++m)
        for (int64_t j = ptr[m]; j < ptr[m + 1]; ++j) x[col[j]] += val[j] * y[m];
}

/*
 * Factored PSF projection y = S (G x) for a LOR list: p = G x on the
 * geometric LORs, then each LOR's p is spread onto the measured pairs of its
 * window with the weights w (the same proportions as orc_rows_psf_dense,
 * without forming A).  Both directions, plain loops.
 */
void orc_spread_apply(const orc_scanner *s, int64_t n, const int32_t *lors,
                      const double *w, int Wt, int Wa, const int64_t *pair_row,
                      const double *p, double *y)
{
    const int E = (2 * Wt + 1) * (2 * Wa + 1);
    const int64_t Nc = (int64_t)orc_nt(s) * orc_nrings(s);
    memset(y, 0, sizeof(double) * n);
    for (int64_t g = 0; g < n; ++g) {
        if (p[g] == 0.0) continue;
        for (int e1 = 0; e1 < E; ++e1)
            for (int e2 = 0; e2 < E; ++e2) {
                double wv = w[(size_t)g * E * E + e1 * E + e2];
                if (wv == 0.0) continue;
                int X, Y;
                if (orc_window_pair(s, lors[2 * g], lors[2 * g + 1], Wt, Wa, e1, e2, &X, &Y))
                    continue;
                int64_t m = pair_row[(int64_t)X * Nc + Y];
                if (m >= 0) y[m] += wv * p[g];
            }
    }
}

void orc_spread_adjoint(const orc_scanner *s, int64_t n, const int32_t *lors,
                        const double *w, int Wt, int Wa, const int64_t *pair_row,
                        const double *r, double *q)
{
    const int E = (2 * Wt + 1) * (2 * Wa + 1);
    const int64_t Nc = (int64_t)orc_nt(s) * orc_nrings(s);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < n; ++g) {
        double acc = 0.0;
        for (int e1 = 0; e1 < E; ++e1)
            for (int e2 = 0; e2 < E; ++e2) {
                double wv = w[(size_t)g * E * E + e1 * E + e2];
                if (wv == 0.0) continue;
                int X, Y;
                if (orc_window_pair(s, lors[2 * g], lors[2 * g + 1], Wt, Wa, e1, e2, &X, &Y))
                    continue;
                int64_t m = pair_row[(int64_t)X * Nc + Y];
                if (m >= 0) acc += wv * r[m];
            }
        q[g] = acc;
    }
}

/*
 * Top-N truncation of each LOR's spread (Sec. 4.3 and Table 3: the extended
 * bins are kept in descending order of their proportion, up to N of them).
 * Readings where the paper is silent:
 *   - the N entries are taken over the LOR's whole window (both ends'
 *     transaxial and axial offsets), since here the window, not a per-angle
 *     bin list, holds the extended bins;
 *   - entries rank by weight (a negative weight ranks as 0); equal weights
 *     rank the entry with the smaller offset |dt1|+|da1|+|dt2|+|da2| first,
 *     then the lower window index e1*E + e2;
 *   - the kept weights are rescaled so that they sum to the untruncated
 *     window's total (the LOR's detection efficiency is kept); a LOR whose
 *     kept weights sum to 0 keeps them unscaled.
 * The ranking compares the given values exactly, so FP32-representable
 * inputs rank as they do in FP32.  w, out: n x E*E; idx: n x N window
 * indices in rank order.
 */
static int orc_topn_E, orc_topn_W2a, orc_topn_Wt, orc_topn_Wa;
static const double *orc_topn_w;

static int orc_topn_dist(int e)
{
    int E = orc_topn_E, W2a = orc_topn_W2a;
    int e1 = e / E, e2 = e % E;
    int dt1 = e1 / W2a - orc_topn_Wt, da1 = e1 % W2a - orc_topn_Wa;
    int dt2 = e2 / W2a - orc_topn_Wt, da2 = e2 % W2a - orc_topn_Wa;
    return abs(dt1) + abs(da1) + abs(dt2) + abs(da2);
}

/* qsort order: rank 0 first (larger weight, then smaller offset, then lower index) */
static int orc_topn_cmp(const void *pa, const void *pb)
{
    int a = *(const int *)pa, b = *(const int *)pb;
    double wa = orc_topn_w[a] > 0.0 ? orc_topn_w[a] : 0.0;
    double wb = orc_topn_w[b] > 0.0 ? orc_topn_w[b] : 0.0;
    if (wa != wb) return wa > wb ? -1 : 1;
    int da = orc_topn_dist(a), db = orc_topn_dist(b);
    if (da != db) return da < db ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

void orc_spread_topn(int64_t n, const double *w, int Wt, int Wa, int N, double *out,
                     int32_t *idx)
{
    const int E = (2 * Wt + 1) * (2 * Wa + 1), EE = E * E;
    int *order = (int *)malloc(sizeof(int) * EE);
    orc_topn_E = E;
    orc_topn_W2a = 2 * Wa + 1;
    orc_topn_Wt = Wt;
    orc_topn_Wa = Wa;
    for (int64_t g = 0; g < n; ++g) {
        const double *wg = w + (size_t)g * EE;
        double *og = out + (size_t)g * EE;
        for (int e = 0; e < EE; ++e) order[e] = e;
        orc_topn_w = wg;
        qsort(order, EE, sizeof(int), orc_topn_cmp);
        double all = 0.0, kept = 0.0;
        for (int e = 0; e < EE; ++e) all += wg[e];
        for (int k = 0; k < N; ++k) kept += wg[order[k]];
        double scale = kept != 0.0 ? all / kept : 1.0;
        memset(og, 0, sizeof(double) * EE);
        for (int k = 0; k < N; ++k) {
            og[order[k]] = wg[order[k]] * scale;
            idx[(size_t)g * N + k] = order[k];
        }
    }
    free(order);
}

/*
 * Sinogram indexing of the histogram organisation (Sec. 4, Table 1: 192
 * angles x 199 bins per angle for 384 crystals per ring).  Reading (the
 * paper gives only the sizes): the ideal-ring convention.  For the pair of
 * transaxial indices a < b with d = b - a within F of N/2, u = a + b:
 *   view = (u mod N) / 2          (two adjacent sums per view: interleaving)
 *   bin  = sg * (d - N/2) + F,    sg = +1 if u < N, else -1
 * which maps the (2F+1) N/2 pairs one to one onto views x bins.
 */
void orc_sino_index(const orc_scanner *s, int a, int b, int F, int *view, int *bin)
{
    int N = orc_nt(s), u = a + b, d = b - a;
    *view = (u % N) / 2;
    *bin = (u < N ? 1 : -1) * (d - N / 2) + F;
}

/* Normal angle phi in [0, pi) and signed distance from the axis of the
 * transaxial line joining the face centres of crystals a and b (ring 0). */
void orc_lor_normal(const orc_scanner *s, int a, int b, double *phi, double *dist)
{
    double A[3], B[3];
    orc_face_point(s, a, 0.0, 0.0, A);
    orc_face_point(s, b, 0.0, 0.0, B);
    double tx = B[0] - A[0], ty = B[1] - A[1];
    double nx = ty, ny = -tx, L = sqrt(nx * nx + ny * ny);
    nx /= L;
    ny /= L;
    double ph = atan2(ny, nx);
    if (ph < 0.0) {
        ph += ORC_PI;
        nx = -nx;
        ny = -ny;
    }
    if (ph >= ORC_PI) {
        ph -= ORC_PI;
        nx = -nx;
        ny = -ny;
    }
    *phi = ph;
    *dist = A[0] * nx + A[1] * ny;
}

/*
 * Voxel-driven homogenization (Sec. 2.3, Eq. 11-12, Figs. 7-8): the paper's
 * own generator, for a planar (single crystal ring) scanner.  A point source
 * at each pixel centre emits k lines, theta_i = pi i / k (Eq. 11), with equal
 * proportion 1/k.  Each line reaches a crystal at both ends: the block whose
 * front-face plane it leaves the ring polygon through, the crystal under the
 * hit point; a hit in an inter-crystal gap or off the faces gives nothing (the
 * paper: a gamma through the gap has proportion zero).  The photon enters
 * that crystal at the sub-position cell of the face holding the hit point
 * (cells of width wt / Pt counted from the -tangent edge; a hit on a cell
 * boundary is shared half and half by the two cells, which keeps the
 * scanner's mirror symmetry), and the
 * single-photon responses of the two ends (orc_composed: block0 and the gap
 * path to block1) give the detected pair (c1 + d1, c2 + d2) the proportion
 * rho1[d1] rho2[d2] (Eq. 10, summed as Eq. 12), over the +-Wt window.
 *   A[m][v] = (1/k) sum_i sum_{d1,d2 -> pair m} rho1[d1] rho2[d2]
 * dense (nrows x nvox, rows by pair_row).  margin[v]: the smallest distance,
 * over the lines of pixel v, of a response decision to its boundary -- the
 * node and gap-path decisions of end_margin, in their own spacings (the cell
 * decision is exact by the sharing rule).
 */

/* Entries of the ray from c along d into the crystal faces: the block whose
 * face plane the ray leaves the ring polygon through, the crystal and
 * sub-position cell under the hit point, with weight 1; a hit within 1e-9
 * cell of a cell boundary lies on it and is shared half and half by the two
 * cells (the neighbouring crystal's edge cell at a crystal edge with no gap;
 * nothing past a block edge or into a gap).  Returns the number of entries
 * (0..2) written to id/ipt/wgt. */
static int orc_ray_entry(const orc_scanner *s, const orc_table *tb, const double c[3],
                         const double d[3], int id[2], int ipt[2], double wgt[2])
{
    int best = -1;
    double tmin = 1e300;
    for (int b = 0; b < s->R; ++b) {
        double phi = 2.0 * ORC_PI * b / s->R;
        double dn = d[0] * cos(phi) + d[1] * sin(phi);
        if (!(dn > 1e-15)) continue;
        double t = (s->radius - (c[0] * cos(phi) + c[1] * sin(phi))) / dn;
        if (t > 0.0 && t < tmin) {
            tmin = t;
            best = b;
        }
    }
    if (best < 0) return 0;
    double phi = 2.0 * ORC_PI * best / s->R;
    double hx = c[0] + tmin * d[0], hy = c[1] + tmin * d[1];
    double st = -hx * sin(phi) + hy * cos(phi);  /* tangential coordinate on the face */
    /* position in sub-position cells of the face lattice: crystal i spans
     * cells [i * Pp, i * Pp + Pt) with Pp = Pt * pitch / width cells per pitch */
    double Pp = tb->Pt * orc_pt(s) / s->wt;
    double u = (st + 0.5 * orc_block_width(s)) / s->wt * tb->Pt;
    int on = fabs(u - rint(u)) < 1e-9;
    if (on) u = rint(u);
    int n = 0;
    for (int side = 0; side < (on ? 2 : 1); ++side) {
        double uu = on ? u - 0.5 + side : u;  /* the cell below / above a boundary */
        int i = (int)floor(uu / Pp);
        if (i < 0 || i >= s->Nb) continue;
        double cell = uu - i * Pp;
        if (cell >= tb->Pt) continue;  /* in the gap after crystal i */
        id[n] = best * s->Nb + i;
        ipt[n] = (int)floor(cell);
        wgt[n] = on ? 0.5 : 1.0;
        ++n;
    }
    return n;
}

void orc_voxel_homog(const orc_scanner *s, const orc_table *tb, const double *T,
                     const orc_image *im, int k, int Wt, const int64_t *pair_row,
                     int64_t nrows, double *A, double *margin)
{
    const int64_t nvox = (int64_t)im->nx * im->ny;
    const int64_t Nc = (int64_t)orc_nt(s) * orc_nrings(s);
    const int cap = 4 * (tb->Mt * tb->Ma) + 16;
    memset(A, 0, sizeof(double) * nrows * nvox);
#pragma omp parallel
    {
        orc_entry *r1 = (orc_entry *)malloc(sizeof(orc_entry) * cap);
        orc_entry *r2 = (orc_entry *)malloc(sizeof(orc_entry) * cap);
#pragma omp for schedule(dynamic, 16)
        for (int64_t v = 0; v < nvox; ++v) {
            int ix = (int)(v % im->nx), iy = (int)(v / im->nx);
            double c[3] = {im->ox + (ix + 0.5) * im->dx, im->oy + (iy + 0.5) * im->dy,
                           orc_ring_z(s, 0)};
            double mg = 1.0;
            for (int i = 0; i < k; ++i) {
                double th = ORC_PI * i / k;
                double d1[3] = {cos(th), sin(th), 0.0}, d2[3] = {-d1[0], -d1[1], 0.0};
                int ia[2], ib[2], pa[2], pb[2];
                double wa[2], wb[2];
                int na = orc_ray_entry(s, tb, c, d1, ia, pa, wa);
                int nb = orc_ray_entry(s, tb, c, d2, ib, pb, wb);
                for (int ea = 0; ea < na; ++ea)
                for (int eb = 0; eb < nb; ++eb) {
                    orc_xtal x1 = orc_decode(s, ia[ea]), x2 = orc_decode(s, ib[eb]);
                    if (x1.block == x2.block) continue;
                    mg = fmin(mg, end_margin(s, tb, T, x1, pa[ea], 0, d1));
                    mg = fmin(mg, end_margin(s, tb, T, x2, pb[eb], 0, d2));
                    double e1, e2, wl = wa[ea] * wb[eb] / k;
                    int n1 = orc_composed(s, tb, T, ia[ea], pa[ea], 0, d1, r1, cap, &e1);
                    int n2 = orc_composed(s, tb, T, ib[eb], pb[eb], 0, d2, r2, cap, &e2);
                    for (int a = 0; a < n1; ++a) {
                        if (abs(r1[a].dt) > Wt || r1[a].da != 0) continue;
                        int X = ((x1.ct + r1[a].dt) % orc_nt(s) + orc_nt(s)) % orc_nt(s);
                        for (int b = 0; b < n2; ++b) {
                            if (abs(r2[b].dt) > Wt || r2[b].da != 0) continue;
                            int Y = ((x2.ct + r2[b].dt) % orc_nt(s) + orc_nt(s)) % orc_nt(s);
                            if (X == Y) continue;
                            int64_t m = pair_row[(int64_t)X * Nc + Y];
                            if (m >= 0) A[m * nvox + v] += r1[a].val * r2[b].val * wl;
                        }
                    }
                }
            }
            margin[v] = mg;
        }
        free(r1);
        free(r2);
    }
}

/* Number of OpenMP threads the oracle runs with (for the baseline record). */
int orc_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
