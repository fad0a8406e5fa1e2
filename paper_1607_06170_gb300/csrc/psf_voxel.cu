// Voxel-driven homogenization (Sec. 2.3, Eq. 11-12, Figs. 7-8), the paper's
// own matrix generator, for a planar (single crystal ring) scanner: a point
// source at each pixel centre emits k lines at theta_i = pi i / k with equal
// proportion 1/k; each line enters a crystal face at both ends and the
// detected pair (c1 + d1, c2 + d2) receives rho1[d1] rho2[d2] / k (Eq. 10,
// summed as Eq. 12) over the +-half_t window.  The hit geometry is FP64 (the
// sub-position decision of a hit on a cell boundary must not depend on
// rounding: such a hit is shared half and half by the two cells); the
// responses are the spread's (end_response: block0 and the gap path).
#include "psf_common.cuh"
#include "psf_end.cuh"
#include "psf_lorset.cuh"

namespace psf {

constexpr int VH_T = 256;
constexpr int VH_MAX_ROWS = 16384;  // one pixel's column in shared memory

struct VhGeom {
    int R, Nb, Pt;
    double radius, wt, pt, width;  // width: transaxial block width
};

// Entries of the ray from (cx, cy) along (dx, dy) into the crystal faces: the
// block whose face plane it leaves the ring polygon through, the crystal and
// sub-position cell under the hit point (weight 1; a hit within 1e-9 cell of a
// cell boundary is shared by the two cells, weight 1/2 each, nothing past a
// block edge or into a gap).  Returns the number of entries (0..2).
__device__ int vh_entry(const VhGeom &g, double cx, double cy, double dx, double dy, int blk[2],
                        int xi[2], int ipt[2], float wgt[2]) {
    int best = -1;
    double tmin = 1e300;
    for (int b = 0; b < g.R; ++b) {
        double sb, cb;
        sincospi(2.0 * b / g.R, &sb, &cb);
        const double dn = dx * cb + dy * sb;
        if (!(dn > 1e-15)) continue;
        const double t = (g.radius - (cx * cb + cy * sb)) / dn;
        if (t > 0.0 && t < tmin) {
            tmin = t;
            best = b;
        }
    }
    if (best < 0) return 0;
    double sb, cb;
    sincospi(2.0 * best / g.R, &sb, &cb);
    const double hx = cx + tmin * dx, hy = cy + tmin * dy;
    const double st = -hx * sb + hy * cb;  // tangential coordinate on the face
    // cells of the face lattice: crystal i spans cells [i Pp, i Pp + Pt)
    const double Pp = g.Pt * g.pt / g.wt;
    double u = (st + 0.5 * g.width) / g.wt * g.Pt;
    const bool on = fabs(u - rint(u)) < 1e-9;
    if (on) u = rint(u);
    int n = 0;
    for (int side = 0; side < (on ? 2 : 1); ++side) {
        const double uu = on ? u - 0.5 + side : u;
        const int i = (int)floor(uu / Pp);
        if (i < 0 || i >= g.Nb) continue;
        const double cell = uu - i * Pp;
        if (cell >= g.Pt) continue;  // in the gap after crystal i
        blk[n] = best;
        xi[n] = i;
        ipt[n] = (int)floor(cell);
        wgt[n] = on ? 0.5f : 1.0f;
        ++n;
    }
    return n;
}

// One CTA per pixel; its threads take the lines and add the pair products to
// the pixel's column in shared memory, written out once.
__global__ void __launch_bounds__(VH_T) voxel_homog_kernel(VhGeom g, Scan sc, Tab tb,
                                                           const float *__restrict__ T,
                                                           const double *__restrict__ eta,
                                                           Img im, LorSet ls, int k, int Wt,
                                                           float *__restrict__ A) {
    extern __shared__ float vh_col[];  // [n_rows]
    int32_t *tp_start = reinterpret_cast<int32_t *>(vh_col + ls.ntp);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    const int t = threadIdx.x;
    ls.stage_prefix(tp_start, rp_start);
    const int64_t nvox = (int64_t)im.nx * im.ny;
    const int nrows = (int)ls.ntp;  // one crystal ring: rows are transaxial pairs
    const float inv_k = 1.0f / (float)k;
    for (int64_t v = blockIdx.x; v < nvox; v += gridDim.x) {
        __syncthreads();  // the previous pixel's column is written out
        for (int m = t; m < nrows; m += VH_T) vh_col[m] = 0.0f;
        __syncthreads();
        const int ix = (int)(v % im.nx), iy = (int)(v / im.nx);
        const double cx = im.ox + (ix + 0.5) * im.dx, cy = im.oy + (iy + 0.5) * im.dy;
        for (int i = t; i < k; i += VH_T) {
            double sth, cth;
            sincospi((double)i / k, &sth, &cth);
            int b1[2], x1[2], p1[2], b2[2], x2[2], p2[2];
            float w1[2], w2[2];
            const int n1 = vh_entry(g, cx, cy, cth, sth, b1, x1, p1, w1);
            const int n2 = vh_entry(g, cx, cy, -cth, -sth, b2, x2, p2, w2);
            for (int e1 = 0; e1 < n1; ++e1)
                for (int e2 = 0; e2 < n2; ++e2) {
                    if (b1[e1] == b2[e2]) continue;
                    EndResp r1, r2;
                    float s1, c1, s2, c2;
                    sincospif(2.0f * b1[e1] / sc.R, &s1, &c1);
                    sincospif(2.0f * b2[e2] / sc.R, &s2, &c2);
                    const float se1 = (x1[e1] - 0.5f * (sc.Nb - 1)) * sc.pt +
                                      ((p1[e1] + 0.5f) / tb.Pt - 0.5f) * sc.wt;
                    const float se2 = (x2[e2] - 0.5f * (sc.Nb - 1)) * sc.pt +
                                      ((p2[e2] + 0.5f) / tb.Pt - 0.5f) * sc.wt;
                    end_response(sc, tb, T, eta, x1[e1], 0, c1, s1, p1[e1], 0, se1, sc.z0,
                                 (float)cth, (float)sth, 0.0f, Wt, 0, r1);
                    end_response(sc, tb, T, eta, x2[e2], 0, c2, s2, p2[e2], 0, se2, sc.z0,
                                 (float)-cth, (float)-sth, 0.0f, Wt, 0, r2);
                    if (!r1.valid || !r2.valid) continue;
                    const float wl = w1[e1] * w2[e2] * inv_k;
                    const int ct1 = b1[e1] * sc.Nb + x1[e1], ct2 = b2[e2] * sc.Nb + x2[e2];
                    for (int a = 0; a <= Wt; ++a) {
                        const float q1 = r1.q[a];
                        if (q1 == 0.0f) continue;
                        int X = ct1 + r1.sgt * a;
                        X += X < 0 ? sc.Nt : (X >= sc.Nt ? -sc.Nt : 0);
                        for (int bb = 0; bb <= Wt; ++bb) {
                            const float q2 = r2.q[bb];
                            if (q2 == 0.0f) continue;
                            int Y = ct2 + r2.sgt * bb;
                            Y += Y < 0 ? sc.Nt : (Y >= sc.Nt ? -sc.Nt : 0);
                            if (X == Y) continue;
                            const int lo = X < Y ? X : Y, hi = X < Y ? Y : X;
                            if (!ls.member(lo, hi, 0, 0)) continue;
                            const int64_t m = ls.row_of(tp_start, rp_start, lo, hi, 0, 0);
                            atomicAdd(vh_col + m, q1 * q2 * wl);
                        }
                    }
                }
        }
        __syncthreads();
        for (int m = t; m < nrows; m += VH_T) A[(int64_t)m * nvox + v] = vh_col[m];
    }
}

}  // namespace psf

using namespace psf;

extern "C" int psf_voxel_homog(const psf_scanner *scanner, const psf_table_desc *desc,
                               const float *table, const double *eta, const psf_image *image,
                               const psf_lor_set *set, int32_t k, int32_t half_t, float *A,
                               void *stream) {
    PSF_RANGE("psf_voxel_homog");
    Scan sc;
    Tab tb;
    Img im;
    LorSet ls;
    int rc = make_scan(scanner, &sc);
    if (rc) return rc;
    rc = make_tab(desc, sc, &tb, true);
    if (rc) return rc;
    rc = make_img(image, &im);
    if (rc) return rc;
    rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    if (ls.NR != 1 || im.nz != 1 || k < 1 || half_t < 0 || half_t + 1 > SP_QMAX) return PSF_EINVAL;
    if (ls.ntp > VH_MAX_ROWS || ls.ntp * (int64_t)im.nx * im.ny > ((int64_t)1 << 31)) return PSF_EINVAL;
    if (!table || !eta || !A) return PSF_EINVAL;
    VhGeom g;
    g.R = scanner->n_blocks;
    g.Nb = scanner->nt_block;
    g.Pt = desc->n_sub_t;
    g.radius = scanner->radius;
    g.wt = scanner->xtal_w_t;
    g.pt = scanner->xtal_w_t + scanner->gap_t;
    g.width = scanner->nt_block * scanner->xtal_w_t + (scanner->nt_block - 1) * scanner->gap_t;
    cudaStream_t st = as_stream(stream);
    const size_t shm = sizeof(float) * ls.ntp + sizeof(int32_t) * (ls.Nt + ls.NR + 2);
    PSF_TRY(cudaFuncSetAttribute(voxel_homog_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shm));
    const int64_t nvox = (int64_t)im.nx * im.ny;
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)(nvox < (int64_t)sms * 8 ? nvox : (int64_t)sms * 8);
    {
        PSF_TIMED("voxel_homog_kernel", st);
        voxel_homog_kernel<<<grid, VH_T, shm, st>>>(g, sc, tb, table, eta, im, ls, k, half_t, A);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}
