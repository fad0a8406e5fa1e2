// Single-photon response seen from the ring, with the neighbouring-block path
// (Sec. 2.1.1-2.1.3, Sec. 2.1.2 Eq. 2, 4, 5), restricted to the quadrant of
// the spread window the photon travels into.  Host-callable so the same code
// can be exercised off the GPU.
#pragma once

#include "psf_common.cuh"

namespace psf {

constexpr int SP_QMAX = 16;  // (half_t+1)*(half_a+1) <= 16

struct EndResp {
    float q[SP_QMAX];  // quadrant-local: q[dxq*(Wa+1) + dzq], |dt| = dxq, |da| = dzq
    double eta;        // total over all crystals reached (block0 + block1)
    int sgt, sga;
    bool valid;
};

// Response of the crystals around the entry crystal (block-local index i,
// crystal ring `ring`, block trig cb/sb) to a photon entering the face at
// geometric sub-position (p, q) -- counted from the -tangent / -axial edges --
// at tangential coordinate s_entry and axial coordinate z_entry, travelling
// along d (pointing out of the ring).
__host__ __device__ __forceinline__ void end_response(const Scan &sc, const Tab &tb,
                                             const float *__restrict__ T,
                                             const double *__restrict__ eta, int i, int ring,
                                             float cb, float sb, int p, int q, float s_entry,
                                             float z_entry, float dx, float dy, float dz, int Wt,
                                             int Wa, EndResp &r) {
#pragma unroll
    for (int k = 0; k < SP_QMAX; ++k) r.q[k] = 0.0f;
    r.eta = 0.0;
    float vn = dx * cb + dy * sb;
    float vt = dy * cb - dx * sb;
    r.sgt = vt >= 0.0f ? 1 : -1;
    r.sga = dz >= 0.0f ? 1 : -1;
    r.valid = vn > 0.0f;
    if (!r.valid) return;
    float alpha = atan2f(fabsf(vt), vn);
    float theta = atan2f(fabsf(dz), sqrtf(vn * vn + vt * vt));
    int iu = r.sgt > 0 ? p : tb.Pt - 1 - p;
    int iv = r.sga > 0 ? q : tb.Pa - 1 - q;
    int kt = angle_node(alpha, tb.inv_dt, tb.Kt);
    int ka = angle_node(theta, tb.inv_da, tb.Ka);
    const int MM = tb.Mt * tb.Ma;
    int64_t ent = table_entry(tb, kt, ka, iu, iv);
    const float *Tb = T + ent * MM;
    const double *Eb = eta + ent * (tb.Mt + 1);
    const int W1 = Wa + 1;
    int edge = r.sgt > 0 ? sc.Nb - 1 - i : i;  // crystals of block0 beyond the entry one
    int nx0 = min(min(edge, Wt), tb.Mt - 1);
    int nz0 = min(Wa, tb.Ma - 1);
    for (int x = 0; x <= nx0; ++x)
        for (int z = 0; z <= nz0; ++z) r.q[x * W1 + z] = ldg(Tb + x * tb.Ma + z);
    double e = ldg(Eb + min(edge + 1, tb.Mt));
    // block1 through the corner gap (Eq. 2, 4, 5)
    float beta = alpha - sc.two_pi_R;
    if (beta > 0.0f) {
        float nu = sc.half_w - r.sgt * s_entry;
        float cbeta = cosf(beta);
        float AP1 = sc.sigma + cosf(alpha) / cbeta * (sc.sigma + nu);
        float qq = fmaxf(AP1 - sc.gt, 0.0f);
        int m = f2i_rd(qq / sc.pt);
        float f = qq - m * sc.pt;
        float u1 = f < sc.wt ? (sc.wt - f) / sc.wt : 0.0f;
        int iu1 = max(min(f2i_rd(u1 * tb.Pt), tb.Pt - 1), 0);
        float run = (sc.sigma + nu) * sc.sin_two_pi_R / cbeta;
        float z1 = z_entry + r.sga * run * tanf(theta);
        float zl = z1 - (sc.z0 - 0.5f * sc.wa);
        int k1 = f2i_rd(zl / sc.pa);
        float fa = zl - k1 * sc.pa;
        float v1;
        if (fa <= sc.wa) {
            v1 = r.sga > 0 ? fa / sc.wa : (sc.wa - fa) / sc.wa;
        } else {
            if (r.sga > 0) k1 += 1;
            v1 = 0.0f;
        }
        int iv1 = max(min(f2i_rd(v1 * tb.Pa), tb.Pa - 1), 0);
        int kt1 = angle_node(beta, tb.inv_dt, tb.Kt);
        int64_t ent1 = table_entry(tb, kt1, ka, iu1, iv1);
        const float *T1 = T + ent1 * MM;
        const double *E1 = eta + ent1 * (tb.Mt + 1);
        e += ldg(E1 + min(m + 1 + sc.Nb, tb.Mt)) - ldg(E1 + min(m + 1, tb.Mt));
        int dzq0 = r.sga * (k1 - ring);
        for (int j = 0; edge + 1 + j <= Wt && j < sc.Nb; ++j) {
            int x = m + 1 + j;
            if (x >= tb.Mt) break;
            for (int z = 0; z < tb.Ma; ++z) {
                int dzq = dzq0 + z;
                if (dzq < 0 || dzq > Wa) continue;
                r.q[(edge + 1 + j) * W1 + dzq] += ldg(T1 + x * tb.Ma + z);
            }
        }
    }
    r.eta = e;
}

}  // namespace psf
