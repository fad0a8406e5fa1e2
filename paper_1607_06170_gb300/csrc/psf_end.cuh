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

namespace psf {

// Direction components of a sub-LOR at one end (normal vn and tangential vt
// against the block's trig cb/sb), with explicit rounding so every caller
// gets the same bits (the travel pattern decided from them must agree
// between the kernel's pattern pre-pass and its main pass).
__device__ __forceinline__ void end_dir(float dx, float dy, float cb, float sb, float &vn,
                                        float &vt) {
    vn = __fadd_rn(__fmul_rn(dx, cb), __fmul_rn(dy, sb));
    vt = __fsub_rn(__fmul_rn(dy, cb), __fmul_rn(dx, sb));
}

// Per-kernel constants of the gap path (reciprocals replace divisions) and
// the node lookup by tangents: the nearest node of an angle a in [0, pi/2)
// is the number of node boundaries (j + 1/2) * step (j = 0 .. K-2) at or
// below a, and a >= b  <=>  opposite >= adjacent * tan(b) for a positive
// adjacent side, so the lookups need no exact arctangent (an approximate one
// only picks where the count starts).  tanB holds the alpha boundaries of the
// block1 angle beta = alpha - 2 pi/R.
struct GapConst {
    float c2, s2, t2;     // cos, sin, tan of the angle between neighbouring block normals
    float ipt, ipa, iwt, iwa;
    float zbase;          // axial origin of the ring lattice (lower edge of ring 0)
    const float *tanT, *tanB, *tanA;  // [Kt - 1], [Kt - 1], [Ka - 1] (shared memory)
};

// Tangent tables in shared memory (2 * Kt + Ka floats); call with every
// thread of the CTA, then synchronise.
__device__ __forceinline__ GapConst make_gapconst(const Scan &sc, const Tab &tb, float *tabs) {
    GapConst k;
    k.c2 = cosf(sc.two_pi_R);
    k.s2 = sc.sin_two_pi_R;
    k.t2 = (float)tan((double)sc.two_pi_R);
    k.ipt = 1.0f / sc.pt;
    k.ipa = 1.0f / sc.pa;
    k.iwt = 1.0f / sc.wt;
    k.iwa = 1.0f / sc.wa;
    k.zbase = sc.z0 - 0.5f * sc.wa;
    float *tT = tabs, *tB = tabs + tb.Kt, *tA = tabs + 2 * tb.Kt;
    const double st = (double)tb.dt, sa = (double)tb.da, g = (double)sc.two_pi_R;
    const double half_pi = 1.5707963267948966;
    for (int j = threadIdx.x; j < 2 * tb.Kt + tb.Ka; j += blockDim.x) {
        double b;
        float* dst;
        if (j < tb.Kt) { b = (j + 0.5) * st; dst = tT + j; }
        else if (j < 2 * tb.Kt) { b = (j - tb.Kt + 0.5) * st + g; dst = tB + (j - tb.Kt); }
        else { b = (j - 2 * tb.Kt + 0.5) * sa; dst = tA + (j - 2 * tb.Kt); }
        *dst = b < half_pi ? (float)tan(b) : CUDART_INF_F;
    }
    k.tanT = tT;
    k.tanB = tB;
    k.tanA = tA;
    return k;
}

// Number of entries j < K - 1 of the ascending table with adj * tab[j] <= opp
// (adj > 0), found by stepping from a starting guess k0: the predicate is
// monotone in j, so the count is the k at which it turns from true to false,
// whatever k0 was (a good guess only saves steps).
__device__ __forceinline__ int node_by_tan(const float *tab, int K, float opp, float adj,
                                           int k0) {
    int k = k0 < 0 ? 0 : (k0 > K - 1 ? K - 1 : k0);
    while (k < K - 1 && adj * tab[k] <= opp) ++k;
    while (k > 0 && adj * tab[k - 1] > opp) --k;
    return k;
}

// Arctangent of y / x for x > 0, y >= 0, good to about 1.5e-3 rad: the
// quadratic approximation on [0, 1] of Rajan, Wang, Inkol and Joyal
// ("Efficient approximations for the arctangent function", IEEE Signal
// Processing Magazine, 2006), reflected about pi/4 above it.  It only seeds
// node_by_tan, so its error costs steps, never a different node.
__device__ __forceinline__ float atan_seed(float y, float x) {
    const bool above = y > x;
    const float r = above ? __fdividef(x, y) : __fdividef(y, x);
    const float a = r * (0.78539816f - (r - 1.0f) * (0.2447f + 0.0663f * r));
    return above ? 1.57079633f - a : a;
}

// The response of end_response() with a compile-time window: the quadrant
// array stays in registers (every index is static after unrolling), the
// trigonometry of the gap path comes from the direction components
// (cos a = vn/h, tan theta = |dz|/h, cos(a - 2pi/R) by the angle-difference
// formula), the nearest nodes come from tangent tables and divisions by
// constants are products with reciprocals.  The response is the same
// quantity: Sec. 2.1.1 table lookup for block0 and Sec. 2.1.2 Eq. 2, 4, 5
// for block1.
template <int WT, int WA>
struct QResp {
    float q[(WT + 1) * (WA + 1)];
    double eta;
};

template <int WT, int WA>
__device__ __forceinline__ void end_resp_q(const Scan &sc, const Tab &tb, const GapConst &k,
                                           const float *__restrict__ T,
                                           const double *__restrict__ eta, int i, int ring,
                                           int p, int q, float s_entry, float z_entry, float vn,
                                           float vt, float dz, QResp<WT, WA> &r) {
    constexpr int W1 = WA + 1;
    const int sgt = vt >= 0.0f ? 1 : -1;
    const int sga = dz >= 0.0f ? 1 : -1;
#pragma unroll
    for (int j = 0; j < (WT + 1) * W1; ++j) r.q[j] = 0.0f;
    const float avt = fabsf(vt), adz = fabsf(dz);
    const float h2 = vn * vn + vt * vt;
    const float ih = rsqrtf(h2);
    const float h = h2 * ih;
    const int iu = sgt > 0 ? p : tb.Pt - 1 - p;
    const int iv = sga > 0 ? q : tb.Pa - 1 - q;
    // nearest nodes: count of node boundaries (j + 1/2) * step at or below
    // the angle, seeded from the approximate angle
    const float alpha = atan_seed(avt, vn);
    const int kt = node_by_tan(k.tanT, tb.Kt, avt, vn, f2i_rd(fmaf(alpha, tb.inv_dt, 0.5f)));
    const int ka = node_by_tan(k.tanA, tb.Ka, adz, h,
                               f2i_rd(fmaf(atan_seed(adz, h), tb.inv_da, 0.5f)));
    const int MM = tb.Mt * tb.Ma;
    // table offsets fit 32 bits (the descriptor holds at most 2^28 values)
    const int ent = ((kt * tb.Ka + ka) * tb.Pt + iu) * tb.Pa + iv;
    const float *Tb = T + ent * MM;
    const int edge = sgt > 0 ? sc.Nb - 1 - i : i;  // crystals of block0 beyond the entry one
    const int nx0 = min(edge, tb.Mt - 1);
    if (WA % 2 == 1 && WA < tb.Ma && (tb.Ma & 1) == 0) {
        // rows of an even length start 8-byte aligned: load z pairs
#pragma unroll
        for (int x = 0; x <= WT; ++x)
            if (x <= nx0) {
#pragma unroll
                for (int z = 0; z <= WA; z += 2) {
                    const float2 v = __ldg(reinterpret_cast<const float2 *>(Tb + x * tb.Ma + z));
                    r.q[x * W1 + z] = v.x;
                    r.q[x * W1 + z + 1] = v.y;
                }
            }
    } else {
        const int nz0 = tb.Ma - 1;
#pragma unroll
        for (int x = 0; x <= WT; ++x)
#pragma unroll
            for (int z = 0; z <= WA; ++z)
                if (x <= nx0 && z <= nz0) r.q[x * W1 + z] = ldg(Tb + x * tb.Ma + z);
    }
    double e = ldg(eta + ent * (tb.Mt + 1) + min(edge + 1, tb.Mt));
    if (avt > vn * k.t2) {  // beta = alpha - 2 pi/R > 0: block1 through the corner gap
        const float nu = sc.half_w - sgt * s_entry;
        const float ca = vn * ih, sa = avt * ih;
        const float icb = 1.0f / (ca * k.c2 + sa * k.s2);
        const float AP1 = sc.sigma + ca * icb * (sc.sigma + nu);
        const float qq = fmaxf(AP1 - sc.gt, 0.0f);
        const int m = f2i_rd(qq * k.ipt);
        const float f = qq - m * sc.pt;
        const float u1 = f < sc.wt ? (sc.wt - f) * k.iwt : 0.0f;
        const int iu1 = max(min(f2i_rd(u1 * tb.Pt), tb.Pt - 1), 0);
        const float run = (sc.sigma + nu) * sc.sin_two_pi_R * icb;
        const float z1 = z_entry + sga * run * (adz * ih);
        const float zl = z1 - k.zbase;
        int k1 = f2i_rd(zl * k.ipa);
        const float fa = zl - k1 * sc.pa;
        float v1;
        if (fa <= sc.wa) {
            v1 = sga > 0 ? fa * k.iwa : (sc.wa - fa) * k.iwa;
        } else {
            if (sga > 0) k1 += 1;
            v1 = 0.0f;
        }
        const int iv1 = max(min(f2i_rd(v1 * tb.Pa), tb.Pa - 1), 0);
        const int kt1 = node_by_tan(k.tanB, tb.Kt, avt, vn,
                                    f2i_rd(fmaf(alpha - sc.two_pi_R, tb.inv_dt, 0.5f)));
        const int ent1 = ((kt1 * tb.Ka + ka) * tb.Pt + iu1) * tb.Pa + iv1;
        const float *T1 = T + ent1 * MM;
        const double *E1 = eta + ent1 * (tb.Mt + 1);
        e += ldg(E1 + min(m + 1 + sc.Nb, tb.Mt)) - ldg(E1 + min(m + 1, tb.Mt));
        const int dzq0 = sga * (k1 - ring);
        // block1 crystals enter the window only from an entry crystal within
        // WT of the block edge (the same for every sub-LOR of the LOR)
        if (edge < WT) {
#pragma unroll
            for (int X = 0; X <= WT; ++X) {
                const int j = X - edge - 1, x = m + 1 + j;  // block1 crystal j, table column x
                if (j < 0 || j >= sc.Nb || x >= tb.Mt) continue;
#pragma unroll
                for (int Z = 0; Z <= WA; ++Z) {
                    const int z = Z - dzq0;
                    if (z >= 0 && z < tb.Ma) r.q[X * W1 + Z] += ldg(T1 + x * tb.Ma + z);
                }
            }
        }
    }
    r.eta = e;
}

}  // namespace psf
