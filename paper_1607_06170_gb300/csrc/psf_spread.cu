// K3: homogenization spread of each LOR (Sec. 2.2 Eq. 10, Sec. 2.3 Eq. 11-12)
// with the neighbouring-block path of Sec. 2.1.2 (Eq. 2, 4, 5).
//
// One CTA per LOR.  The sub-position centres of both crystal faces are staged
// in shared memory; each thread takes one sub-LOR (pair of sub-positions) at a
// time and evaluates the two single-photon responses restricted to the window
// quadrant the photon travels into (the response is one-sided).  Sub-LORs are
// grouped by their pair of travel directions, and each group's contribution is
// a small dense product sum_s r1_s (x) r2_s accumulated by the threads that own
// the outputs, chunk by chunk (FP32, deterministic order).  The per-LOR
// normalisation totals are FP64 block reductions.
#include "psf_common.cuh"
#include "psf_end.cuh"
#include "psf_lorset.cuh"

namespace psf {

constexpr int SP_THREADS = 256;
constexpr int SP_PATS = 16;  // travel-sign patterns of the two ends
struct SpreadSmem {
    float *R1, *R2;        // [SP_THREADS][Q]
    float *accp;           // [SP_PATS][Q*Q]
    float *wwin;           // [E*E]
    float *pts;            // end points: [2][Pt*Pa][4] = (x, y, z, s_entry)
    int *pat;              // [SP_THREADS]
    int *order;            // [SP_THREADS]
    int *cnt;              // [SP_PATS + 1] starts
    int *wcnt;             // [8 warps][SP_PATS]
    double *red;           // [2 * 8]
};

__global__ void __launch_bounds__(SP_THREADS) spread_kernel(
    Scan sc, Tab tb, const float *__restrict__ T, const double *__restrict__ eta,
    const int32_t *__restrict__ lors, int64_t n_lors, int Wt, int Wa, int norm,
    float *__restrict__ out, const int32_t *__restrict__ sym) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Q = (Wt + 1) * (Wa + 1);
    const int E = (2 * Wt + 1) * (2 * Wa + 1);
    const int NP = tb.Pt * tb.Pa;
    const int nsub = NP * NP;
    SpreadSmem s;
    {
        unsigned char *p = smraw;
        s.red = (double *)p; p += sizeof(double) * 16;
        s.R1 = (float *)p; p += sizeof(float) * SP_THREADS * (Q + 1);
        s.R2 = (float *)p; p += sizeof(float) * SP_THREADS * (Q + 1);
        s.accp = (float *)p; p += sizeof(float) * SP_PATS * Q * Q;
        s.wwin = (float *)p; p += sizeof(float) * E * E;
        s.pts = (float *)p; p += sizeof(float) * 2 * NP * 4;
        s.pat = (int *)p; p += sizeof(int) * SP_THREADS;
        s.order = (int *)p; p += sizeof(int) * SP_THREADS;
        s.cnt = (int *)p; p += sizeof(int) * (SP_PATS + 1);
        s.wcnt = (int *)p;
    }
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int64_t lor = blockIdx.x; lor < n_lors; lor += gridDim.x) {
        const int id1 = lors[2 * lor], id2 = lors[2 * lor + 1];
        const int ring1 = id1 / sc.Nt, c1 = id1 - ring1 * sc.Nt;
        const int ring2 = id2 / sc.Nt, c2 = id2 - ring2 * sc.Nt;
        if (sym && sym[lor] >= 0) continue;  // an image of another class under the mirrors
        const int b1 = c1 / sc.Nb, i1 = c1 - b1 * sc.Nb;
        const int b2 = c2 / sc.Nb, i2 = c2 - b2 * sc.Nb;
        float *o = out + lor * (int64_t)E * E;
        const int nc = sc.Nt * sc.NR;
        // same block: the chord runs along a block face and enters neither
        // crystal; invalid crystal ids also get no spread
        if (b1 == b2 || id1 < 0 || id2 < 0 || id1 >= nc || id2 >= nc) {
            for (int k = t; k < E * E; k += SP_THREADS) o[k] = 0.0f;
            continue;
        }
        float sb1, cb1, sb2, cb2;
        sincospif(2.0f * b1 / sc.R, &sb1, &cb1);
        sincospif(2.0f * b2 / sc.R, &sb2, &cb2);
        // stage the sub-position centres of both faces
        for (int k = t; k < 2 * NP; k += SP_THREADS) {
            int end = k / NP, sp = k - end * NP;
            int p = sp / tb.Pa, q = sp - p * tb.Pa;
            int i = end ? i2 : i1, ring = end ? ring2 : ring1;
            float cb = end ? cb2 : cb1, sb = end ? sb2 : sb1;
            float se = (i - 0.5f * (sc.Nb - 1)) * sc.pt + ((p + 0.5f) / tb.Pt - 0.5f) * sc.wt;
            float ze = sc.z0 + ring * sc.pa + ((q + 0.5f) / tb.Pa - 0.5f) * sc.wa;
            float *P = s.pts + k * 4;
            P[0] = sc.radius * cb - se * sb;
            P[1] = sc.radius * sb + se * cb;
            P[2] = ze;
            P[3] = se;
        }
        for (int k = t; k < SP_PATS * Q * Q; k += SP_THREADS) s.accp[k] = 0.0f;
        double sfull = 0.0, swin = 0.0;
        __syncthreads();
        for (int base = 0; base < nsub; base += SP_THREADS) {
            int sidx = base + t;
            int pt_ = SP_PATS;  // empty slot
            if (sidx < nsub) {
                int s1 = sidx / NP, s2 = sidx - s1 * NP;
                const float *P1 = s.pts + s1 * 4;
                const float *P2 = s.pts + (NP + s2) * 4;
                float dx = P1[0] - P2[0], dy = P1[1] - P2[1], dz = P1[2] - P2[2];
                EndResp r1, r2;
                end_response(sc, tb, T, eta, i1, ring1, cb1, sb1, s1 / tb.Pa, s1 % tb.Pa, P1[3],
                             P1[2], dx, dy, dz, Wt, Wa, r1);
                end_response(sc, tb, T, eta, i2, ring2, cb2, sb2, s2 / tb.Pa, s2 % tb.Pa, P2[3],
                             P2[2], -dx, -dy, -dz, Wt, Wa, r2);
                if (r1.valid && r2.valid) {
                    float w1 = 0.0f, w2 = 0.0f;
                    for (int k = 0; k < Q; ++k) {
                        s.R1[t * (Q + 1) + k] = r1.q[k];  // odd stride: conflict-free
                        s.R2[t * (Q + 1) + k] = r2.q[k];
                        w1 += r1.q[k];
                        w2 += r2.q[k];
                    }
                    sfull += r1.eta * r2.eta;
                    swin += (double)w1 * (double)w2;
                    pt_ = ((r1.sgt > 0) << 3) | ((r1.sga > 0) << 2) | ((r2.sgt > 0) << 1) |
                          (r2.sga > 0);
                }
            }
            s.pat[t] = pt_;
            // stable counting sort of this chunk by pattern (warp ballots)
            for (int P = 0; P < SP_PATS; ++P) {
                unsigned m = __ballot_sync(0xffffffffu, pt_ == P);
                if (lane == 0) s.wcnt[warp * SP_PATS + P] = __popc(m);
            }
            __syncthreads();
            if (t == 0) {
                int acc = 0;
                for (int P = 0; P < SP_PATS; ++P) {
                    s.cnt[P] = acc;
                    for (int w = 0; w < SP_THREADS / 32; ++w) {
                        int c = s.wcnt[w * SP_PATS + P];
                        s.wcnt[w * SP_PATS + P] = acc;
                        acc += c;
                    }
                }
                s.cnt[SP_PATS] = acc;
            }
            __syncthreads();
            // rank within (warp, pattern)
            for (int P = 0; P < SP_PATS; ++P) {
                unsigned m = __ballot_sync(0xffffffffu, pt_ == P);
                if (pt_ == P) {
                    int r = __popc(m & ((1u << lane) - 1u));
                    s.order[s.wcnt[warp * SP_PATS + P] + r] = t;
                }
            }
            __syncthreads();
            if (t < Q * Q) {
                const int e1 = t / Q, e2 = t - e1 * Q;
                for (int P = 0; P < SP_PATS; ++P) {
                    int k0 = s.cnt[P], k1 = s.cnt[P + 1];
                    if (k1 == k0) continue;
                    float acc = 0.0f;
                    for (int k = k0; k < k1; ++k) {
                        int sl = s.order[k];
                        acc = fmaf(s.R1[sl * (Q + 1) + e1], s.R2[sl * (Q + 1) + e2], acc);
                    }
                    s.accp[P * Q * Q + t] += acc;
                }
            }
            __syncthreads();
        }
        // FP64 totals over the CTA
        sfull = warp_sum_d(sfull);
        swin = warp_sum_d(swin);
        if (lane == 0) {
            s.red[warp] = sfull;
            s.red[8 + warp] = swin;
        }
        for (int k = t; k < E * E; k += SP_THREADS) s.wwin[k] = 0.0f;
        __syncthreads();
        if (t == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < SP_THREADS / 32; ++w) {
                a += s.red[w];
                b += s.red[8 + w];
            }
            s.red[0] = a;
            s.red[8] = b;
        }
        // fold the pattern-local blocks into the window
        const int W2a = 2 * Wa + 1;
        for (int P = 0; P < SP_PATS; ++P) {
            if (t < Q * Q) {
                float v = s.accp[P * Q * Q + t];
                if (v != 0.0f) {
                    int sgt1 = (P >> 3) & 1 ? 1 : -1, sga1 = (P >> 2) & 1 ? 1 : -1;
                    int sgt2 = (P >> 1) & 1 ? 1 : -1, sga2 = P & 1 ? 1 : -1;
                    int e1 = t / Q, e2 = t - e1 * Q;
                    int x1 = e1 / (Wa + 1), z1 = e1 - x1 * (Wa + 1);
                    int x2 = e2 / (Wa + 1), z2 = e2 - x2 * (Wa + 1);
                    int w1 = (sgt1 * x1 + Wt) * W2a + (sga1 * z1 + Wa);
                    int w2 = (sgt2 * x2 + Wt) * W2a + (sga2 * z2 + Wa);
                    s.wwin[w1 * E + w2] += v;
                }
            }
            __syncthreads();
        }
        // wwin holds sums over sub-LORs; sw is its total, sf the untruncated one
        double sf = s.red[0], sw = s.red[8];
        double scale = 1.0 / nsub;                                     // NONE: mean
        if (norm == PSF_NORM_EFF && sw > 0.0) scale = sf / (sw * nsub);  // total = mean eta1 eta2
        if (norm == PSF_NORM_UNIT && sw > 0.0) scale = 1.0 / sw;         // total = 1
        float fs = (float)scale;
        for (int k = t; k < E * E; k += SP_THREADS) o[k] = s.wwin[k] * fs;
        __syncthreads();
    }
}

static size_t spread_smem(const Tab &tb, int Wt, int Wa) {
    int Q = (Wt + 1) * (Wa + 1), E = (2 * Wt + 1) * (2 * Wa + 1);
    int NP = tb.Pt * tb.Pa;
    size_t b = sizeof(double) * 16;
    b += sizeof(float) * 2 * SP_THREADS * (Q + 1);
    b += sizeof(float) * SP_PATS * Q * Q;
    b += sizeof(float) * E * E;
    b += sizeof(float) * 2 * NP * 4;
    b += sizeof(int) * (2 * SP_THREADS + SP_PATS + 1 + 8 * SP_PATS);
    return b;
}


// K3 with a compile-time window (the common windows).  A warp evaluates 32
// sub-LORs at a time, one per lane, into warp-private rows of shared memory,
// then accumulates their outer products r1 (x) r2: each half-warp takes every
// other staged sub-LOR, its 16 lanes owning fixed RB x CB blocks of the Q x Q
// quadrant-local product (two shared-memory reads per 16 FMA).  Sub-LORs with
// different travel patterns land in different quadrants of the window, so
// each pattern present in the LOR gets its own register accumulator ("slot");
// a pre-pass finds the patterns present and a LOR with more than SQ_SLOTS
// patterns is done in several passes, each evaluating the responses of only
// its patterns' sub-LORs.  The per-warp accumulators are summed in a fixed
// order at the end of each pass (FP32, deterministic), folded into the window,
// and normalised with FP64 totals.  One slot (a pass per pattern) leaves the
// registers for three CTAs per SM, which hides more latency than the extra
// passes over the sub-LOR directions cost (22.1 ms against 24.2 ms with four
// slots at two CTAs per SM, 3D ring classes).
constexpr int SQ_SLOTS = 1;
constexpr int SQ_WARPS = SP_THREADS / 32;
constexpr int SQ_TA_LOG = 3, SQ_TB_LOG = 2;  // sub-LOR tile of a warp: 8 x 4
constexpr int SQ_TA = 1 << SQ_TA_LOG, SQ_TB = 1 << SQ_TB_LOG;
static_assert(SQ_TA * SQ_TB == 32, "one sub-LOR per lane");

template <int WT, int WA>
struct SqShape {
    static constexpr int Q = (WT + 1) * (WA + 1);
    static constexpr int E = (2 * WT + 1) * (2 * WA + 1);
    // each half-warp covers the Q x Q product with its 16 lanes, lane (rb, cb)
    // owning rows rb*RB.. and columns cb*CB.. of it; the two halves take
    // alternate staged sub-LORs and are summed at the end of a pass
    static constexpr int RB = (Q + 3) / 4;
    static constexpr int CB = (Q + 3) / 4;
    // row stride of the staged responses: covers every lane's reads, 16-byte
    // rows, and an odd number of 16-byte units so 8 lanes storing 16 bytes
    // each hit distinct banks; then rows r and r + 4 (the two halves' rows at
    // one step) lie 16 banks apart
    static constexpr int QR = 4 * RB;
    static constexpr int QS = ((QR + 3) / 4) % 2 == 0 ? ((QR + 3) / 4) * 4 + 4 : ((QR + 3) / 4) * 4;
    static_assert((4 * QS) % 32 == 16 || QR <= 8, "halves' rows 16 banks apart");
};

// One staged sub-LOR's operands of a lane: RB entries of r1, CB of r2.
template <int N>
__device__ __forceinline__ void load_n(const float *p, float (&v)[N]) {
    if constexpr (N == 4) {
        const float4 w = *reinterpret_cast<const float4 *>(p);
        v[0] = w.x;
        v[1] = w.y;
        v[2] = w.z;
        v[3] = w.w;
    } else if constexpr (N == 2) {
        const float2 w = *reinterpret_cast<const float2 *>(p);
        v[0] = w.x;
        v[1] = w.y;
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = p[i];
    }
}

template <int RB, int CB>
__device__ __forceinline__ void load_ab(const float *ra, const float *rbp, float (&a)[RB],
                                        float (&b)[CB]) {
    load_n<RB>(ra, a);
    load_n<CB>(rbp, b);
}

// Staged row of a half-warp at step k (0..15): the halves take rows r and
// r + 4 of each group of eight.
__device__ __forceinline__ int half_row(int k, int h) { return ((k >> 2) << 3) + (k & 3) + (h << 2); }

// All 32 staged sub-LORs of a warp into one accumulator (same slot): each
// half-warp takes 16 of them.
template <int RB, int CB, int QS>
__device__ __forceinline__ void acc_all32(float (&acc)[RB][CB], const float *ra,
                                          const float *rbp, int h) {
#pragma unroll 8
    for (int k = 0; k < 16; ++k) {
        float a[RB], b[CB];
        const int row = half_row(k, h);
        load_ab<RB, CB>(ra + row * QS, rbp + row * QS, a, b);
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int j = 0; j < CB; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
}

// A response into its staging row (16-byte aligned when Q is a multiple of 4).
template <int Q>
__device__ __forceinline__ void stage_row(float *dst, const float (&q)[Q]) {
    if constexpr (Q % 4 == 0) {
#pragma unroll
        for (int k = 0; k < Q; k += 4)
            *reinterpret_cast<float4 *>(dst + k) = make_float4(q[k], q[k + 1], q[k + 2], q[k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) dst[k] = q[k];
    }
}

template <int WT, int WA>
static size_t spread_q_smem(const Tab &tb) {
    using S = SqShape<WT, WA>;
    const int NP = tb.Pt * tb.Pa;
    size_t b = sizeof(double) * 2 * SQ_WARPS;                       // FP64 partial totals
    b += sizeof(int) * 20;                                           // pattern mask, slots
    b += sizeof(float) * SQ_WARPS * 2 * 32 * S::QS;                  // staged responses
    b += sizeof(float) * S::E * S::E;                                // window
    b += sizeof(float) * 2 * NP * 4;                                 // sub-position centres
    b += sizeof(float) * (2 * tb.Kt + tb.Ka);                        // node tangents
    return b + 64;
}

template <int WT, int WA>
__global__ void __launch_bounds__(SP_THREADS, 3) spread_q_kernel(
    Scan sc, Tab tb, const float *__restrict__ T, const double *__restrict__ eta,
    const int32_t *__restrict__ lors, int64_t n_lors, int norm, float *__restrict__ out,
    const int32_t *__restrict__ sym) {
    using S = SqShape<WT, WA>;
    constexpr int Q = S::Q, E = S::E, RB = S::RB, CB = S::CB, QS = S::QS;
    constexpr int W2a = 2 * WA + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int NP = tb.Pt * tb.Pa;
    const int nsub = NP * NP;
    double *red = reinterpret_cast<double *>(smraw);                 // [2][SQ_WARPS]
    int *ipat = reinterpret_cast<int *>(red + 2 * SQ_WARPS);        // [0] mask, [1] npat, [4..19] slot pattern
    float *Rw = reinterpret_cast<float *>(ipat + 20);               // [warps][2][32][QS]
    float *pts = Rw + SQ_WARPS * 2 * 32 * QS;                       // [2][NP][4]
    float *wwin = pts + 2 * NP * 4;                                 // [E*E]
    float *part = Rw;  // [warps][SQ_SLOTS][Q*Q], reuses the staging rows at the end of a LOR
    static_assert(SQ_WARPS * SQ_SLOTS * Q * Q <= SQ_WARPS * 2 * 32 * QS, "part fits the staging rows");
    static_assert(QS % 4 == 0 && (2 * 8 * SQ_WARPS + 4 * 20) % 16 == 0,
                  "staging rows and sub-position centres start 16-byte aligned");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float *R1w = Rw + warp * 2 * 32 * QS, *R2w = R1w + 32 * QS;
    const int hw = lane >> 4, rb = (lane >> 2) & 3, cb = lane & 3;
    const GapConst gk = make_gapconst(sc, tb, wwin + E * E);  // visible after the first barrier
    for (int k = t; k < SQ_WARPS * 2 * 32 * QS; k += SP_THREADS) Rw[k] = 0.0f;
    for (int64_t lor = blockIdx.x; lor < n_lors; lor += gridDim.x) {
        const int id1 = lors[2 * lor], id2 = lors[2 * lor + 1];
        const int ring1 = id1 / sc.Nt, c1 = id1 - ring1 * sc.Nt;
        const int ring2 = id2 / sc.Nt, c2 = id2 - ring2 * sc.Nt;
        if (sym && sym[lor] >= 0) continue;  // an image of another class under the mirrors
        const int b1 = c1 / sc.Nb, i1 = c1 - b1 * sc.Nb;
        const int b2 = c2 / sc.Nb, i2 = c2 - b2 * sc.Nb;
        float *o = out + lor * (int64_t)E * E;
        const int nc = sc.Nt * sc.NR;
        __syncthreads();  // previous LOR's readers of pts / wwin / part are done
        if (b1 == b2 || id1 < 0 || id2 < 0 || id1 >= nc || id2 >= nc) {
            for (int k = t; k < E * E; k += SP_THREADS) o[k] = 0.0f;
            continue;
        }
        float sb1, cb1, sb2, cb2;
        sincospif(2.0f * b1 / sc.R, &sb1, &cb1);
        sincospif(2.0f * b2 / sc.R, &sb2, &cb2);
        for (int k = t; k < 2 * NP; k += SP_THREADS) {
            const int end = k / NP, sp = k - end * NP;
            const int p = sp / tb.Pa, q = sp - p * tb.Pa;
            const int i = end ? i2 : i1, ring = end ? ring2 : ring1;
            const float cbk = end ? cb2 : cb1, sbk = end ? sb2 : sb1;
            const float se = (i - 0.5f * (sc.Nb - 1)) * sc.pt + ((p + 0.5f) / tb.Pt - 0.5f) * sc.wt;
            const float ze = sc.z0 + ring * sc.pa + ((q + 0.5f) / tb.Pa - 0.5f) * sc.wa;
            reinterpret_cast<float4 *>(pts)[k] =
                make_float4(sc.radius * cbk - se * sbk, sc.radius * sbk + se * cbk, ze, se);
        }
        for (int k = t; k < E * E; k += SP_THREADS) wwin[k] = 0.0f;
        if (t == 0) ipat[0] = 0;
        __syncthreads();
        // pre-pass: the travel patterns present among the valid sub-LORs
        unsigned mine = 0;
        for (int s = t; s < nsub; s += SP_THREADS) {
            const int s1 = s / NP, s2 = s - s1 * NP;
            const float4 P1 = reinterpret_cast<const float4 *>(pts)[s1];
            const float4 P2 = reinterpret_cast<const float4 *>(pts)[NP + s2];
            const float dx = P1.x - P2.x, dy = P1.y - P2.y, dz = P1.z - P2.z;
            float vn1, vt1, vn2, vt2;
            end_dir(dx, dy, cb1, sb1, vn1, vt1);
            end_dir(-dx, -dy, cb2, sb2, vn2, vt2);
            if (vn1 > 0.0f && vn2 > 0.0f)
                mine |= 1u << (((vt1 >= 0.0f) << 3) | ((dz >= 0.0f) << 2) | ((vt2 >= 0.0f) << 1) |
                               (-dz >= 0.0f));
        }
        mine = __reduce_or_sync(0xffffffffu, mine);
        if (lane == 0 && mine) atomicOr(ipat, (int)mine);
        __syncthreads();
        const unsigned present = (unsigned)ipat[0];
        // a warp takes the sub-LORs of a tile of SQ_TA end-1 by SQ_TB end-2
        // sub-positions: its table reads then hit about SQ_TA + SQ_TB rows
        // instead of 33 for a run of 32 end-2 positions (17.3 ms against
        // 22.1 ms on the 3D ring classes; 4 x 8 18.3, 16 x 2 18.1, 32 x 1 21.3)
        const int ntb = (NP + SQ_TB - 1) >> SQ_TB_LOG;
        const int ntile = ((NP + SQ_TA - 1) >> SQ_TA_LOG) * ntb;
        const int npat = __popc(present);
        double sfull = 0.0;
        for (int pass = 0; pass * SQ_SLOTS < npat; ++pass) {
            float acc[SQ_SLOTS][RB][CB];
#pragma unroll
            for (int a = 0; a < SQ_SLOTS; ++a)
#pragma unroll
                for (int i = 0; i < RB; ++i)
#pragma unroll
                    for (int j = 0; j < CB; ++j) acc[a][i][j] = 0.0f;
            for (int tile = warp; tile < ntile; tile += SQ_WARPS) {
                const int ta = tile / ntb;
                const int s1 = (ta << SQ_TA_LOG) + (lane >> SQ_TB_LOG);
                const int s2 = ((tile - ta * ntb) << SQ_TB_LOG) + (lane & (SQ_TB - 1));
                int slot = -1;
                if (s1 < NP && s2 < NP) {
                    const float4 P1 = reinterpret_cast<const float4 *>(pts)[s1];
                    const float4 P2 = reinterpret_cast<const float4 *>(pts)[NP + s2];
                    const float dx = P1.x - P2.x, dy = P1.y - P2.y, dz = P1.z - P2.z;
                    float vn1, vt1, vn2, vt2;
                    end_dir(dx, dy, cb1, sb1, vn1, vt1);
                    end_dir(-dx, -dy, cb2, sb2, vn2, vt2);
                    if (vn1 > 0.0f && vn2 > 0.0f) {
                        const int P = ((vt1 >= 0.0f) << 3) | ((dz >= 0.0f) << 2) |
                                      ((vt2 >= 0.0f) << 1) | (-dz >= 0.0f);
                        // slot = rank of the pattern among those present
                        const int sl = __popc(present & ((1u << P) - 1u)) - pass * SQ_SLOTS;
                        if (sl >= 0 && sl < SQ_SLOTS) {
                            slot = sl;
                            QResp<WT, WA> r;
                            end_resp_q<WT, WA>(sc, tb, gk, T, eta, i1, ring1, s1 / tb.Pa,
                                               s1 % tb.Pa, P1.w, P1.z, vn1, vt1, dz, r);
                            const double e1 = r.eta;
                            stage_row<Q>(R1w + lane * QS, r.q);
                            end_resp_q<WT, WA>(sc, tb, gk, T, eta, i2, ring2, s2 / tb.Pa,
                                               s2 % tb.Pa, P2.w, P2.z, vn2, vt2, -dz, r);
                            stage_row<Q>(R2w + lane * QS, r.q);
                            sfull += e1 * r.eta;
                        }
                    }
                }
                __syncwarp();
                const float *ra = R1w + rb * RB, *rbp = R2w + cb * CB;
                const int s0 = __shfl_sync(0xffffffffu, slot, 0);
                if (__all_sync(0xffffffffu, slot == s0)) {
                    // common case: one travel pattern for the whole warp
#pragma unroll
                    for (int sl = 0; sl < SQ_SLOTS; ++sl)
                        if (s0 == sl) acc_all32<RB, CB, QS>(acc[sl], ra, rbp, hw);
                } else {
#pragma unroll 4
                    for (int k = 0; k < 16; ++k) {
                        const int row = half_row(k, hw);
                        const int sk = __shfl_sync(0xffffffffu, slot, row);
                        if (sk < 0) continue;
                        float a[RB], b[CB];
                        load_ab<RB, CB>(ra + row * QS, rbp + row * QS, a, b);
#pragma unroll
                        for (int sl = 0; sl < SQ_SLOTS; ++sl)
                            if (sk == sl) {
#pragma unroll
                                for (int i = 0; i < RB; ++i)
#pragma unroll
                                    for (int j = 0; j < CB; ++j)
                                        acc[sl][i][j] = fmaf(a[i], b[j], acc[sl][i][j]);
                            }
                    }
                }
                __syncwarp();
            }
            // per-warp accumulators (the two halves summed) -> part, then fold
            // into the window
#pragma unroll
            for (int sl = 0; sl < SQ_SLOTS; ++sl)
#pragma unroll
                for (int i = 0; i < RB; ++i)
#pragma unroll
                    for (int j = 0; j < CB; ++j)
                        acc[sl][i][j] += __shfl_xor_sync(0xffffffffu, acc[sl][i][j], 16);
            __syncthreads();
            if (hw == 0) {
#pragma unroll
                for (int sl = 0; sl < SQ_SLOTS; ++sl)
#pragma unroll
                    for (int i = 0; i < RB; ++i)
#pragma unroll
                        for (int j = 0; j < CB; ++j) {
                            const int e1 = rb * RB + i, e2 = cb * CB + j;
                            if (e1 < Q && e2 < Q)
                                part[(warp * SQ_SLOTS + sl) * Q * Q + e1 * Q + e2] = acc[sl][i][j];
                        }
            }
            __syncthreads();
            const int nsl = min(SQ_SLOTS, npat - pass * SQ_SLOTS);
            // fold slot by slot, in pattern order: within one pattern the
            // quadrant-to-window map is one-to-one, so no two threads meet
            unsigned rest = present;
            for (int c = 0; c < pass * SQ_SLOTS; ++c) rest &= rest - 1u;
            for (int sl = 0; sl < nsl; ++sl) {
                const int P = __ffs(rest) - 1;
                rest &= rest - 1u;
                const int g1 = (P >> 3) & 1 ? 1 : -1, a1 = (P >> 2) & 1 ? 1 : -1;
                const int g2 = (P >> 1) & 1 ? 1 : -1, a2 = P & 1 ? 1 : -1;
                for (int e = t; e < Q * Q; e += SP_THREADS) {
                    const int e1 = e / Q, e2 = e - e1 * Q;
                    const int x1 = e1 / (WA + 1), z1 = e1 - x1 * (WA + 1);
                    const int x2 = e2 / (WA + 1), z2 = e2 - x2 * (WA + 1);
                    const int w1 = (g1 * x1 + WT) * W2a + (a1 * z1 + WA);
                    const int w2 = (g2 * x2 + WT) * W2a + (a2 * z2 + WA);
                    float sum = 0.0f;
#pragma unroll
                    for (int w = 0; w < SQ_WARPS; ++w) sum += part[(w * SQ_SLOTS + sl) * Q * Q + e];
                    wwin[w1 * E + w2] += sum;
                }
                __syncthreads();  // the next slot may meet these entries; part aliases the staging rows
            }
        }
        // FP64 totals: sfull over sub-LORs, sw over the accumulated window
        double swin = 0.0;
        for (int wc = t; wc < E * E; wc += SP_THREADS) swin += (double)wwin[wc];
        sfull = warp_sum_d(sfull);
        swin = warp_sum_d(swin);
        if (lane == 0) {
            red[warp] = sfull;
            red[SQ_WARPS + warp] = swin;
        }
        __syncthreads();
        double sf = 0.0, sw = 0.0;
#pragma unroll
        for (int w = 0; w < SQ_WARPS; ++w) {
            sf += red[w];
            sw += red[SQ_WARPS + w];
        }
        double scale = 1.0 / nsub;                                       // NONE: mean
        if (norm == PSF_NORM_EFF && sw > 0.0) scale = sf / (sw * nsub);    // total = mean eta1 eta2
        if (norm == PSF_NORM_UNIT && sw > 0.0) scale = 1.0 / sw;           // total = 1
        const float fs = (float)scale;
        for (int k = t; k < E * E; k += SP_THREADS) o[k] = wwin[k] * fs;
    }
}

template <int WT, int WA>
static int launch_spread_q(const Scan &sc, const Tab &tb, const float *T, const double *eta,
                           const int32_t *lors, int64_t n_lors, int norm, float *out,
                           const int32_t *sym, cudaStream_t st) {
    const size_t shm = spread_q_smem<WT, WA>(tb);
    if (shm > 200 * 1024) return PSF_EINVAL;
    PSF_TRY(cudaFuncSetAttribute(spread_q_kernel<WT, WA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    int dev = 0, sms = 148, per_sm = 0;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PSF_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spread_q_kernel<WT, WA>,
                                                          SP_THREADS, shm));
    if (per_sm < 1) per_sm = 1;
    const int64_t cap = (int64_t)sms * per_sm;
    const int64_t grid = n_lors < cap ? n_lors : cap;
    {
        PSF_TIMED("spread_q_kernel", st);
        spread_q_kernel<WT, WA><<<(int)grid, SP_THREADS, shm, st>>>(sc, tb, T, eta, lors, n_lors,
                                                                    norm, out, sym);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

}  // namespace psf

using namespace psf;


namespace psf {

// Symmetries of the spread classes of a structured set.  A: reflection
// through the axial centre plane (ring r -> NR-1-r for both crystals; the ring
// lattice has one pitch): ring difference d -> -d, every axial window offset
// negated.  T: reflection through block 0's centre plane (crystal x ->
// (Nb-1-x) mod Nt): every transaxial offset negated; when the reflected first
// crystal comes after the second the ends swap (the spread is transposed and
// d -> -d).  A and T are commuting involutions, so a class's orbit is
// {c, A c, T c, AT c}; the spread kernel computes the smallest class index of
// each orbit and the others are its images.  sym[c] = -1 for a computed class,
// else the computed class | SYM_A << 28 | SYM_T << 29 | SYM_SWAP << 30.
constexpr int SYM_A = 1, SYM_T = 2, SYM_SWAP = 4;

// T image of transaxial class tp: its class and whether the ends swap.
__device__ __forceinline__ void t_image(const LorSet &ls, const int32_t *tp_start, int64_t tp,
                                        int64_t *tp_t, bool *swap) {
    int a0, b0;
    ls.tp_decode(tp_start, tp, &a0, &b0);
    const int ma = (ls.Nb - 1 - a0 + ls.Nt) % ls.Nt, mb = (ls.Nb - 1 - b0 + ls.Nt) % ls.Nt;
    *swap = ma > mb;
    const int a1 = *swap ? mb : ma, b1 = *swap ? ma : mb;
    const int a10 = a1 % ls.Nb, b10 = b1 - (a1 - a10);
    *tp_t = tp_start[a10] + (b10 - ls.tp_lo(a10));
}

__global__ void spread_sym_kernel(LorSet ls, int32_t *__restrict__ sym) {
    extern __shared__ int32_t sy_pre[];  // tp_start [Nt + 1], rp_start [NR + 1]
    ls.stage_prefix(sy_pre, sy_pre + ls.Nt + 1);
    __syncthreads();
    const int D = 2 * ls.Dm + 1;
    const int64_t n_cls = ls.ntp_cls * D;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cls;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tp = c / D;
        const int d = (int)(c - tp * D) - ls.Dm;
        int64_t tpt;
        bool sw;
        t_image(ls, sy_pre, tp, &tpt, &sw);
        const int dt = sw ? -d : d;
        const int64_t cA = tp * D + (-d + ls.Dm), cT = tpt * D + (dt + ls.Dm),
                      cAT = tpt * D + (-dt + ls.Dm);
        int64_t can = c < cA ? c : cA;
        can = can < cT ? can : cT;
        can = can < cAT ? can : cAT;
        if (can == c) {
            sym[c] = -1;
            continue;
        }
        // the map from the computed class to this one
        const int64_t ctp = can / D;
        const int cd = (int)(can - ctp * D) - ls.Dm;
        int64_t ctpt;
        bool csw;
        t_image(ls, sy_pre, ctp, &ctpt, &csw);
        const int cdt = csw ? -cd : cd;
        int flags;
        if (ctp * D + (-cd + ls.Dm) == c)
            flags = SYM_A;
        else if (ctpt * D + (cdt + ls.Dm) == c)
            flags = SYM_T | (csw ? SYM_SWAP : 0);
        else
            flags = SYM_A | SYM_T | (csw ? SYM_SWAP : 0);
        sym[c] = (int32_t)can | (flags << 28);
    }
}

// The classes that are images: W_c[e1][e2] = W_s[h(e1')][h(e2')] with
// (e1', e2') = (e2, e1) when the ends swap, h negating the axial offset
// (A) and/or the transaxial offset (T) of a window index.
__global__ void spread_mirror_kernel(int64_t n_cls, int Wt, int Wa,
                                     const int32_t *__restrict__ sym, float *__restrict__ out) {
    __shared__ int16_t hperm[4][256];  // window index maps per (A, T) flag pair
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a, EE = E * E;
    for (int i = threadIdx.x; i < 4 * E; i += blockDim.x) {
        const int f = i / E, e = i - f * E;
        const int x = e / W2a, z = e - x * W2a;
        hperm[f][e] = (int16_t)(((f & SYM_T) ? 2 * Wt - x : x) * W2a + ((f & SYM_A) ? 2 * Wa - z : z));
    }
    __syncthreads();
    for (int64_t c = blockIdx.x; c < n_cls; c += gridDim.x) {
        const int32_t sv = sym[c];
        if (sv < 0) continue;
        const int64_t src = sv & 0x0fffffff;
        const int flags = sv >> 28;
        const int16_t *h = hperm[flags & 3];
        const bool swap = flags & SYM_SWAP;
        float *o = out + c * EE;
        const float *sp = out + src * EE;
        for (int e = threadIdx.x; e < EE; e += blockDim.x) {
            const int e1 = e / E, e2 = e - e1 * E;
            const int s1 = swap ? e2 : e1, s2 = swap ? e1 : e2;
            o[e] = sp[h[s1] * E + h[s2]];
        }
    }
}

static int bin_spread(const psf_scanner *scanner, const psf_table_desc *desc, const float *table,
                      const double *eta, const int32_t *lors, int64_t n_lors, int32_t half_t,
                      int32_t half_a, int32_t norm, float *spread, const int32_t *sym,
                      cudaStream_t st) {
    Scan sc;
    Tab tb;
    int rc = make_scan(scanner, &sc);
    if (rc) return rc;
    rc = make_tab(desc, sc, &tb, true);
    if (rc) return rc;
    if (half_t < 0 || half_a < 0 || (half_t + 1) * (half_a + 1) > SP_QMAX) return PSF_EINVAL;
    if (norm < PSF_NORM_NONE || norm > PSF_NORM_UNIT) return PSF_EINVAL;
    if (n_lors < 0) return PSF_EINVAL;
    if (n_lors == 0) return PSF_OK;
    if (!table || !eta || !lors || !spread) return PSF_EINVAL;
    if (tb.Pt * tb.Pa > 1024) return PSF_EINVAL;
    if (half_t == 3 && half_a == 3)
        return launch_spread_q<3, 3>(sc, tb, table, eta, lors, n_lors, norm, spread, sym, st);
    if (half_t == 3 && half_a == 2)
        return launch_spread_q<3, 2>(sc, tb, table, eta, lors, n_lors, norm, spread, sym, st);
    if (half_t == 3 && half_a == 0)
        return launch_spread_q<3, 0>(sc, tb, table, eta, lors, n_lors, norm, spread, sym, st);
    size_t shm = spread_smem(tb, half_t, half_a);
    if (shm > 200 * 1024) return PSF_EINVAL;
    PSF_TRY(cudaFuncSetAttribute(spread_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shm));
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = n_lors < (int64_t)sms * 8 ? n_lors : (int64_t)sms * 8;
    {
        PSF_TIMED("spread_kernel", st);
        spread_kernel<<<(int)grid, SP_THREADS, shm, st>>>(sc, tb, table, eta, lors, n_lors, half_t,
                                                          half_a, norm, spread, sym);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

}  // namespace psf

extern "C" int psf_bin_spread(const psf_scanner *scanner, const psf_table_desc *desc,
                              const float *table, const double *eta, const int32_t *lors,
                              int64_t n_lors, int32_t half_t, int32_t half_a, int32_t norm,
                              float *spread, void *stream) {
    PSF_RANGE("psf_bin_spread");
    return bin_spread(scanner, desc, table, eta, lors, n_lors, half_t, half_a, norm, spread,
                      nullptr, as_stream(stream));
}

extern "C" int psf_bin_spread_classes(const psf_scanner *scanner, const psf_table_desc *desc,
                                      const float *table, const double *eta,
                                      const psf_lor_set *set, const int32_t *class_lors,
                                      int32_t half_t, int32_t half_a, int32_t norm,
                                      float *spread, void *stream) {
    PSF_RANGE("psf_bin_spread_classes");
    LorSet ls;
    int rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    const int64_t n_cls = ls.ntp_cls * (2 * (int64_t)ls.Dm + 1);
    if (n_cls == 0) return PSF_OK;
    if (n_cls >= (1 << 28) || (2 * half_t + 1) * (2 * half_a + 1) > 256) return PSF_EINVAL;
    if (!class_lors || !spread) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    int32_t *sym = nullptr;
    PSF_TRY(cudaMallocAsync(&sym, sizeof(int32_t) * n_cls, st));
    int dev = 0, sms = 148;
    rc = cudaGetDevice(&dev) != cudaSuccess ||
                 cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess
             ? PSF_ECUDA
             : PSF_OK;
    if (!rc) {
        PSF_TIMED("spread_sym_kernel", st);
        spread_sym_kernel<<<grid_for(n_cls, 256), 256, sizeof(int32_t) * (ls.Nt + ls.NR + 2),
                            st>>>(ls, sym);
        if (cudaGetLastError() != cudaSuccess) rc = PSF_ECUDA;
    }
    // the smallest class of each orbit through the spread kernel ...
    if (!rc)
        rc = bin_spread(scanner, desc, table, eta, class_lors, n_cls, half_t, half_a, norm,
                        spread, sym, st);
    // ... the others as its images
    if (!rc) {
        PSF_TIMED("spread_mirror_kernel", st);
        spread_mirror_kernel<<<(int)(n_cls < (int64_t)sms * 8 ? n_cls : (int64_t)sms * 8), 256, 0,
                               st>>>(n_cls, half_t, half_a, sym, spread);
        if (cudaGetLastError() != cudaSuccess) rc = PSF_ECUDA;
    }
    cudaFreeAsync(sym, st);
    return rc;
}
