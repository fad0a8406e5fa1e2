// K8/K9: forward and back projection with the system matrix (used inside MLEM,
// Sec. 3), in two forms:
//  - stored rows (CSR of A, or of G): y = A x is a warp-per-row gather over
//    the row's columns; x = A^T y scatters each row with FP32 atomics into the
//    image, which stays resident in L2.
//  - factored PSF form A = S G for a structured LOR set (Sec. 2.3): p = G x,
//    then every measured LOR gathers the spread-weighted p of the geometric
//    LORs whose window lands on it; the adjoint gathers, for every geometric
//    LOR, the measured values its window lands on, then x = G^T q.
// Values may be FP32 or BF16/FP16 with a per-row FP32 scale; accumulation is
// FP32.
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "psf_common.cuh"
#include "psf_lorset.cuh"

struct psf_matrix {
    int64_t n_rows, n_cols;
    const int64_t *row_ptr;
    const int32_t *col;
    const void *val;
    int dtype;
    const float *row_scale;
    bool factored;
    psf::LorSet ls;
    int Wt, Wa, E;
    const float *cls;
    float *p, *q;  // plan-owned scratch [n_rows]
};

namespace psf {

template <typename VT>
__device__ __forceinline__ float ld_val(const VT *v, int64_t j);
template <>
__device__ __forceinline__ float ld_val<float>(const float *v, int64_t j) { return __ldg(v + j); }
template <>
__device__ __forceinline__ float ld_val<__nv_bfloat16>(const __nv_bfloat16 *v, int64_t j) {
    return __bfloat162float(v[j]);
}
template <>
__device__ __forceinline__ float ld_val<__half>(const __half *v, int64_t j) {
    return __half2float(v[j]);
}

constexpr int PJ_T = 256;

template <typename VT>
__global__ void __launch_bounds__(PJ_T) csr_fwd_kernel(int64_t n, const int64_t *__restrict__ ptr,
                                                      const int32_t *__restrict__ col,
                                                      const VT *__restrict__ val,
                                                      const float *__restrict__ scale,
                                                      const float *__restrict__ x,
                                                      float *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = PJ_T / 32;
    for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < n; r += gridDim.x * wpb) {
        const int64_t j0 = ptr[r], j1 = ptr[r + 1];
        float acc = 0.0f;
        for (int64_t j = j0 + lane; j < j1; j += 32) acc = fmaf(ld_val(val, j), __ldg(x + col[j]), acc);
        acc = warp_sum_f(acc);
        if (lane == 0) y[r] = scale ? acc * scale[r] : acc;
    }
}

template <typename VT>
__global__ void __launch_bounds__(PJ_T) csr_back_kernel(int64_t n, const int64_t *__restrict__ ptr,
                                                       const int32_t *__restrict__ col,
                                                       const VT *__restrict__ val,
                                                       const float *__restrict__ scale,
                                                       const float *__restrict__ y,
                                                       float *__restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = PJ_T / 32;
    for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < n; r += gridDim.x * wpb) {
        float yr = y[r];
        if (scale) yr *= scale[r];
        if (yr == 0.0f) continue;
        const int64_t j0 = ptr[r], j1 = ptr[r + 1];
        for (int64_t j = j0 + lane; j < j1; j += 32) atomicAdd(x + col[j], ld_val(val, j) * yr);
    }
}

// Tiled S and S^T.  The window of a LOR splits into 49 transaxial offsets
// (dt1, dt2) times 7 x 7 axial offsets (da1, da2).  For a fixed transaxial
// pair and a fixed (dt1, dt2), all ring pairs of the pair talk to all ring
// pairs of one other transaxial pair, and the weight depends only on the
// source's ring difference -- a 2D stencil over the ring-pair plane.  One CTA
// owns one transaxial pair (all its ring pairs, accumulated in registers) and
// walks the 49 partner pairs; each partner's values and weights are staged
// densely in shared memory (zero padded, so out-of-set ring pairs contribute
// nothing without a branch).
constexpr int ST_T = 256;
constexpr int ST_OUT = 8;  // ring pairs per thread (NR*NR <= ST_T*ST_OUT)

struct StencilSmem {
    int32_t *tp_start, *rp_start;
    short2 *rp;        // [nrp] ring pair of each row offset
    float *plane;      // [(NR+2Wa)^2] partner values, indexed [ring at end1 side][ring at end2 side]
    float *wt;         // [(2Dm+1+4Wa)][W2a][W2a] weights by source ring difference
};

__device__ __forceinline__ void stencil_smem(StencilSmem &s, unsigned char *raw, const LorSet &ls,
                                             int Wa) {
    const int P = ls.NR + 2 * Wa, W2a = 2 * Wa + 1, ND = 2 * ls.Dm + 1 + 4 * Wa;
    s.plane = reinterpret_cast<float *>(raw);
    s.wt = s.plane + P * P;
    s.rp = reinterpret_cast<short2 *>(s.wt + ND * W2a * W2a);
    s.tp_start = reinterpret_cast<int32_t *>(s.rp + ls.nrp);
    s.rp_start = s.tp_start + ls.Nt + 1;
}

static size_t stencil_smem_bytes(const LorSet &ls, int Wa) {
    const int P = ls.NR + 2 * Wa, W2a = 2 * Wa + 1, ND = 2 * ls.Dm + 1 + 4 * Wa;
    return sizeof(float) * (P * P + ND * W2a * W2a) + sizeof(short2) * ls.nrp +
           sizeof(int32_t) * (ls.Nt + ls.NR + 2) + 16;
}

__device__ __forceinline__ int tp_index(const LorSet &ls, const int32_t *tp_start, int a, int b) {
    return tp_start[a] + (b - ls.tp_lo(a));
}

__device__ __forceinline__ bool tp_member(const LorSet &ls, int a, int b) {
    int d = b - a;
    return a < b && d >= ls.Nt / 2 - ls.F && d <= ls.Nt / 2 + ls.F;
}

// adjoint == false: y[m] = sum_g w_g[e(g->m)] p[g]   (rows of this CTA are outputs m)
// adjoint == true : q[g] = sum_m w_g[e(g->m)] r[m]   (rows of this CTA are sources g)
template <bool adjoint>
__global__ void __launch_bounds__(ST_T) stencil_kernel(LorSet ls, int Wt, int Wa,
                                                       const float *__restrict__ w,
                                                       const float *__restrict__ in,
                                                       float *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char raw[];
    StencilSmem s;
    stencil_smem(s, raw, ls, Wa);
    ls.stage_prefix(s.tp_start, s.rp_start);
    __syncthreads();
    for (int j = threadIdx.x; j < ls.nrp; j += ST_T) {
        int r1, r2;
        ls.rp_decode(s.rp_start, j, &r1, &r2);
        s.rp[j] = make_short2((short)r1, (short)r2);
    }
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a, P = ls.NR + 2 * Wa;
    const int ND = 2 * ls.Dm + 1 + 4 * Wa, D0 = ls.Dm + 2 * Wa;  // weight slot of difference 0
    const int nrp = (int)ls.nrp;
    for (int64_t T = blockIdx.x; T < ls.ntp; T += gridDim.x) {
        int a, b;
        ls.tp_decode(s.tp_start, T, &a, &b);
        float acc[ST_OUT];
#pragma unroll
        for (int k = 0; k < ST_OUT; ++k) acc[k] = 0.0f;
        // this CTA's own transaxial class (adjoint: weights of the sources = own rows)
        const int a0 = a % ls.Nb;
        const int own_cls = tp_index(ls, s.tp_start, a0, b - (a - a0));
        for (int dt = 0; dt < (2 * Wt + 1) * (2 * Wt + 1); ++dt) {
            const int dt1 = dt / (2 * Wt + 1) - Wt, dt2 = dt % (2 * Wt + 1) - Wt;
            // partner crystals on the side of a and of b
            int pa = adjoint ? a + dt1 : a - dt1, pb = adjoint ? b + dt2 : b - dt2;
            pa += pa < 0 ? ls.Nt : (pa >= ls.Nt ? -ls.Nt : 0);
            pb += pb < 0 ? ls.Nt : (pb >= ls.Nt ? -ls.Nt : 0);
            if (pa == pb) continue;
            const bool sw = pa > pb;  // partner's canonical first crystal is pb
            const int c1 = sw ? pb : pa, c2 = sw ? pa : pb;
            if (!tp_member(ls, c1, c2)) continue;
            const int64_t prow = (int64_t)tp_index(ls, s.tp_start, c1, c2) * nrp;
            __syncthreads();  // previous partner fully consumed
            for (int i = threadIdx.x; i < P * P; i += ST_T) s.plane[i] = 0.0f;
            for (int i = threadIdx.x; i < ND * W2a * W2a; i += ST_T) s.wt[i] = 0.0f;
            __syncthreads();
            // partner values, oriented [ring on a's side][ring on b's side]
            for (int j = threadIdx.x; j < nrp; j += ST_T) {
                short2 rr = s.rp[j];
                int ra = sw ? rr.y : rr.x, rb = sw ? rr.x : rr.y;
                s.plane[(ra + Wa) * P + (rb + Wa)] = __ldg(in + prow + j);
            }
            // weights: forward uses the partner's class, adjoint its own; the
            // window entry of the end on a's side is (dt1, da1)
            const int cls = adjoint ? own_cls : tp_index(ls, s.tp_start, c1 % ls.Nb,
                                                         c2 - (c1 - c1 % ls.Nb));
            const bool wsw = adjoint ? false : sw;  // whose end 1 sits on a's side
            for (int i = threadIdx.x; i < (2 * ls.Dm + 1) * W2a * W2a; i += ST_T) {
                const int dl = i / (W2a * W2a) - ls.Dm;          // ring difference, a->b frame
                const int da1 = (i / W2a) % W2a, da2 = i % W2a;  // offset indices
                const int e_a = (dt1 + Wt) * W2a + da1, e_b = (dt2 + Wt) * W2a + da2;
                const int e1 = wsw ? e_b : e_a, e2 = wsw ? e_a : e_b;
                const int dc = wsw ? -dl : dl;  // canonical ring difference
                s.wt[(dl + D0) * W2a * W2a + da1 * W2a + da2] =
                    __ldg(w + ((int64_t)cls * (2 * ls.Dm + 1) + dc + ls.Dm) * E * E + e1 * E + e2);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < ST_OUT; ++k) {
                const int j = threadIdx.x + k * ST_T;
                if (j >= nrp) break;
                const short2 rr = s.rp[j];
                const int ra = rr.x, rb = rr.y;  // this row's rings (end on a's side, b's side)
                float v = 0.0f;
                // L1, L2 index the window offsets o = L - Wa of the ends on a's
                // and b's side.  Forward: the source sits at rings (ra - o1,
                // rb - o2) and its own ring difference picks the weight; adjoint:
                // the target sits at (ra + o1, rb + o2), weight by this row's
                // difference.  Plane rows/cols are ring + Wa.
                for (int L1 = 0; L1 < W2a; ++L1) {
                    for (int L2 = 0; L2 < W2a; ++L2) {
                        const int pr = adjoint ? ra + L1 : ra + 2 * Wa - L1;
                        const int pc = adjoint ? rb + L2 : rb + 2 * Wa - L2;
                        const int dl = adjoint ? rb - ra : (rb - ra) - (L2 - L1);
                        v = fmaf(s.wt[(dl + D0) * W2a * W2a + L1 * W2a + L2], s.plane[pr * P + pc], v);
                    }
                }
                acc[k] += v;
            }
        }
        const int64_t orow = T * nrp;
#pragma unroll
        for (int k = 0; k < ST_OUT; ++k) {
            const int j = threadIdx.x + k * ST_T;
            if (j < nrp) out[orow + j] = acc[k];
        }
        __syncthreads();
    }
}

// Register-blocked form of the same stencil.  The partner's plane is stored by
// (ring on a's side, ring difference) so that threads with consecutive ring
// differences read consecutive words.  Thread (dl, strip) owns the K rows
// (ra, ra + dl), ra in [strip*K, strip*K + K): along such a diagonal the ring
// difference, hence the weight of every axial offset pair, is constant.  For
// each offset difference e = o1 - o2 the partner values the K rows need lie in
// one plane column (difference dl + e forward, dl - e adjoint) and K + 2*WA
// consecutive rows; they are loaded once into registers and reused by every
// offset pair (o1, o1 - e).
template <bool adjoint, int WA, int K>
__global__ void __launch_bounds__(ST_T) stencil2_kernel(LorSet ls, int Wt,
                                                        const float *__restrict__ w,
                                                        const float *__restrict__ in,
                                                        float *__restrict__ out) {
    constexpr int W2a = 2 * WA + 1;
    extern __shared__ __align__(16) unsigned char raw[];
    const int Dm = ls.Dm, NR = ls.NR;
    const int PD = 2 * Dm + 1 + 4 * WA;  // plane columns: differences -Dm-2WA .. Dm+2WA
    // plane rows: rings -WA .. nstrip*K-1+WA (every strip reads K + 2WA rows)
    const int PR = (NR + K - 1) / K * K + 2 * WA;
    const int D0 = Dm + 2 * WA;          // column / weight slot of difference 0
    const int E = (2 * Wt + 1) * W2a;
    float *plane = reinterpret_cast<float *>(raw);
    float *wt = plane + PR * PD;                                   // [PD][W2a][W2a]
    short2 *rp = reinterpret_cast<short2 *>(wt + PD * W2a * W2a);  // [nrp]
    int32_t *tp_start = reinterpret_cast<int32_t *>(rp + ls.nrp);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    for (int j = threadIdx.x; j < ls.nrp; j += ST_T) {
        int r1, r2;
        ls.rp_decode(rp_start, j, &r1, &r2);
        rp[j] = make_short2((short)r1, (short)r2);
    }
    const int nd = 2 * Dm + 1, nstrip = (NR + K - 1) / K;
    const int items = nd * nstrip;
    const int nrp = (int)ls.nrp;
    for (int64_t T = blockIdx.x; T < ls.ntp; T += gridDim.x) {
        int a, b;
        ls.tp_decode(tp_start, T, &a, &b);
        const int a0 = a % ls.Nb;
        const int own_cls = tp_index(ls, tp_start, a0, b - (a - a0));
        for (int it0 = 0; it0 < items; it0 += ST_T) {
            const int item = it0 + threadIdx.x;
            const bool active = item < items;
            const int dl = (active ? item % nd : 0) - Dm;  // this thread's ring difference
            const int r0 = (active ? item / nd : 0) * K;   // first ring of its strip
            float acc[K];
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = 0.0f;
            for (int dt = 0; dt < (2 * Wt + 1) * (2 * Wt + 1); ++dt) {
                const int dt1 = dt / (2 * Wt + 1) - Wt, dt2 = dt % (2 * Wt + 1) - Wt;
                int pa = adjoint ? a + dt1 : a - dt1, pb = adjoint ? b + dt2 : b - dt2;
                pa += pa < 0 ? ls.Nt : (pa >= ls.Nt ? -ls.Nt : 0);
                pb += pb < 0 ? ls.Nt : (pb >= ls.Nt ? -ls.Nt : 0);
                if (pa == pb) continue;
                const bool sw = pa > pb;
                const int c1 = sw ? pb : pa, c2 = sw ? pa : pb;
                if (!tp_member(ls, c1, c2)) continue;
                const int64_t prow = (int64_t)tp_index(ls, tp_start, c1, c2) * nrp;
                __syncthreads();
                for (int i = threadIdx.x; i < PR * PD; i += ST_T) plane[i] = 0.0f;
                for (int i = threadIdx.x; i < PD * W2a * W2a; i += ST_T) wt[i] = 0.0f;
                __syncthreads();
                for (int j = threadIdx.x; j < nrp; j += ST_T) {
                    const short2 rr = rp[j];
                    const int ra = sw ? rr.y : rr.x, rb = sw ? rr.x : rr.y;
                    plane[(ra + WA) * PD + (rb - ra + D0)] = __ldg(in + prow + j);
                }
                const int cls = adjoint ? own_cls
                                        : tp_index(ls, tp_start, c1 % ls.Nb, c2 - (c1 - c1 % ls.Nb));
                const bool wsw = adjoint ? false : sw;
                for (int i = threadIdx.x; i < nd * W2a * W2a; i += ST_T) {
                    const int d = i / (W2a * W2a) - Dm;
                    const int L1 = (i / W2a) % W2a, L2 = i % W2a;
                    const int e_a = (dt1 + Wt) * W2a + L1, e_b = (dt2 + Wt) * W2a + L2;
                    const int e1 = wsw ? e_b : e_a, e2 = wsw ? e_a : e_b;
                    const int dc = wsw ? -d : d;
                    wt[(d + D0) * W2a * W2a + L1 * W2a + L2] =
                        __ldg(w + ((int64_t)cls * nd + dc + Dm) * E * E + e1 * E + e2);
                }
                __syncthreads();
                if (!active) continue;
#pragma unroll
                for (int e = -2 * WA; e <= 2 * WA; ++e) {
                    // forward: sources at (ra - o1, rb - o2), difference dl + e, weight by it;
                    // adjoint: targets at (ra + o1, rb + o2), difference dl - e, weight by dl
                    const int colp = (adjoint ? dl - e : dl + e) + D0;
                    const float *wrow = wt + (adjoint ? dl + D0 : colp) * W2a * W2a;
                    float v[K + 2 * WA];
#pragma unroll
                    for (int i = 0; i < K + 2 * WA; ++i) {
                        // v[i] = plane row (r0 + i - WA) + WA
                        v[i] = plane[(r0 + i) * PD + colp];
                    }
#pragma unroll
                    for (int o1 = -WA; o1 <= WA; ++o1) {
                        const int o2 = o1 - e;
                        if (o2 < -WA || o2 > WA) continue;
                        const float wv = wrow[(o1 + WA) * W2a + (o2 + WA)];
#pragma unroll
                        for (int k = 0; k < K; ++k)
                            acc[k] = fmaf(wv, v[adjoint ? k + o1 + WA : k - o1 + WA], acc[k]);
                    }
                }
            }
            if (active) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int ra = r0 + k, rb = ra + dl;
                    if (ra < NR && rb >= 0 && rb < NR)
                        out[T * nrp + rp_start[ra] + (rb - ls.rp_lo(ra))] = acc[k];
                }
            }
        }
        __syncthreads();
    }
}

constexpr int ST2_K = 8;  // rows per thread in stencil2_kernel

static size_t stencil2_smem_bytes(const LorSet &ls, int Wa) {
    const int PD = 2 * ls.Dm + 1 + 4 * Wa, W2a = 2 * Wa + 1;
    const int PR = (ls.NR + ST2_K - 1) / ST2_K * ST2_K + 2 * Wa;
    return sizeof(float) * (PR * PD + PD * W2a * W2a) + sizeof(short2) * ls.nrp +
           sizeof(int32_t) * (ls.Nt + ls.NR + 2) + 16;
}

template <typename F>
static int dispatch_dtype(int dtype, F &&f) {
    if (dtype == PSF_F32) return f((const float *)nullptr);
    if (dtype == PSF_BF16) return f((const __nv_bfloat16 *)nullptr);
    return f((const __half *)nullptr);
}

static int rows_fwd(const psf_matrix *m, const float *x, float *y, cudaStream_t st) {
    int grid = grid_for(m->n_rows * 32, PJ_T);
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        csr_fwd_kernel<VT><<<grid, PJ_T, 0, st>>>(m->n_rows, m->row_ptr, m->col,
                                                   (const VT *)m->val, m->row_scale, x, y);
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

static int rows_back(const psf_matrix *m, const float *y, float *x, cudaStream_t st) {
    PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
    int grid = grid_for(m->n_rows * 32, PJ_T);
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        csr_back_kernel<VT><<<grid, PJ_T, 0, st>>>(m->n_rows, m->row_ptr, m->col,
                                                    (const VT *)m->val, m->row_scale, y, x);
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

// S (adjoint == false) or S^T on LOR-space vectors of a factored plan.
template <bool adjoint, int WA>
static int launch_stencil2(const psf_matrix *m, const float *in, float *out, int grid,
                           cudaStream_t st) {
    const size_t shm = stencil2_smem_bytes(m->ls, WA);
    PSF_TRY(cudaFuncSetAttribute(stencil2_kernel<adjoint, WA, ST2_K>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    stencil2_kernel<adjoint, WA, ST2_K><<<grid, ST_T, shm, st>>>(m->ls, m->Wt, m->cls, in, out);
    PSF_LAUNCHED();
    return PSF_OK;
}

static int stencil(const psf_matrix *m, const float *in, float *out, bool adjoint,
                   cudaStream_t st) {
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t grid = m->ls.ntp < (int64_t)sms * 8 ? m->ls.ntp : (int64_t)sms * 8;
    switch (m->Wa * 2 + (adjoint ? 1 : 0)) {  // register-blocked form for axial windows <= 3
        case 0: return launch_stencil2<false, 0>(m, in, out, (int)grid, st);
        case 1: return launch_stencil2<true, 0>(m, in, out, (int)grid, st);
        case 2: return launch_stencil2<false, 1>(m, in, out, (int)grid, st);
        case 3: return launch_stencil2<true, 1>(m, in, out, (int)grid, st);
        case 4: return launch_stencil2<false, 2>(m, in, out, (int)grid, st);
        case 5: return launch_stencil2<true, 2>(m, in, out, (int)grid, st);
        case 6: return launch_stencil2<false, 3>(m, in, out, (int)grid, st);
        case 7: return launch_stencil2<true, 3>(m, in, out, (int)grid, st);
        default: break;
    }
    const size_t shm = stencil_smem_bytes(m->ls, m->Wa);
    if (adjoint) {
        PSF_TRY(cudaFuncSetAttribute(stencil_kernel<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        stencil_kernel<true><<<(int)grid, ST_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->cls, in, out);
    } else {
        PSF_TRY(cudaFuncSetAttribute(stencil_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        stencil_kernel<false><<<(int)grid, ST_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->cls, in, out);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

}  // namespace psf

using namespace psf;

extern "C" int psf_matrix_create(psf_matrix **out, int64_t n_rows, int64_t n_cols,
                                 const int64_t *row_ptr, const int32_t *col, const void *val,
                                 int32_t dtype, const float *row_scale, void *stream) {
    (void)stream;
    if (!out || n_rows < 0 || n_cols < 1 || !row_ptr) return PSF_EINVAL;
    if (n_rows > 0 && (!col || !val)) return PSF_EINVAL;
    if (dtype < PSF_F32 || dtype > PSF_F16) return PSF_EINVAL;
    if ((dtype == PSF_F32) != (row_scale == nullptr)) return PSF_EINVAL;
    psf_matrix *m = new psf_matrix();
    m->n_rows = n_rows;
    m->n_cols = n_cols;
    m->row_ptr = row_ptr;
    m->col = col;
    m->val = val;
    m->dtype = dtype;
    m->row_scale = row_scale;
    m->factored = false;
    m->p = m->q = nullptr;
    if (n_rows > 0) {
        if (cudaMalloc(&m->p, sizeof(float) * n_rows) != cudaSuccess ||
            cudaMalloc(&m->q, sizeof(float) * n_rows) != cudaSuccess) {
            cudaFree(m->p);
            delete m;
            return PSF_ECUDA;
        }
    }
    *out = m;
    return PSF_OK;
}

extern "C" int psf_matrix_set_spread(psf_matrix *m, const psf_scanner *scanner,
                                     const psf_lor_set *set, int32_t half_t, int32_t half_a,
                                     const float *class_spread) {
    if (!m || !class_spread || half_t < 0 || half_a < 0) return PSF_EINVAL;
    LorSet ls;
    int rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    if (ls.ntp * ls.nrp != m->n_rows) return PSF_EINVAL;
    if (ls.nrp > ST_T * ST_OUT || stencil_smem_bytes(ls, half_a) > 200 * 1024 ||
        stencil2_smem_bytes(ls, half_a) > 200 * 1024 || ls.NR > 32000)
        return PSF_EINVAL;
    m->factored = true;
    m->ls = ls;
    m->Wt = half_t;
    m->Wa = half_a;
    m->E = (2 * half_t + 1) * (2 * half_a + 1);
    m->cls = class_spread;
    return PSF_OK;
}

extern "C" int psf_matrix_destroy(psf_matrix *m) {
    if (!m) return PSF_EINVAL;
    cudaFree(m->p);
    cudaFree(m->q);
    delete m;
    return PSF_OK;
}

extern "C" int psf_forward(const psf_matrix *m, const float *x, float *y, void *stream) {
    if (!m || !x || !y) return PSF_EINVAL;
    if (m->n_rows == 0) return PSF_OK;
    cudaStream_t st = as_stream(stream);
    if (!m->factored) return rows_fwd(m, x, y, st);
    int rc = rows_fwd(m, x, m->p, st);
    if (rc) return rc;
    return stencil(m, m->p, y, false, st);
}

extern "C" int psf_back(const psf_matrix *m, const float *y, float *x, void *stream) {
    if (!m || !x || !y) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (m->n_rows == 0) {
        PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
        return PSF_OK;
    }
    if (!m->factored) return rows_back(m, y, x, st);
    int rc = stencil(m, y, m->q, true, st);
    if (rc) return rc;
    return rows_back(m, m->q, x, st);
}
