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

// y[m] = sum over geometric LORs g and window entries (e1, e2) landing on m of
// w_class(g)[e1][e2] * p[g].
__global__ void __launch_bounds__(PJ_T) spread_fwd_kernel(LorSet ls, int Wt, int Wa,
                                                         const float *__restrict__ w,
                                                         const float *__restrict__ p,
                                                         float *__restrict__ y) {
    extern __shared__ int32_t shp[];
    int32_t *tp_start = shp, *rp_start = shp + ls.Nt + 1;
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a;
    const int64_t n = ls.ntp * ls.nrp;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x) {
        int a, b, ra, rb;
        ls.tp_decode(tp_start, m / ls.nrp, &a, &b);
        ls.rp_decode(rp_start, m % ls.nrp, &ra, &rb);
        float acc = 0.0f;
        for (int cs = 0; cs < 2; ++cs) {
            const int t1 = cs ? b : a, r1 = cs ? rb : ra, t2 = cs ? a : b, r2 = cs ? ra : rb;
            for (int e1 = 0; e1 < E; ++e1) {
                const int dt1 = e1 / W2a - Wt, da1 = e1 - (e1 / W2a) * W2a - Wa;
                int g1t = t1 - dt1;
                g1t += g1t < 0 ? ls.Nt : (g1t >= ls.Nt ? -ls.Nt : 0);
                const int g1r = r1 - da1;
                for (int e2 = 0; e2 < E; ++e2) {
                    const int dt2 = e2 / W2a - Wt, da2 = e2 - (e2 / W2a) * W2a - Wa;
                    int g2t = t2 - dt2;
                    g2t += g2t < 0 ? ls.Nt : (g2t >= ls.Nt ? -ls.Nt : 0);
                    const int g2r = r2 - da2;
                    if (!ls.member(g1t, g2t, g1r, g2r)) continue;
                    int64_t g = ls.row_of(tp_start, rp_start, g1t, g2t, g1r, g2r);
                    int64_t c = ls.class_of(tp_start, g1t, g2t, g1r, g2r);
                    acc = fmaf(__ldg(w + c * E * E + e1 * E + e2), __ldg(p + g), acc);
                }
            }
        }
        y[m] = acc;
    }
}

// q[g] = sum over window entries (e1, e2) of g of w_class(g)[e1][e2] * r[m(e1, e2)].
__global__ void __launch_bounds__(PJ_T) spread_adj_kernel(LorSet ls, int Wt, int Wa,
                                                         const float *__restrict__ w,
                                                         const float *__restrict__ r,
                                                         float *__restrict__ q) {
    extern __shared__ int32_t shp[];
    int32_t *tp_start = shp, *rp_start = shp + ls.Nt + 1;
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a;
    const int64_t n = ls.ntp * ls.nrp;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
        int g1t, g2t, g1r, g2r;
        ls.tp_decode(tp_start, g / ls.nrp, &g1t, &g2t);
        ls.rp_decode(rp_start, g % ls.nrp, &g1r, &g2r);
        const float *wc = w + ls.class_of(tp_start, g1t, g2t, g1r, g2r) * E * E;
        float acc = 0.0f;
        for (int e1 = 0; e1 < E; ++e1) {
            const int dt1 = e1 / W2a - Wt, da1 = e1 - (e1 / W2a) * W2a - Wa;
            int xt = g1t + dt1;
            xt += xt < 0 ? ls.Nt : (xt >= ls.Nt ? -ls.Nt : 0);
            const int xr = g1r + da1;
            if (xr < 0 || xr >= ls.NR) continue;
            for (int e2 = 0; e2 < E; ++e2) {
                const int dt2 = e2 / W2a - Wt, da2 = e2 - (e2 / W2a) * W2a - Wa;
                int yt = g2t + dt2;
                yt += yt < 0 ? ls.Nt : (yt >= ls.Nt ? -ls.Nt : 0);
                const int yr = g2r + da2;
                if (yr < 0 || yr >= ls.NR || yt == xt) continue;
                const bool sw = yt < xt;
                const int a = sw ? yt : xt, b = sw ? xt : yt;
                const int ra = sw ? yr : xr, rb = sw ? xr : yr;
                if (!ls.member(a, b, ra, rb)) continue;
                acc = fmaf(__ldg(wc + e1 * E + e2),
                           __ldg(r + ls.row_of(tp_start, rp_start, a, b, ra, rb)), acc);
            }
        }
        q[g] = acc;
    }
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
    size_t shm = sizeof(int32_t) * (m->ls.Nt + m->ls.NR + 2);
    spread_fwd_kernel<<<grid_for(m->n_rows, PJ_T), PJ_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->cls,
                                                                    m->p, y);
    PSF_LAUNCHED();
    return PSF_OK;
}

extern "C" int psf_back(const psf_matrix *m, const float *y, float *x, void *stream) {
    if (!m || !x || !y) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (m->n_rows == 0) {
        PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
        return PSF_OK;
    }
    if (!m->factored) return rows_back(m, y, x, st);
    size_t shm = sizeof(int32_t) * (m->ls.Nt + m->ls.NR + 2);
    spread_adj_kernel<<<grid_for(m->n_rows, PJ_T), PJ_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->cls,
                                                                    y, m->q);
    PSF_LAUNCHED();
    return rows_back(m, m->q, x, st);
}
