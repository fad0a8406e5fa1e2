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
    // stored-row projectors: persistent work-queue launch when wq_chunk > 0
    // (chosen by psf_matrix_autotune), else the grid-stride kernels
    int wq_chunk, wq_threads;     // back projection (and forward unless fwd_chunk set)
    int fwd_chunk, fwd_threads;   // forward: -1 streaming tiles, 0 grid-stride, > 0 queue
    unsigned long long *queue;  // plan-owned row counter
    // factored plans: stencil form per direction (0: default order, 3 or 4:
    // that form), chosen by psf_matrix_autotune
    int st_form[2];
    float2 *img2;  // plan-owned [n_cols]: the image pair of psf_back_sens
    // factored plans: per spread class, its window weights summed over all
    // transaxial partners (plan-owned, sized at psf_matrix_set_spread)
    float *csum;
    int64_t csum_n;
    // factored plans with top-N spreads (psf_matrix_set_spread_topn): the
    // kept window entries and weights of each class, N per class
    int topn;
    const int32_t *tidx;
    const float *tw;
    // or the kept weights as BF16 codes with one FP32 scale per class
    // (psf_matrix_set_spread_topn_bf16): weight = code x scale
    const __nv_bfloat16 *twh;
    const float *tsc;
    // bulk-staged projector forms (launch form -2, FP32 rows): the first row
    // of each BK_CAP-entry chunk (plan-owned, built on first use), and the
    // form of the pair back-projection of psf_back_sens (-2 bulk, else the
    // back projection's launch)
    int64_t *bk_first;
    int64_t bk_nch, bk_nnz;
    int pair_form;
    int *status;  // plan-owned device status word (PSF_ETIMEOUT from a bounded wait)
    // top-N plans after psf_matrix_build_sparse_adjoint (plan-owned): the
    // transpose of S (per measured LOR, its sources and weights), a list of
    // an input's nonzero entries and their count
    int64_t *tr_ptr;
    int32_t *tr_src;
    float *tr_w;
    int32_t *tr_list;
    unsigned long long *tr_nz;
    // stencil form 5 (plan-owned): the LOR-space input packed into padded
    // ring-pair planes, and the class spreads re-laid out as one contiguous
    // slice per (transaxial class, partner offset); wpad_dirty after
    // psf_matrix_set_spread (rebuilt by the next form-5 stencil)
    float *pin, *wpad;
    int64_t pin_n, wpad_n;
    bool wpad_dirty;
    // a plan without stored rows (psf_matrix_create_otf): the rows of the
    // structured set otf_ls are traced whenever they are needed
    bool otf;
    psf::Scan otf_sc;
    psf::Img otf_im;
    psf::LorSet otf_ls;
    // the voxel grid of the columns (psf_matrix_set_image): nx, ny, nz and the
    // multiply-shift forms of the divisions by nx * ny and nx; enables the
    // per-pair shared-memory accumulation of psf_back_sens (pair form -3)
    int img_nx, img_ny, img_nz;
    unsigned dv_xy_m, dv_x_m;
    int dv_xy_k, dv_x_k;
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

// Streamed (read-once) matrix entries: evict-first, so the image keeps L2.
template <typename VT>
__device__ __forceinline__ float ld_val_cs(const VT *v, int64_t j);
template <>
__device__ __forceinline__ float ld_val_cs<float>(const float *v, int64_t j) { return __ldcs(v + j); }
template <>
__device__ __forceinline__ float ld_val_cs<__nv_bfloat16>(const __nv_bfloat16 *v, int64_t j) {
    return __bfloat162float(v[j]);
}
template <>
__device__ __forceinline__ float ld_val_cs<__half>(const __half *v, int64_t j) {
    return __half2float(v[j]);
}

// Warp per row.  A lane issues the column and value loads of up to four of
// its row entries before the image gathers that depend on them, so a row of
// up to 128 entries costs one round trip for each.
template <typename VT>
__global__ void __launch_bounds__(PJ_T) csr_fwd_kernel(int64_t n, const int64_t *__restrict__ ptr,
                                                      const int32_t *__restrict__ col,
                                                      const VT *__restrict__ val,
                                                      const float *__restrict__ scale,
                                                      const float *__restrict__ x,
                                                      float *__restrict__ y) {
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const int64_t wpb = PJ_T / 32;
    for (int64_t r = blockIdx.x * wpb + (threadIdx.x >> 5); r < n; r += gridDim.x * wpb) {
        const int64_t j0 = ptr[r], j1 = ptr[r + 1];
        float acc = 0.0f;
        for (int64_t j = j0 + lane; j < j1; j += 32 * U) {
            int c[U];
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t jj = j + 32 * u;
                c[u] = jj < j1 ? __ldcs(col + jj) : 0;
                v[u] = jj < j1 ? ld_val_cs(val, jj) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j + 32 * u < j1) acc = fmaf(v[u], __ldg(x + c[u]), acc);
        }
        acc = warp_sum_f(acc);
        if (lane == 0) y[r] = scale ? acc * scale[r] : acc;
    }
}

// Scatter of one row into the image by a warp (FP32 atomics in L2).
template <typename VT>
__device__ __forceinline__ void csr_row_scatter(const int32_t *__restrict__ col,
                                                const VT *__restrict__ val, int64_t j0,
                                                int64_t j1, float yr, float *__restrict__ x,
                                                int lane) {
    for (int64_t j = j0 + lane; j < j1; j += 32)
        atomicAdd(x + __ldcs(col + j), ld_val_cs(val, j) * yr);
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
        csr_row_scatter(col, val, ptr[r], ptr[r + 1], yr, x, lane);
    }
}

// Persistent forms for rows of uneven length: the grid is sized to the
// resident CTAs and each warp takes the next `chunk` rows from a row counter
// (the work queue), so long and short rows balance across warps without a
// launch per batch.  Per row the arithmetic is the grid-stride kernels'.
template <typename VT>
__device__ __forceinline__ float csr_seg_dot(const int32_t *__restrict__ col,
                                             const VT *__restrict__ val,
                                             const float *__restrict__ x, int64_t j0, int nr,
                                             int lane) {
    constexpr int U = 4;
    const int32_t *cr = col + j0;
    const VT *vr = val + j0;
    float acc = 0.0f;
    for (int j = lane; j < nr; j += 32 * U) {
        int c[U];
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int jj = j + 32 * u;
            c[u] = jj < nr ? __ldcs(cr + jj) : 0;
            v[u] = jj < nr ? ld_val_cs(vr, jj) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + 32 * u < nr) acc = fmaf(v[u], __ldg(x + c[u]), acc);
    }
    return warp_sum_f(acc);
}

template <typename VT>
__device__ __forceinline__ float csr_row_dot(const int64_t *__restrict__ ptr,
                                             const int32_t *__restrict__ col,
                                             const VT *__restrict__ val,
                                             const float *__restrict__ x, int64_t r, int lane) {
    const int64_t j0 = ptr[r];
    return csr_seg_dot(col, val, x, j0, (int)(ptr[r + 1] - j0), lane);
}

__device__ __forceinline__ int64_t wq_take(unsigned long long *queue, int chunk, int lane) {
    unsigned long long r0 = 0;
    if (lane == 0) r0 = atomicAdd(queue, (unsigned long long)chunk);
    return (int64_t)__shfl_sync(0xffffffffu, r0, 0);
}

template <typename VT>
__global__ void csr_fwd_wq_kernel(int64_t n, const int64_t *__restrict__ ptr,
                                  const int32_t *__restrict__ col, const VT *__restrict__ val,
                                  const float *__restrict__ scale, const float *__restrict__ x,
                                  float *__restrict__ y, unsigned long long *queue, int chunk) {
    const int lane = threadIdx.x & 31;
    for (int64_t r0 = wq_take(queue, chunk, lane); r0 < n; r0 = wq_take(queue, chunk, lane)) {
        const int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
        // 32 rows at a time: their extents loaded one per lane, each row's sum
        // kept by its lane and stored together
        for (int64_t rb = r0; rb < r1; rb += 32) {
            const int64_t rr = rb + lane;
            int64_t pa = 0, pb = 0;
            if (rr < r1) {
                pa = ptr[rr];
                pb = ptr[rr + 1];
            }
            const int nb = r1 - rb < 32 ? (int)(r1 - rb) : 32;
            float mine = 0.0f;
            for (int i = 0; i < nb; ++i) {
                const int64_t a = __shfl_sync(0xffffffffu, pa, i);
                const int64_t b = __shfl_sync(0xffffffffu, pb, i);
                const float acc = csr_seg_dot(col, val, x, a, (int)(b - a), lane);
                if (lane == i) mine = acc;
            }
            if (rr < r1) y[rr] = scale ? mine * scale[rr] : mine;
        }
    }
}

template <typename VT>
__global__ void csr_back_wq_kernel(int64_t n, const int64_t *__restrict__ ptr,
                                   const int32_t *__restrict__ col, const VT *__restrict__ val,
                                   const float *__restrict__ scale, const float *__restrict__ y,
                                   float *__restrict__ x, unsigned long long *queue, int chunk,
                                   const unsigned long long *listed = nullptr) {
    const int lane = threadIdx.x & 31;
    if (listed && *listed <= (unsigned long long)(n >> 2)) return;  // the list form has it
    for (int64_t r0 = wq_take(queue, chunk, lane); r0 < n; r0 = wq_take(queue, chunk, lane)) {
        const int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
        // 32 rows at a time: values and extents loaded one per lane, rows with
        // y = 0 skipped by a ballot
        for (int64_t rb = r0; rb < r1; rb += 32) {
            const int64_t rr = rb + lane;
            float yr = 0.0f;
            int64_t pa = 0, pb = 0;
            if (rr < r1) {
                yr = y[rr];
                if (scale) yr *= scale[rr];
                if (yr != 0.0f) {
                    pa = ptr[rr];
                    pb = ptr[rr + 1];
                }
            }
            unsigned todo = __ballot_sync(0xffffffffu, yr != 0.0f && pb > pa);
            while (todo) {
                const int i = __ffs(todo) - 1;
                todo &= todo - 1;
                csr_row_scatter(col, val, __shfl_sync(0xffffffffu, pa, i),
                                __shfl_sync(0xffffffffu, pb, i), __shfl_sync(0xffffffffu, yr, i),
                                x, lane);
            }
        }
    }
}

// Masked forward (psf_forward_masked): the rows with a nonzero mask are
// listed (warp-aggregated appends; the list's order does not matter, each
// row's dot product is computed alone), then one warp per listed row.
__global__ void mask_rows_kernel(const float *__restrict__ mask, int64_t n,
                                 int32_t *__restrict__ list, unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = base + lane;
        const bool on = r < n && mask[r] != 0.0f;
        const unsigned b = __ballot_sync(0xffffffffu, on);
        unsigned long long at = 0;
        if (lane == 0 && b) at = atomicAdd(count, (unsigned long long)__popc(b));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (on) list[at + __popc(b & ((1u << lane) - 1u))] = (int32_t)r;
    }
}

// The same list from 16-byte loads (mask 16-byte aligned): a thread takes a
// quad, a warp scan of the quads' counts places its entries.
__global__ void mask_rows4_kernel(const float *__restrict__ mask, int64_t n,
                                  int32_t *__restrict__ list, unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    const int64_t nq = (n + 3) / 4;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31;
         base < nq; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t qd = base + lane, i0 = 4 * qd;
        unsigned bits = 0;
        if (qd < nq) {
            if (i0 + 3 < n) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(mask + i0));
                bits = (v.x != 0.0f) | (v.y != 0.0f) << 1 | (v.z != 0.0f) << 2 | (v.w != 0.0f) << 3;
            } else {
                for (int u = 0; i0 + u < n; ++u) bits |= (mask[i0 + u] != 0.0f) << u;
            }
        }
        const int c = __popc(bits);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        unsigned long long at = 0;
        if (lane == 31 && incl) at = atomicAdd(count, (unsigned long long)incl);
        at = __shfl_sync(0xffffffffu, at, 31);
        unsigned long long pos = at + (incl - c);
        for (int u = 0; u < 4; ++u)
            if ((bits >> u) & 1u) list[pos++] = (int32_t)(i0 + u);
    }
}

// List the rows with mask != 0 into list, their number into *count (which
// the caller zeroed); the order of the list is not defined.
static void list_nonzero(const float *mask, int64_t n, int32_t *list, unsigned long long *count,
                         cudaStream_t st) {
    PSF_TIMED("mask_rows_kernel", st);
    if (reinterpret_cast<uintptr_t>(mask) & 15)
        mask_rows_kernel<<<grid_for(n, 256), 256, 0, st>>>(mask, n, list, count);
    else
        mask_rows4_kernel<<<grid_for((n + 3) / 4, 256), 256, 0, st>>>(mask, n, list, count);
}

// x += A^T y over a list of rows (the rows with y != 0), one warp per listed
// row; returns at once when more than a quarter of the rows are listed (the
// work-queue pass runs instead).
template <typename VT>
__global__ void __launch_bounds__(PJ_T) csr_back_list_kernel(
    const int32_t *__restrict__ list, const unsigned long long *count, int64_t n,
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, const VT *__restrict__ val,
    const float *__restrict__ scale, const float *__restrict__ y, float *__restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int64_t nl = (int64_t)*count;
    if (nl > (n >> 2)) return;
    const int64_t wpb = PJ_T / 32;
    for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nl; i += gridDim.x * wpb) {
        const int64_t r = list[i];
        float yr = y[r];
        if (scale) yr *= scale[r];
        csr_row_scatter(col, val, ptr[r], ptr[r + 1], yr, x, lane);
    }
}

template <typename VT>
__global__ void __launch_bounds__(PJ_T) csr_fwd_list_kernel(
    const int32_t *__restrict__ list, const unsigned long long *count,
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, const VT *__restrict__ val,
    const float *__restrict__ scale, const float *__restrict__ x, float *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t nl = (int64_t)*count;
    const int64_t wpb = PJ_T / 32;
    for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nl; i += gridDim.x * wpb) {
        const int64_t r = list[i];
        const float acc = csr_row_dot(ptr, col, val, x, r, lane);
        if (lane == 0) y[r] = scale ? acc * scale[r] : acc;
    }
}

__global__ void keep_masked_kernel(const float *__restrict__ mask, float *__restrict__ y,
                                   int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i] == 0.0f) y[i] = 0.0f;
}

// Streaming form of y = A x for FP32 rows: a CTA takes a tile of CS_ROWS
// consecutive rows and streams their entries with 16-byte loads, four
// entries per thread per step regardless of where rows begin, so the loads
// of a whole step are in flight at once.  The products go to shared memory
// and each warp then adds the part of its rows that lies in the step (a
// fixed order, so the result is deterministic).
constexpr int CS_T = 256, CS_ROWS = 64, CS_STEP = CS_T * 4;

__global__ void __launch_bounds__(CS_T) csr_fwd_stream_kernel(
    int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y) {
    __shared__ int64_t rp[CS_ROWS + 1];
    __shared__ __align__(16) float prod[CS_STEP];
    __shared__ float racc[CS_ROWS];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t ntile = (n + CS_ROWS - 1) / CS_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t r0 = tile * CS_ROWS;
        const int nr = n - r0 < CS_ROWS ? (int)(n - r0) : CS_ROWS;
        __syncthreads();  // the previous tile's readers are done
        for (int i = t; i <= nr; i += CS_T) rp[i] = ptr[r0 + i];
        for (int i = t; i < CS_ROWS; i += CS_T) racc[i] = 0.0f;
        __syncthreads();
        const int64_t j0 = rp[0], j1 = rp[nr];
        for (int64_t base = j0 & ~(int64_t)3; base < j1; base += CS_STEP) {
            const int64_t jj = base + 4 * t;
            float p[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (jj >= j0 && jj + 3 < j1) {
                const int4 c = __ldcs(reinterpret_cast<const int4 *>(col + jj));
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(val + jj));
                p[0] = v.x * __ldg(x + c.x);
                p[1] = v.y * __ldg(x + c.y);
                p[2] = v.z * __ldg(x + c.z);
                p[3] = v.w * __ldg(x + c.w);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (jj + u >= j0 && jj + u < j1)
                        p[u] = __ldcs(val + jj + u) * __ldg(x + __ldcs(col + jj + u));
            }
            reinterpret_cast<float4 *>(prod)[t] = make_float4(p[0], p[1], p[2], p[3]);
            __syncthreads();
            const int64_t s1 = base + CS_STEP;
            for (int r = warp; r < nr; r += CS_T / 32) {
                const int64_t a = rp[r] > base ? rp[r] : base;
                const int64_t b = rp[r + 1] < s1 ? rp[r + 1] : s1;
                if (a >= b) continue;
                float acc = 0.0f;
                for (int64_t j = a + lane; j < b; j += 32) acc += prod[j - base];
                acc = warp_sum_f(acc);
                if (lane == 0) racc[r] += acc;
            }
            __syncthreads();
        }
        for (int i = t; i < nr; i += CS_T) y[r0 + i] = racc[i];
    }
}

// Two back-projections in one pass over the rows: x2[v] += val * (ya[r], yb[r])
// with one 8-byte vector atomic per entry into the interleaved image pair.
// Rows are taken grid-stride (queue == nullptr) or from the work queue.
template <typename VT>
__global__ void csr_back_pair_kernel(int64_t n, const int64_t *__restrict__ ptr,
                                     const int32_t *__restrict__ col, const VT *__restrict__ val,
                                     const float *__restrict__ scale,
                                     const float *__restrict__ ya, const float *__restrict__ yb,
                                     float2 *__restrict__ x2, unsigned long long *queue,
                                     int chunk) {
    const int lane = threadIdx.x & 31;
    const int64_t wpg = (int64_t)gridDim.x * (blockDim.x / 32);
    int64_t r0 = queue ? wq_take(queue, chunk, lane)
                       : (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int step = queue ? chunk : 1;
    while (r0 < n) {
        const int64_t r1 = r0 + step < n ? r0 + step : n;
        // 32 rows at a time: values and extents loaded one per lane, rows with
        // both values 0 skipped by a ballot
        for (int64_t rb = r0; rb < r1; rb += 32) {
            const int64_t rr = rb + lane;
            float wa = 0.0f, wb = 0.0f;
            int64_t pa = 0, pb = 0;
            if (rr < r1) {
                wa = ya[rr];
                wb = yb[rr];
                if (scale) {
                    wa *= scale[rr];
                    wb *= scale[rr];
                }
                if (wa != 0.0f || wb != 0.0f) {
                    pa = ptr[rr];
                    pb = ptr[rr + 1];
                }
            }
            unsigned todo = __ballot_sync(0xffffffffu, (wa != 0.0f || wb != 0.0f) && pb > pa);
            while (todo) {
                const int i = __ffs(todo) - 1;
                todo &= todo - 1;
                const float a = __shfl_sync(0xffffffffu, wa, i);
                const float b = __shfl_sync(0xffffffffu, wb, i);
                const int64_t j0 = __shfl_sync(0xffffffffu, pa, i);
                const int nr = (int)(__shfl_sync(0xffffffffu, pb, i) - j0);
                const int32_t *cr = col + j0;
                const VT *vr = val + j0;
                constexpr int U = 4;
                for (int j = lane; j < nr; j += 32 * U) {
                    int c[U];
                    float v[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int jj = j + 32 * u;
                        c[u] = jj < nr ? __ldcs(cr + jj) : -1;
                        v[u] = jj < nr ? ld_val_cs(vr, jj) : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (c[u] >= 0) atomicAdd(x2 + c[u], make_float2(v[u] * a, v[u] * b));
                }
            }
        }
        r0 = queue ? wq_take(queue, chunk, lane) : r0 + wpg;
    }
}

// Division by a fixed divisor with a multiply and a shift (Granlund and
// Montgomery, 1994): for d >= 1 and every n < 2^N, n / d = (n m) >> k with
// k = N + ceil(log2 d) and m = ceil(2^k / d).
struct DivMagic {
    unsigned m;  // < 2^32 for N <= 30
    int k;
    __host__ __device__ unsigned div(unsigned n) const {
        return (unsigned)(((unsigned long long)n * m) >> k);
    }
};

static DivMagic div_magic(unsigned d, unsigned long long n_end) {
    int N = 1, l = 0;
    while (N < 32 && (1ull << N) < n_end) ++N;
    while ((1ull << l) < d) ++l;
    DivMagic q;
    q.k = N + l;
    q.m = (unsigned)(((1ull << q.k) + d - 1) / d);
    return q;
}

// Pair back-projection with each transaxial pair's voxels accumulated in
// shared memory (pair form -3, factored plans whose image is set).  All ring
// pairs of a transaxial pair cut the same 2D cells, each voxel of the pair is
// hit by about 12 of its 1,372 rows (RING3D), and the global 8-byte reductions
// of the row-by-row form are bound by the L2's reduction rate; here one CTA
// per SM takes pairs from a counter, adds every entry's two products into a
// [z slice][cell] array of float pairs in shared memory, and flushes each
// touched voxel with one global reduction.  The cells and their voxel-order
// positions are read from the pair's direct-plane row of the middle ring
// (one z slice holding every cell of a pair whose plane crosses the image):
// a per-y-row table gives a voxel's position from its x index for the y rows
// whose cells form one run of consecutive x, so an entry outside the list
// (or past the array's capacity) is reduced into the image directly; a
// voxel's z slice and x/y index come from multiply-shift divisions.  The
// entries are read 128 per warp step, independently of row boundaries.
// Each lane keeps the start of its entries' next row in a register, so
// following the rows costs a shared-memory read only when a row ends.
// RING3D: 12.6 ms against 13.7 ms for the row-by-row form (timing copies
// with parts skipped, before the register: entry stream and set-up 7.0 ms,
// row tracking 2.2 ms, shared atomics 1.5 ms, voxel decode 1.2 ms).
constexpr int PP_T = 1024;

struct PatchGrid {
    int nx, ny, nz, nxy;
    DivMagic dxy, dx;  // column -> z slice, x/y index -> y row
    int cap;           // cells of a pair held in shared memory
    int jm;            // ring-pair index of the cell-list row
};

static size_t patch_smem_bytes(const PatchGrid &g, int nrp) {
    return sizeof(float) * 2 * (size_t)g.nz * g.cap + sizeof(int) * (size_t)g.cap +
           sizeof(int2) * (size_t)g.ny + sizeof(int) * 4 * (size_t)g.ny +
           sizeof(int) * ((size_t)nrp + 1) + sizeof(float2) * (size_t)nrp;
}

static bool patch_grid(const psf_matrix *m, PatchGrid *g, int *sms_out, size_t *shm_out);

template <typename VT>
__global__ void __launch_bounds__(PP_T, 1) csr_back_patch_kernel(
    int64_t ntp, int nrp, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
    const VT *__restrict__ val, const float *__restrict__ scale, const float *__restrict__ ya,
    const float *__restrict__ yb, float2 *__restrict__ x2, unsigned long long *pair_ctr,
    PatchGrid g) {
    extern __shared__ __align__(16) unsigned char pp_raw[];
    float *px = reinterpret_cast<float *>(pp_raw);  // [nz][cap] sums of the first LOR vector
    float *ps = px + (size_t)g.nz * g.cap;          // [nz][cap] and of the second
    float2 *rq = reinterpret_cast<float2 *>(ps + (size_t)g.nz * g.cap);  // [nrp] row values
    int2 *run = reinterpret_cast<int2 *>(rq + nrp);  // [ny] y row -> x of its first cell,
                                                     //   first cell << 16 | cells (0: none)
    int *xyl = reinterpret_cast<int *>(run + g.ny);  // [cap] cell -> x/y index
    int *rs = xyl + g.cap;                           // [nrp + 1] row starts in the pair
    int *r_first = rs + nrp + 1, *r_x = r_first + g.ny, *r_end = r_x + g.ny,
        *r_gap = r_end + g.ny;  // [ny] each: run assembly
    __shared__ long long s_T;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NW = PP_T / 32;
    for (int i = t; i < 2 * g.nz * g.cap; i += PP_T) px[i] = 0.0f;
    for (;;) {
        __syncthreads();  // the previous pair's flush is complete
        if (t == 0) s_T = (long long)atomicAdd(pair_ctr, 1ull);
        __syncthreads();
        const long long T = s_T;
        if (T >= ntp) return;
        const int64_t row0 = T * nrp;
        const int64_t E0 = ptr[row0];
        for (int i = t; i <= nrp; i += PP_T) rs[i] = (int)(ptr[row0 + i] - E0);
        for (int i = t; i < nrp; i += PP_T) {
            const float sc = scale ? scale[row0 + i] : 1.0f;
            rq[i] = make_float2(ya[row0 + i] * sc, yb[row0 + i] * sc);
        }
        for (int i = t; i < g.ny; i += PP_T) {
            r_first[i] = -1;
            r_gap[i] = 0;  // runs started in this y row, or 2 when one has a gap
        }
        __syncthreads();
        const int m0 = rs[g.jm];
        const int nc_all = rs[g.jm + 1] - m0, nc = nc_all < g.cap ? nc_all : g.cap;
        for (int i = t; i < nc; i += PP_T) {  // the cell list and its y runs
            const int c = col[E0 + m0 + i];
            const int xy = c - (int)g.dxy.div((unsigned)c) * g.nxy;
            const int iy = (int)g.dx.div((unsigned)xy), ix = xy - iy * g.nx;
            xyl[i] = xy;
            int iyp = -1, ixp = 0, iyn = -1;
            if (i > 0) {
                const int cp = col[E0 + m0 + i - 1];
                const int xyp = cp - (int)g.dxy.div((unsigned)cp) * g.nxy;
                iyp = (int)g.dx.div((unsigned)xyp);
                ixp = xyp - iyp * g.nx;
            }
            if (i + 1 < nc) {
                const int cn = col[E0 + m0 + i + 1];
                const int xyn = cn - (int)g.dxy.div((unsigned)cn) * g.nxy;
                iyn = (int)g.dx.div((unsigned)xyn);
            }
            if (iyp != iy) {
                r_first[iy] = i;
                r_x[iy] = ix;
                atomicAdd(r_gap + iy, 1);
            } else if (ix != ixp + 1) {
                atomicAdd(r_gap + iy, 2);  // not consecutive in x
            }
            if (iyn != iy) r_end[iy] = i + 1;
        }
        __syncthreads();
        for (int i = t; i < g.ny; i += PP_T) {
            // a y row's cells are used only as one run of consecutive x (a
            // cell list out of voxel order could split a y row in two)
            const int f = r_first[i];
            run[i] = f >= 0 && r_gap[i] == 1 ? make_int2(r_x[i], (f << 16) | (r_end[i] - f))
                                             : make_int2(0, 0);
        }
        __syncthreads();
        // entries in blocks of 128, entry base + lane + 32 u of each block to
        // lane u-th (consecutive entries of a row are neighbouring cells of
        // one z slice: consecutive words of the arrays, so the lanes' shared
        // atomics fall on different banks); each warp takes a contiguous run
        // of blocks, every lane finds the row of its entries by stepping
        // forward, and the next block's entries are loaded while the current
        // one is added
        const int E = rs[nrp];
        const int nblk = (E + 127) >> 7;
        const int per = (nblk + NW - 1) / NW;
        const int b0 = warp * per, b1 = b0 + per < nblk ? b0 + per : nblk;
        if (b0 < b1) {
            int r[4];    // per u: largest r with rs[r] <= the lane's entry
            int nxt[4];  // and rs[r + 1], the start of the next row
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int key = (b0 << 7) + lane + 32 * u;
                int lo = 0, hi = nrp - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (rs[mid] <= key) lo = mid; else hi = mid - 1;
                }
                r[u] = lo;
                nxt[u] = rs[lo + 1];
            }
            int c4[4];
            float v4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int rel = (b0 << 7) + lane + 32 * u;
                c4[u] = rel < E ? __ldcs(col + E0 + rel) : 0;
                v4[u] = rel < E ? ld_val_cs(val, E0 + rel) : 0.0f;
            }
            const int32_t *cb = col + E0 + lane;
            const VT *vb = val + E0 + lane;
            for (int bk = b0; bk < b1; ++bk) {
                int cn[4];
                float vn[4];
                const int nx0 = ((bk + 1) << 7) + lane;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ld = bk + 1 < b1 && nx0 + 32 * u < E;
                    cn[u] = ld ? __ldcs(cb + ((bk + 1) << 7) + 32 * u) : 0;
                    vn[u] = ld ? ld_val_cs(vb, ((bk + 1) << 7) + 32 * u) : 0.0f;
                }
                const int rel0 = (bk << 7) + lane;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int rel = rel0 + 32 * u;
                    if (rel < E) {
                        while (nxt[u] <= rel) {
                            ++r[u];
                            nxt[u] = rs[r[u] + 1];
                        }
                        const float2 q = rq[r[u]];
                        const float pa = v4[u] * q.x, pb = v4[u] * q.y;
                        const int c = c4[u];
                        const int iz = (int)g.dxy.div((unsigned)c), xy = c - iz * g.nxy;
                        const int iy = (int)g.dx.div((unsigned)xy);
                        const int2 ru = run[iy];
                        const int k = xy - iy * g.nx - ru.x;
                        const int pc = (ru.y >> 16) + k;
                        if (((unsigned)k < (unsigned)(ru.y & 0xffff)) & (iz < g.nz)) {
                            const int slot = iz * g.cap + pc;
                            atomicAdd(px + slot, pa);
                            atomicAdd(ps + slot, pb);
                        } else {
                            atomicAdd(x2 + c, make_float2(pa, pb));
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    c4[u] = cn[u];
                    v4[u] = vn[u];
                }
            }
        }
        __syncthreads();
        // flush each touched voxel with one reduction, and clear the array
        const float inv = 1.0f / (float)(nc > 0 ? nc : 1);
        for (int i = t; i < g.nz * nc; i += PP_T) {
            int iz = (int)((float)i * inv);
            iz -= iz * nc > i ? 1 : 0;
            iz += (iz + 1) * nc <= i ? 1 : 0;
            const int pc = i - iz * nc, slot = iz * g.cap + pc;
            const float2 v = make_float2(px[slot], ps[slot]);
            if (v.x != 0.0f || v.y != 0.0f) {
                atomicAdd(x2 + (int64_t)iz * g.nxy + xyl[pc], v);
                px[slot] = 0.0f;
                ps[slot] = 0.0f;
            }
        }
    }
}

// Bulk-staged forms of the FP32 projectors (launch form -2).  The entry
// arrays are cut into fixed chunks of BK_CAP entries; a CTA takes chunks
// grid-stride and one of its threads brings each chunk's columns and values
// into shared memory with two cp.async.bulk copies that complete on an
// mbarrier, one chunk ahead of the one being used (two stages), so the HBM
// stream runs independently of the image gathers and atomics.  A chunk owns
// the rows that start in it (first_row, a plan-owned table); entries of its
// rows that lie past the chunk, or in the ragged tail after the last whole 16
// bytes, are read from global memory.
constexpr int BK_T = 256, BK_CAP = 4096;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Global -> shared bulk copy completing on `bar`, marked evict-first in L2 (the
// entries are read once; the image they gather from or add into stays in L2).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for a phase of the barrier; false after `limit` SM cycles (at once for
// a negative limit).
constexpr long long BK_DRAIN_LIMIT = 1ll << 31;  // about a second at the SM clock
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    if (limit < 0) return false;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

struct BkStage {
    int32_t *col;
    float *val;
    uint64_t *bar;
};

__device__ __forceinline__ BkStage bk_stage(unsigned char *raw, int s) {
    BkStage g;
    g.col = reinterpret_cast<int32_t *>(raw) + s * BK_CAP;
    g.val = reinterpret_cast<float *>(raw + sizeof(int32_t) * 2 * BK_CAP) + s * BK_CAP;
    g.bar = reinterpret_cast<uint64_t *>(raw + (sizeof(int32_t) + sizeof(float)) * 2 * BK_CAP) + s;
    return g;
}

// Entries of chunk c copied to shared memory (a multiple of 4).
__device__ __forceinline__ int bk_copied(int64_t c, int64_t nnz) {
    const int64_t ne = nnz - c * BK_CAP;
    return (int)((ne < BK_CAP ? ne : BK_CAP) & ~(int64_t)3);
}

__device__ __forceinline__ void bk_issue(int64_t c, int64_t nnz, const int32_t *col,
                                         const float *val, const BkStage &g) {
    const uint32_t bytes = (uint32_t)bk_copied(c, nnz) * 4u;
    mbar_expect(g.bar, 2u * bytes);
    if (bytes) {
        bulk_g2s(g.col, col + c * BK_CAP, bytes, g.bar);
        bulk_g2s(g.val, val + c * BK_CAP, bytes, g.bar);
    }
}

__device__ __forceinline__ void bk_rows(const int64_t *__restrict__ first_row, int64_t c,
                                        int64_t nch, int64_t n, int64_t &r0, int64_t &r1) {
    r0 = c < nch ? first_row[c] : 0;
    r1 = c + 1 < nch ? first_row[c + 1] : (c < nch ? n : 0);
}

// After a wait gave up: record it, wait (bounded) for the copies still in
// flight into this CTA's stages, return.
__device__ __forceinline__ void bk_give_up(unsigned char *raw, int it, bool next_issued,
                                           int *status) {
    if (threadIdx.x == 0) {
        atomicExch(status, PSF_ETIMEOUT);
        mbar_wait(bk_stage(raw, it & 1).bar, (it >> 1) & 1, BK_DRAIN_LIMIT);
        if (next_issued)
            mbar_wait(bk_stage(raw, (it + 1) & 1).bar, ((it + 1) >> 1) & 1, BK_DRAIN_LIMIT);
    }
}

// End of a row's staged part, chunk-local: min(b - j0, copied), at least 0.
__device__ __forceinline__ int bk_local_end(int64_t b, int64_t j0, int copied) {
    const int64_t e = b - j0;
    return e < copied ? (e > 0 ? (int)e : 0) : copied;
}

template <bool PAIR>
__device__ __forceinline__ void bk_add(float *x, float2 *x2, int c, float v, float qa, float qb) {
    if (PAIR)
        atomicAdd(x2 + c, make_float2(v * qa, v * qb));
    else
        atomicAdd(x + c, v * qa);
}

__global__ void __launch_bounds__(BK_T) csr_fwd_bulk_kernel(
    int64_t n, int64_t nnz, int64_t nch, const int64_t *__restrict__ first_row,
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y,
    int *status, long long limit) {
    extern __shared__ __align__(128) unsigned char bk_raw[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NW = BK_T / 32, PER_T = BK_CAP / BK_T;
    if (t == 0) {
        mbar_init(bk_stage(bk_raw, 0).bar);
        mbar_init(bk_stage(bk_raw, 1).bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int64_t c = blockIdx.x;
    if (t == 0 && c < nch) bk_issue(c, nnz, col, val, bk_stage(bk_raw, 0));
    int64_t r0, r1;
    bk_rows(first_row, c, nch, n, r0, r1);
    for (int it = 0; c < nch; ++it, c += gridDim.x) {
        const BkStage g = bk_stage(bk_raw, it & 1);
        const int64_t cn = c + gridDim.x;
        if (t == 0 && cn < nch) bk_issue(cn, nnz, col, val, bk_stage(bk_raw, (it + 1) & 1));
        int64_t nr0, nr1;
        bk_rows(first_row, cn, nch, n, nr0, nr1);
        // extents of this warp's first 32 rows (rows r0 + warp + NW i)
        const int64_t rr = r0 + warp + (int64_t)NW * lane;
        int64_t pa = 0, pb = 0;
        if (rr < r1) {
            pa = ptr[rr];
            pb = ptr[rr + 1];
        }
        const bool ok = mbar_wait(g.bar, (it >> 1) & 1, limit);
        if (__syncthreads_or(!ok)) {
            bk_give_up(bk_raw, it, cn < nch, status);
            return;
        }
        const int64_t j0 = c * BK_CAP;
        const int copied = bk_copied(c, nnz);
        // products of the staged entries, in place
        int ci[PER_T];
#pragma unroll
        for (int k = 0; k < PER_T; ++k) ci[k] = t + k * BK_T < copied ? g.col[t + k * BK_T] : -1;
        float xv[PER_T];
#pragma unroll
        for (int k = 0; k < PER_T; ++k) xv[k] = ci[k] >= 0 ? __ldg(x + ci[k]) : 0.0f;
#pragma unroll
        for (int k = 0; k < PER_T; ++k)
            if (ci[k] >= 0) g.val[t + k * BK_T] *= xv[k];
        __syncthreads();
        // rows in batches of 32 per warp (lane k: row r0 + warp + NW (32 batch + k));
        // empty rows are written by their lanes, the others one at a time
        for (int64_t bb = r0 + warp; bb < r1; bb += 32 * NW) {
            const int64_t rl = bb + (int64_t)NW * lane;
            if (bb != r0 + warp) {
                pa = pb = 0;
                if (rl < r1) {
                    pa = ptr[rl];
                    pb = ptr[rl + 1];
                }
            }
            // rows of at most 32 entries: summed by their own lane
            if (rl < r1 && pb - pa <= 32) {
                float acc = 0.0f;
                const int la = (int)(pa - j0), lb = bk_local_end(pb, j0, copied);
                for (int l = la; l < lb; ++l) acc += g.val[l];
                for (int64_t j = j0 + lb > pa ? j0 + lb : pa; j < pb; ++j)
                    acc += __ldg(val + j) * __ldg(x + __ldg(col + j));
                y[rl] = acc;
            }
            unsigned todo = __ballot_sync(0xffffffffu, rl < r1 && pb - pa > 32);
            while (todo) {
                const int i = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t a = __shfl_sync(0xffffffffu, pa, i);
                const int64_t b = __shfl_sync(0xffffffffu, pb, i);
                float acc = 0.0f;
                const int la = (int)(a - j0), lb = bk_local_end(b, j0, copied);
                for (int l = la + lane; l < lb; l += 32) acc += g.val[l];
                for (int64_t j = (j0 + lb > a ? j0 + lb : a) + lane; j < b; j += 32)
                    acc += __ldg(val + j) * __ldg(x + __ldg(col + j));
                acc = warp_sum_f(acc);
                if (lane == 0) y[bb + (int64_t)NW * i] = acc;
            }
        }
        // the products were generic-proxy writes into a stage the next bulk
        // copy overwrites
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        r0 = nr0;
        r1 = nr1;
    }
}

// x += A^T y (PAIR: x2 += A^T (ya, yb) into the interleaved pair), rows of a
// chunk one per warp, entries from the staged chunk.
template <bool PAIR>
__global__ void __launch_bounds__(BK_T) csr_back_bulk_kernel(
    int64_t n, int64_t nnz, int64_t nch, const int64_t *__restrict__ first_row,
    const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ ya, const float *__restrict__ yb,
    float *__restrict__ x, float2 *__restrict__ x2, int *status, long long limit) {
    extern __shared__ __align__(128) unsigned char bk_raw[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NW = BK_T / 32;
    if (t == 0) {
        mbar_init(bk_stage(bk_raw, 0).bar);
        mbar_init(bk_stage(bk_raw, 1).bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int64_t c = blockIdx.x;
    if (t == 0 && c < nch) bk_issue(c, nnz, col, val, bk_stage(bk_raw, 0));
    int64_t r0, r1;
    bk_rows(first_row, c, nch, n, r0, r1);
    for (int it = 0; c < nch; ++it, c += gridDim.x) {
        const BkStage g = bk_stage(bk_raw, it & 1);
        const int64_t cn = c + gridDim.x;
        if (t == 0 && cn < nch) bk_issue(cn, nnz, col, val, bk_stage(bk_raw, (it + 1) & 1));
        int64_t nr0, nr1;
        bk_rows(first_row, cn, nch, n, nr0, nr1);
        const int64_t rr = r0 + warp + (int64_t)NW * lane;
        int64_t pa = 0, pb = 0;
        float wa = 0.0f, wb = 0.0f;
        if (rr < r1) {
            pa = ptr[rr];
            pb = ptr[rr + 1];
            wa = ya[rr];
            if (PAIR) wb = yb[rr];
        }
        const bool ok = mbar_wait(g.bar, (it >> 1) & 1, limit);
        if (__syncthreads_or(!ok)) {
            bk_give_up(bk_raw, it, cn < nch, status);
            return;
        }
        const int64_t j0 = c * BK_CAP;
        const int copied = bk_copied(c, nnz);
        for (int64_t bb = r0 + warp; bb < r1; bb += 32 * NW) {
            const int64_t rl = bb + (int64_t)NW * lane;
            if (bb != r0 + warp) {
                pa = pb = 0;
                wa = wb = 0.0f;
                if (rl < r1) {
                    pa = ptr[rl];
                    pb = ptr[rl + 1];
                    wa = ya[rl];
                    if (PAIR) wb = yb[rl];
                }
            }
            const bool live = rl < r1 && (wa != 0.0f || wb != 0.0f);
            // rows of at most 32 entries: added by their own lane
            if (live && pb - pa <= 32) {
                const int la = (int)(pa - j0), lb = bk_local_end(pb, j0, copied);
                for (int l = la; l < lb; ++l) bk_add<PAIR>(x, x2, g.col[l], g.val[l], wa, wb);
                for (int64_t j = j0 + lb > pa ? j0 + lb : pa; j < pb; ++j)
                    bk_add<PAIR>(x, x2, __ldg(col + j), __ldg(val + j), wa, wb);
            }
            unsigned todo = __ballot_sync(0xffffffffu, live && pb - pa > 32);
            while (todo) {
                const int i = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t a = __shfl_sync(0xffffffffu, pa, i);
                const int64_t b = __shfl_sync(0xffffffffu, pb, i);
                const float qa = __shfl_sync(0xffffffffu, wa, i);
                const float qb = PAIR ? __shfl_sync(0xffffffffu, wb, i) : 0.0f;
                const int la = (int)(a - j0), lb = bk_local_end(b, j0, copied);
                for (int l = la + lane; l < lb; l += 32)
                    bk_add<PAIR>(x, x2, g.col[l], g.val[l], qa, qb);
                for (int64_t j = (j0 + lb > a ? j0 + lb : a) + lane; j < b; j += 32)
                    bk_add<PAIR>(x, x2, __ldg(col + j), __ldg(val + j), qa, qb);
            }
        }
        __syncthreads();
        r0 = nr0;
        r1 = nr1;
    }
}

// first_row[c] = the first row r in [0, n] with ptr[r] >= c * BK_CAP.
__global__ void bk_first_row_kernel(const int64_t *__restrict__ ptr, int64_t n, int64_t nch,
                                    int64_t *__restrict__ first_row) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    const int64_t key = c * BK_CAP;
    int64_t lo = 0, hi = n;  // ptr[n] = nnz > key
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (ptr[mid] >= key)
            hi = mid;
        else
            lo = mid + 1;
    }
    first_row[c] = lo;
}

__global__ void split_pair_kernel(const float2 *__restrict__ x2, float *__restrict__ xa,
                                  float *__restrict__ xb, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = x2[i];
        xa[i] = v.x;
        xb[i] = v.y;
    }
}

__global__ void fill_kernel(float *__restrict__ a, float v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
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

// Third form of the same stencil.  One CTA of 128 threads owns one
// transaxial pair; a thread owns K = 8 rings x M = 2 consecutive ring
// differences.  Each partner's plane (by ring-difference column, rings
// contiguous, so the K + 2*WA values of one column are four 16-byte loads) and
// its weight slice (per column and e = o1 - o2, the o1 entries contiguous) are
// brought into shared memory by asynchronous copies, two partners deep, so
// the copies of the next partner overlap the arithmetic of this one.  Every
// partner writes the same cells, so the padding cells zeroed at the start stay
// zero.  For one partner column and one of the thread's differences, e is a
// compile-time constant, so every register index is static.
constexpr int ST3_T = 128, ST3_K = 8, ST3_M = 2;

struct St3Shape {
    int nd, nstrip, ndg, items, PRp, ne;
    int plane_f, w_f, buf_f;  // floats of one partner buffer
};

__host__ __device__ inline St3Shape st3_shape(const LorSet &ls, int WA) {
    St3Shape s;
    s.nd = 2 * ls.Dm + 1;
    s.nstrip = (ls.NR + ST3_K - 1) / ST3_K;
    s.ndg = (s.nd + ST3_M - 1) / ST3_M;
    s.items = s.nstrip * s.ndg;
    // rows = ring + WA, a strip reads 16 rows from its first; a column stride
    // of 4 (mod 32) words spreads consecutive columns over the banks
    s.PRp = s.nstrip * ST3_K + 8;
    s.PRp += (36 - s.PRp % 32) % 32;
    s.ne = 4 * WA + 1;
    s.plane_f = s.nd * s.PRp;
    s.w_f = s.nd * s.ne * 8;
    s.buf_f = s.plane_f + s.w_f;
    return s;
}

static size_t stencil3_smem_bytes(const LorSet &ls, int WA) {
    const St3Shape s = st3_shape(ls, WA);
    return sizeof(float) * 2 * (size_t)s.buf_f + sizeof(short2) * ls.nrp +
           sizeof(int32_t) * (ls.Nt + ls.NR + 2) + 32;
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// Transaxial partner dt of pair (a, b): false if it is not in the set.
struct St3Partner {
    int64_t prow;
    int cls, dt1, dt2;
    bool sw, wsw;
};

template <bool adjoint>
__device__ __forceinline__ bool st3_partner(const LorSet &ls, const int32_t *tp_start, int a,
                                            int b, int dt, int Wt, int own_cls, St3Partner &P) {
    P.dt1 = dt / (2 * Wt + 1) - Wt;
    P.dt2 = dt % (2 * Wt + 1) - Wt;
    int pa = adjoint ? a + P.dt1 : a - P.dt1, pb = adjoint ? b + P.dt2 : b - P.dt2;
    pa += pa < 0 ? ls.Nt : (pa >= ls.Nt ? -ls.Nt : 0);
    pb += pb < 0 ? ls.Nt : (pb >= ls.Nt ? -ls.Nt : 0);
    if (pa == pb) return false;
    P.sw = pa > pb;
    const int c1 = P.sw ? pb : pa, c2 = P.sw ? pa : pb;
    if (!tp_member(ls, c1, c2)) return false;
    P.prow = (int64_t)tp_index(ls, tp_start, c1, c2) * ls.nrp;
    P.cls = adjoint ? own_cls : tp_index(ls, tp_start, c1 % ls.Nb, c2 - (c1 - c1 % ls.Nb));
    P.wsw = adjoint ? false : P.sw;
    return true;
}

template <bool adjoint>
__device__ __forceinline__ int st3_next(const LorSet &ls, const int32_t *tp_start, int a, int b,
                                        int dt, int nwin, int Wt, int own_cls, St3Partner &P) {
    for (; dt < nwin; ++dt)
        if (st3_partner<adjoint>(ls, tp_start, a, b, dt, Wt, own_cls, P)) return dt;
    return nwin;
}

// Issue (without waiting) the copies of one partner into a buffer.
template <int WA, class Shape>
__device__ __forceinline__ void st3_stage(const LorSet &ls, const Shape &S, const short2 *rp,
                                          const St3Partner &P, int Wt,
                                          const float *__restrict__ w,
                                          const float *__restrict__ in, float *buf) {
    constexpr int W2a = 2 * WA + 1, NE = 4 * WA + 1;
    const int Dm = ls.Dm, nd = S.nd, PRp = S.PRp, nrp = (int)ls.nrp;
    const int E = (2 * Wt + 1) * W2a;
    float *plane = buf, *w3 = buf + S.plane_f;
    for (int j = threadIdx.x; j < nrp; j += blockDim.x) {
        const short2 rr = rp[j];
        const int ra = P.sw ? rr.y : rr.x, rb = P.sw ? rr.x : rr.y;
        cp_async4(plane + (rb - ra + Dm) * PRp + (ra + WA), in + P.prow + j);
    }
    // weights: one (difference, o1) pair per step, its W2a o2 entries as one
    // run -- window entry e1 = (dt1 + Wt) W2a + L1 of the end on a's side,
    // e2 = (dt2 + Wt) W2a + L2 of the other (swapped roles when the partner's
    // first crystal sits on b's side); slot (d, e = L1 - L2, L1)
    // (consecutive threads take the index that is contiguous in the class
    // table, so a warp's copies read runs of consecutive words)
    const float *wc = w + (int64_t)P.cls * nd * E * E;
    const int ea0 = (P.dt1 + Wt) * W2a, eb0 = (P.dt2 + Wt) * W2a;
    for (int i = threadIdx.x; i < nd * W2a; i += blockDim.x) {
        const int d = i / W2a - Dm, u = i % W2a;
        const float *src = wc + (int64_t)((P.wsw ? -d : d) + Dm) * E * E;
        if (!P.wsw) {  // entry (ea0 + L1) * E + eb0 + L2: thread over L2, run over L1
            const float *s0 = src + ea0 * E + eb0 + u;
            float *d0 = w3 + ((d + Dm) * NE - u + 2 * WA) * 8;
#pragma unroll
            for (int L1 = 0; L1 < W2a; ++L1) cp_async4(d0 + 9 * L1, s0 + L1 * E);
        } else {  // entry (eb0 + L2) * E + ea0 + L1: thread over L1, run over L2
            const float *s0 = src + eb0 * E + ea0 + u;
            float *d0 = w3 + ((d + Dm) * NE + u + 2 * WA) * 8 + u;
#pragma unroll
            for (int L2 = 0; L2 < W2a; ++L2) cp_async4(d0 - 8 * L2, s0 + L2 * E);
        }
    }
    cp_async_commit();
}

template <bool adjoint, int WA>
__global__ void __launch_bounds__(ST3_T, 4) stencil3_kernel(LorSet ls, int Wt,
                                                            const float *__restrict__ w,
                                                            const float *__restrict__ in,
                                                            float *__restrict__ out) {
    constexpr int NE = 4 * WA + 1, K = ST3_K, M = ST3_M;
    extern __shared__ __align__(16) unsigned char raw[];
    const St3Shape S = st3_shape(ls, WA);
    const int Dm = ls.Dm, NR = ls.NR, PRp = S.PRp;
    const int nwin = (2 * Wt + 1) * (2 * Wt + 1);
    float *bufs = reinterpret_cast<float *>(raw);  // [2][buf_f]
    short2 *rp = reinterpret_cast<short2 *>(bufs + 2 * S.buf_f);
    int32_t *tp_start = reinterpret_cast<int32_t *>(rp + ls.nrp);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    const int t = threadIdx.x;
    for (int i = t; i < 2 * S.buf_f; i += ST3_T) bufs[i] = 0.0f;
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    for (int j = t; j < ls.nrp; j += ST3_T) {
        int r1, r2;
        ls.rp_decode(rp_start, j, &r1, &r2);
        rp[j] = make_short2((short)r1, (short)r2);
    }
    __syncthreads();
    const int nrp = (int)ls.nrp;
    const bool active = t < S.items;
    const int q = active ? t / S.nstrip : 0, strip = active ? t % S.nstrip : 0;
    const int dl0 = q * M - Dm, r0 = strip * K;
    for (int64_t T = blockIdx.x; T < ls.ntp; T += gridDim.x) {
        int a, b;
        ls.tp_decode(tp_start, T, &a, &b);
        const int a0 = a % ls.Nb;
        const int own_cls = tp_index(ls, tp_start, a0, b - (a - a0));
        float acc[M][K];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[m][k] = 0.0f;
        St3Partner P;
        int dt = st3_next<adjoint>(ls, tp_start, a, b, 0, nwin, Wt, own_cls, P);
        if (dt < nwin) st3_stage<WA>(ls, S, rp, P, Wt, w, in, bufs);
        int cur = 0;
        while (dt < nwin) {
            St3Partner Pn;
            const int nxt = st3_next<adjoint>(ls, tp_start, a, b, dt + 1, nwin, Wt, own_cls, Pn);
            if (nxt < nwin)
                st3_stage<WA>(ls, S, rp, Pn, Wt, w, in, bufs + (cur ^ 1) * S.buf_f);
            else
                cp_async_commit();  // empty group keeps the count uniform
            cp_async_wait1();       // this partner's copies (all but the newest group)
            __syncthreads();
            if (active) {
                const float *plane = bufs + cur * S.buf_f, *w3 = plane + S.plane_f;
#pragma unroll
                for (int cc = 0; cc < M + 4 * WA; ++cc) {
                    const int c = dl0 - 2 * WA + cc;  // partner column (ring difference)
                    if (c < -Dm || c > Dm) continue;
                    float v[16];
                    const float4 *pv =
                        reinterpret_cast<const float4 *>(plane + (c + Dm) * PRp + r0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 f = pv[u];
                        v[4 * u] = f.x;
                        v[4 * u + 1] = f.y;
                        v[4 * u + 2] = f.z;
                        v[4 * u + 3] = f.w;
                    }
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        // forward: source difference c = dl + e, weights by c;
                        // adjoint: target difference c = dl - e, weights by dl
                        const int e = adjoint ? m + 2 * WA - cc : cc - 2 * WA - m;
                        if (e < -2 * WA || e > 2 * WA) continue;
                        const int wd = adjoint ? dl0 + m : c;
                        if (adjoint && wd > Dm) continue;
                        const float4 *pw = reinterpret_cast<const float4 *>(
                            w3 + ((wd + Dm) * NE + e + 2 * WA) * 8);
                        const float4 w0 = pw[0], w1 = pw[1];
                        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                        for (int o1 = -WA; o1 <= WA; ++o1) {
                            const int o2 = o1 - e;
                            if (o2 < -WA || o2 > WA) continue;
                            const float wgt = wv[o1 + WA];
#pragma unroll
                            for (int k = 0; k < K; ++k)
                                acc[m][k] =
                                    fmaf(wgt, v[adjoint ? k + o1 + WA : k - o1 + WA], acc[m][k]);
                        }
                    }
                }
            }
            __syncthreads();  // this buffer is free for the partner after next
            cur ^= 1;
            dt = nxt;
            P = Pn;
        }
        if (active) {
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int ra = r0 + k, dl = dl0 + m, rb = ra + dl;
                    if (ra < NR && dl <= Dm && rb >= 0 && rb < NR)
                        out[T * nrp + rp_start[ra] + (rb - ls.rp_lo(ra))] = acc[m][k];
                }
        }
    }
}

// Fourth form, for fewer distinct shared-memory addresses per warp.  Each
// half-warp owns one group of M = 4 consecutive ring differences and its 16
// lanes the strips of K = 4 rings, so a weight load has two addresses per
// warp (one per half) and a plane load is 8 bytes per lane on consecutive
// rows; a thread does K x M = 16 products per partner value pair it loads.
// Scanners of 65 to 128 rings use whole warps per group (32 strips).
// (M = 4 gives 128-thread CTAs, twice the warps per SM of M = 8 at the same
// shared memory: 12.5 / 13.3 ms against 15.4 / 17.0 ms forward / adjoint on
// the 3D ring; M = 2 14.0 / 14.2 ms.)  Staging and the partner walk are those
// of the third form.
constexpr int ST4_K = 4, ST4_M = 4;

struct St4Shape {
    int nd, nstrip, nqg, threads, PRp, ne;
    int lpg_log;  // lanes per difference group: 16 (up to 64 rings) or 32 (up to 128)
    int plane_f, w_f, buf_f;
};

__host__ __device__ inline St4Shape st4_shape(const LorSet &ls, int WA) {
    St4Shape s;
    s.nd = 2 * ls.Dm + 1;
    s.nstrip = (ls.NR + ST4_K - 1) / ST4_K;
    s.nqg = (s.nd + ST4_M - 1) / ST4_M;
    s.lpg_log = s.nstrip <= 16 ? 4 : 5;
    const int gpw = 32 >> s.lpg_log;  // groups per warp
    s.threads = 32 * ((s.nqg + gpw - 1) / gpw);
    s.PRp = s.nstrip * ST4_K + 2 * WA;  // rows = ring + WA; a strip reads K + 2 WA rows
    s.ne = 4 * WA + 1;
    s.plane_f = (s.nd * s.PRp + 3) / 4 * 4;
    s.w_f = s.nd * s.ne * 8;
    s.buf_f = s.plane_f + s.w_f;
    return s;
}

static size_t stencil4_smem_bytes(const LorSet &ls, int WA) {
    const St4Shape s = st4_shape(ls, WA);
    return sizeof(float) * 2 * (size_t)s.buf_f + sizeof(short2) * ls.nrp +
           sizeof(int32_t) * (ls.Nt + ls.NR + 2) + 32;
}

template <bool adjoint, int WA>
__global__ void __launch_bounds__(256) stencil4_kernel(LorSet ls, int Wt,
                                                        const float *__restrict__ w,
                                                        const float *__restrict__ in,
                                                        float *__restrict__ out) {
    constexpr int NE = 4 * WA + 1, K = ST4_K, M = ST4_M, NV = K + 2 * WA;
    static_assert(NV % 2 == 0, "8-byte plane loads");
    extern __shared__ __align__(16) unsigned char raw[];
    const St4Shape S = st4_shape(ls, WA);
    const int Dm = ls.Dm, NR = ls.NR, PRp = S.PRp;
    const int nwin = (2 * Wt + 1) * (2 * Wt + 1);
    float *bufs = reinterpret_cast<float *>(raw);  // [2][buf_f]
    short2 *rp = reinterpret_cast<short2 *>(bufs + 2 * S.buf_f);
    int32_t *tp_start = reinterpret_cast<int32_t *>(rp + ls.nrp);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    const int t = threadIdx.x, lane = t & 31;
    for (int i = t; i < 2 * S.buf_f; i += blockDim.x) bufs[i] = 0.0f;
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    for (int j = t; j < ls.nrp; j += blockDim.x) {
        int r1, r2;
        ls.rp_decode(rp_start, j, &r1, &r2);
        rp[j] = make_short2((short)r1, (short)r2);
    }
    __syncthreads();
    const int nrp = (int)ls.nrp;
    const int q = ((t >> 5) << (5 - S.lpg_log)) + (lane >> S.lpg_log),
              strip = lane & ((1 << S.lpg_log) - 1);
    const bool active = q < S.nqg && strip < S.nstrip;
    const int dl0 = q * M - Dm, r0 = strip * K;
    for (int64_t it = blockIdx.x; it < ls.ntp; it += gridDim.x) {
        // pairs in crystal-difference order: concurrent CTAs share the
        // partners' planes and the classes' weights in L2
        int a, b;
        ls.tp_decode_diff(it, &a, &b);
        const int64_t T = tp_index(ls, tp_start, a, b);
        const int a0 = a % ls.Nb;
        const int own_cls = tp_index(ls, tp_start, a0, b - (a - a0));
        float acc[M][K];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[m][k] = 0.0f;
        St3Partner P;
        int dt = st3_next<adjoint>(ls, tp_start, a, b, 0, nwin, Wt, own_cls, P);
        if (dt < nwin) st3_stage<WA>(ls, S, rp, P, Wt, w, in, bufs);
        int cur = 0;
        while (dt < nwin) {
            St3Partner Pn;
            const int nxt = st3_next<adjoint>(ls, tp_start, a, b, dt + 1, nwin, Wt, own_cls, Pn);
            if (nxt < nwin)
                st3_stage<WA>(ls, S, rp, Pn, Wt, w, in, bufs + (cur ^ 1) * S.buf_f);
            else
                cp_async_commit();
            cp_async_wait1();
            __syncthreads();
            if (active) {
                const float *plane = bufs + cur * S.buf_f, *w3 = plane + S.plane_f;
#pragma unroll
                for (int cc = 0; cc < M + 4 * WA; ++cc) {
                    const int c = dl0 - 2 * WA + cc;  // partner column (ring difference)
                    if (c < -Dm || c > Dm) continue;
                    float v[NV];
                    const float2 *pv =
                        reinterpret_cast<const float2 *>(plane + (c + Dm) * PRp + r0);
#pragma unroll
                    for (int u = 0; u < NV / 2; ++u) {
                        const float2 f = pv[u];
                        v[2 * u] = f.x;
                        v[2 * u + 1] = f.y;
                    }
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const int e = adjoint ? m + 2 * WA - cc : cc - 2 * WA - m;
                        if (e < -2 * WA || e > 2 * WA) continue;
                        const int wd = adjoint ? dl0 + m : c;
                        if (adjoint && wd > Dm) continue;
                        const float4 *pw = reinterpret_cast<const float4 *>(
                            w3 + ((wd + Dm) * NE + e + 2 * WA) * 8);
                        const float4 w0 = pw[0], w1 = pw[1];
                        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                        for (int o1 = -WA; o1 <= WA; ++o1) {
                            const int o2 = o1 - e;
                            if (o2 < -WA || o2 > WA) continue;
                            const float wgt = wv[o1 + WA];
#pragma unroll
                            for (int k = 0; k < K; ++k)
                                acc[m][k] =
                                    fmaf(wgt, v[adjoint ? k + o1 + WA : k - o1 + WA], acc[m][k]);
                        }
                    }
                }
            }
            __syncthreads();
            cur ^= 1;
            dt = nxt;
            P = Pn;
        }
        if (active) {
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int ra = r0 + k, dl = dl0 + m, rb = ra + dl;
                    if (ra < NR && dl <= Dm && rb >= 0 && rb < NR)
                        out[T * nrp + rp_start[ra] + (rb - ls.rp_lo(ra))] = acc[m][k];
                }
        }
    }
}

// Fifth form, a warp-specialised pipeline.  A CTA takes transaxial pairs from
// a pair counter (in the crystal-difference order of tp_decode_diff, so that
// the pairs in flight on the whole GPU at any moment share their partners'
// planes and weight slices in L2), and for each pair one producer warp brings
// each partner's data into a ring of S shared-memory stages with two
// cp.async.bulk copies completing on the stage's "full" mbarrier, while the
// consumer warps compute on earlier stages and release each one on its
// "empty" mbarrier -- no CTA-wide barrier per partner.  The input LOR vector
// is first packed into padded ring-pair planes (st5_pack_kernel: [pair][ring
// difference][ring + WA], zero padding), and the class spreads into one
// contiguous slice per (transaxial class, partner offset) (st5_wpad_kernel).
// Partners whose first crystal wraps past the last one (a few per cent of the
// pairs near crystal 0) need the transposed orientation; the producer writes
// those with plain loads and stores.
//
// Consumer tiling: a thread owns M = 4 ring differences x K = 4 rings of the
// pair's (ring difference, ring) plane; only the (difference group, ring
// strip) tiles that hold an in-set ring pair get a thread (92 of the 8 x 13
// tiles of 52 rings with |ra - rb| <= 15: three warps), dealt to threads by
// shared-memory bank group (st5_tile).  A tile's 4 + 2 WA plane rows are read
// with 16-byte loads.
//
// Weight slice layout: for ring difference d and offset e = o1 - o2 of the two
// ends' axial window positions, the run of 2 WA + 1 - |e| weights over o1 =
// max(-WA, e - WA) ... min(WA, e + WA), padded to a multiple of 4 floats; the
// runs of one difference take st5_wrun(WA) floats, at row offset st5_wrow
// (skewed so that the difference groups of one warp read different banks).
//
// Every wait is bounded (the wait limit): a wait that gives up records
// PSF_ETIMEOUT in the status word, the CTA stops, and the producer first waits
// (bounded) for the copies it has in flight.
constexpr int ST5_S = 2;  // stages (2 x 17 KB)

__host__ __device__ constexpr int st5_rlen(int WA, int e) { return 2 * WA + 1 - (e < 0 ? -e : e); }
// offset of run e (e = -2 WA ... 2 WA + 1) within one ring difference's block
__host__ __device__ constexpr int st5_roff(int WA, int e) {
    int o = 0;
    for (int f = -2 * WA; f < e; ++f) o += (st5_rlen(WA, f) + 3) & ~3;
    return o;
}
__host__ __device__ constexpr int st5_wrun(int WA) {
    return st5_roff(WA, 2 * WA + 1) % 8 == 0 ? st5_roff(WA, 2 * WA + 1) + 4
                                             : st5_roff(WA, 2 * WA + 1);
}

// Offset of ring difference row r (0 ... nd - 1) in a weight slice: rows of
// wrun floats with 16 bytes of padding after every 4 rows, so that the rows
// of 8 consecutive consumer groups (4 rows apart, 4 wrun + 4 floats: an odd
// number of 16-byte units) start in 8 different bank groups.
__host__ __device__ constexpr int st5_wrow(int r, int wrun) { return r * wrun + 4 * (r >> 2); }

struct St5Shape {
    int nd, nstrip, nqg;
    int ntask;      // (difference group, ring strip) tiles with an in-set ring pair
    int cthreads;   // consumer threads (ntask rounded up to whole warps)
    int PRp;        // floats per plane column (a multiple of 4, 4 mod 8)
    int wrun;       // floats per ring difference in a weight slice
    int plane_f;    // floats of one packed plane
    int w_f;        // floats of one weight slice
    int stage_f;    // floats of one stage
};

// Ring strips [s0, s1] of difference group g that hold an in-set ring pair:
// rings ra with (ra, ra + d) in the set for some difference d of the group.
__host__ __device__ inline void st5_strips(const LorSet &ls, int g, int *s0, int *s1) {
    const int d0 = g * ST4_M - ls.Dm;
    const int d1 = d0 + ST4_M - 1 < ls.Dm ? d0 + ST4_M - 1 : ls.Dm;
    const int lo = d1 < 0 ? -d1 : 0, hi = ls.NR - 1 - (d0 > 0 ? d0 : 0);
    const int nstrip = (ls.NR + ST4_K - 1) / ST4_K;
    *s0 = lo / ST4_K;
    *s1 = hi / ST4_K < nstrip - 1 ? hi / ST4_K : nstrip - 1;
}

__host__ __device__ inline St5Shape st5_shape(const LorSet &ls, int WA) {
    St5Shape s;
    s.nd = 2 * ls.Dm + 1;
    s.nstrip = (ls.NR + ST4_K - 1) / ST4_K;
    s.nqg = (s.nd + ST4_M - 1) / ST4_M;
    s.ntask = 0;
    for (int g = 0; g < s.nqg; ++g) {
        int s0, s1;
        st5_strips(ls, g, &s0, &s1);
        s.ntask += s1 - s0 + 1;
    }
    s.PRp = (s.nstrip * ST4_K + 2 * WA + 3) / 4 * 4;  // a strip reads 4 + 2 WA rows
    if (s.PRp % 8 == 0) s.PRp += 4;
    s.cthreads = (8 * ((s.ntask + 7) / 8) + 31) / 32 * 32;  // see st5_tile
    s.wrun = st5_wrun(WA);
    s.plane_f = s.nd * s.PRp;
    s.w_f = s.nd * s.wrun + 4 * ((s.nd + 3) / 4);
    s.stage_f = s.plane_f + s.w_f;
    return s;
}

// Consumer thread t's tile (false: none).  A tile's plane reads start at the
// 16-byte unit 4 g P + strip (+ a per-instruction constant) of the stage,
// P = PRp / 4, so tiles of different bank groups b = (4 g P + strip) mod 8
// never share a bank; threads 8 j + b (j < nq = ceil(ntask / 8)) take the
// j-th tile of group b, and the tiles of groups with more than nq take the
// remaining threads in order.  In a warp each bank then holds the plane
// words of 4 threads at most, the 4 wavefronts a 16-byte warp load needs.
__host__ __device__ __noinline__ bool st5_tile(const LorSet &ls, const St5Shape &S5, int t,
                                               int *qg, int *strip) {
    const int nq = (S5.ntask + 7) / 8, P = S5.PRp / 4;
    if (t >= 8 * nq) return false;
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int g = 0; g < S5.nqg; ++g) {
        int s0, s1;
        st5_strips(ls, g, &s0, &s1);
        for (int s = s0; s <= s1; ++s) ++cnt[(4 * g * P + s) & 7];
    }
    const int b = t & 7, j = t >> 3;
    int want_rank = -1, want_extra = -1;
    if (j < cnt[b]) {
        want_rank = j;
    } else {  // a free thread: its index among the free threads
        want_extra = 0;
        for (int u = 0; u < t; ++u)
            if ((u >> 3) >= cnt[u & 7]) ++want_extra;
    }
    int rank[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int extra = 0;
    for (int g = 0; g < S5.nqg; ++g) {
        int s0, s1;
        st5_strips(ls, g, &s0, &s1);
        for (int s = s0; s <= s1; ++s) {
            const int bs = (4 * g * P + s) & 7, r = rank[bs]++;
            if (r < nq ? (bs == b && r == want_rank) : extra++ == want_extra) {
                *qg = g;
                *strip = s;
                return true;
            }
        }
    }
    return false;
}

static size_t stencil5_smem_bytes(const LorSet &ls, int WA) {
    const St5Shape s = st5_shape(ls, WA);
    return sizeof(float) * (size_t)ST5_S * s.stage_f + sizeof(uint64_t) * 3 * ST5_S +
           sizeof(short2) * ls.nrp + sizeof(int32_t) * (ls.Nt + ls.NR + 2 + 16) + 64;
}

// in (set order) -> padded planes: cell (ring difference d, ring ra) of pair T
// at T * plane_f + (d + Dm) * PRp + ra + WA, every other word of the plane 0.
// A CTA per pair: the pair's ring-pair values are read into shared memory
// with coalesced loads, then the whole plane is written with coalesced
// stores (the scattered form ran at 1.1 TB/s).
__global__ void st5_pack_kernel(LorSet ls, int PRp, int plane_f, int WA,
                                const float *__restrict__ in, float *__restrict__ pin) {
    extern __shared__ int32_t pk_pre[];  // tp part (unused), rp_start [NR + 1], values [nrp]
    int32_t *rp_start = pk_pre + ls.Nt + 1;
    float *v = reinterpret_cast<float *>(rp_start + ls.NR + 1);
    ls.stage_prefix(pk_pre, rp_start);
    const int nrp = (int)ls.nrp, Dm = ls.Dm;
    for (int64_t T = blockIdx.x; T < ls.ntp; T += gridDim.x) {
        __syncthreads();  // the previous pair's values are no longer read
        for (int j = threadIdx.x; j < nrp; j += blockDim.x) v[j] = __ldcs(in + T * nrp + j);
        __syncthreads();
        float *dst = pin + T * plane_f;
        for (int i = threadIdx.x; i < plane_f; i += blockDim.x) {
            const int dd = i / PRp, ra = i - dd * PRp - WA, rb = ra + dd - Dm;
            float x = 0.0f;
            if (dd <= 2 * Dm && ra >= 0 && ra < ls.NR && rb >= 0 && rb < ls.NR)
                x = v[rp_start[ra] + (rb - ls.rp_lo(ra))];
            dst[i] = x;
        }
    }
}

// Class spreads -> weight slices: slice (transaxial class ct, partner offset
// dt) holds, per ring difference d and per e = L1 - L2, the run of window
// entries e1 = (dt1 + Wt) W2a + L1, e2 = (dt2 + Wt) W2a + L2 of class (ct, d)
// at st5_wrow(d) + roff(e) + L1 - max(e, 0).  One CTA per class (ct, d): its
// E x E window is read into shared memory with coalesced loads, then each of
// the nwin slices receives its W2a x W2a entries for this d.  The runs'
// padding slots are never read.
__global__ void st5_wpad_kernel(LorSet ls, int Wt, int WA, int wrun, int w_f,
                                const float *__restrict__ w, float *__restrict__ wpad) {
    extern __shared__ float wp_win[];  // [E * E], then the run offsets
    const int W2a = 2 * WA + 1, nd = 2 * ls.Dm + 1;
    const int E = (2 * Wt + 1) * W2a, nwin = (2 * Wt + 1) * (2 * Wt + 1);
    int *roff = reinterpret_cast<int *>(wp_win + E * E);
    if (threadIdx.x <= 4 * WA) roff[threadIdx.x] = st5_roff(WA, (int)threadIdx.x - 2 * WA);
    const int64_t ncls = ls.ntp_cls * nd;
    for (int64_t cl = blockIdx.x; cl < ncls; cl += gridDim.x) {
        __syncthreads();  // the previous class's window is no longer read
        const float *src = w + cl * E * E;
        for (int i = threadIdx.x; i < E * E; i += blockDim.x) wp_win[i] = __ldg(src + i);
        __syncthreads();
        const int64_t ct = cl / nd;
        const int d = (int)(cl - ct * nd);
        const int nv = W2a * W2a;
        for (int i = threadIdx.x; i < nwin * nv; i += blockDim.x) {
            const int dt = i / nv, r = i - dt * nv;
            const int L1 = r / W2a, L2 = r - L1 * W2a, e = L1 - L2;
            wpad[(ct * nwin + dt) * w_f + st5_wrow(d, wrun) + roff[e + 2 * WA] + L1 -
                 (e > 0 ? e : 0)] =
                wp_win[((dt / (2 * Wt + 1)) * W2a + L1) * E + (dt % (2 * Wt + 1)) * W2a + L2];
        }
    }
}

// Bounded wait for a phase in which the waiting thread may sleep: each test
// asks the hardware to suspend it for up to hint_ns nanoseconds before the
// phase completes (so a waiting warp does not take issue slots from the
// computing ones); false after `limit` SM cycles (at once for a negative
// limit).
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity, long long limit,
                                                uint32_t hint_ns) {
    if (limit < 0) return false;
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void mbar_init_n(uint64_t *bar, int n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Global -> shared bulk copy completing on `bar` (L2 default policy: the
// planes and weight slices are re-read by neighbouring pairs).
__device__ __forceinline__ void bulk_g2s_keep(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <bool adjoint, int WA>
__global__ void __launch_bounds__(160, 4) stencil5_kernel(LorSet ls, int Wt,
                                                        const float *__restrict__ w,
                                                        const float *__restrict__ wpad,
                                                        const float *__restrict__ in,
                                                        const float *__restrict__ pin,
                                                        float *__restrict__ out,
                                                        unsigned long long *pair_ctr, int *status,
                                                        long long limit) {
    constexpr int K = ST4_K, M = ST4_M, S = ST5_S, W2a = 2 * WA + 1;
    constexpr int NV4 = (K + 2 * WA + 3) / 4;  // 16-byte plane loads per column
    extern __shared__ __align__(128) unsigned char raw5[];
    const St5Shape S5 = st5_shape(ls, WA);
    constexpr int WR = st5_wrun(WA);
    const int Dm = ls.Dm, NR = ls.NR, PRp = S5.PRp;
    const int nwin = (2 * Wt + 1) * (2 * Wt + 1);
    float *stages = reinterpret_cast<float *>(raw5);  // [S][stage_f]
    uint64_t *full = reinterpret_cast<uint64_t *>(stages + (size_t)S * S5.stage_f);
    uint64_t *empty = full + S;
    // stage header: the output pair's index (-1: no more pairs) and whether
    // the stage holds the pair's last partner
    long long *hdr = reinterpret_cast<long long *>(empty + S);
    short2 *rp = reinterpret_cast<short2 *>(hdr + S);
    int32_t *tp_start = reinterpret_cast<int32_t *>(rp + ls.nrp);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    int *roff = rp_start + ls.NR + 1;  // [4 WA + 2]
    int *abort_flag = roff + 15;
    const int t = threadIdx.x, lane = t & 31;
    const int ncw = S5.cthreads / 32;  // consumer warps
    const bool producer = t >= S5.cthreads;
    for (int i = t; i < S * S5.stage_f; i += blockDim.x) stages[i] = 0.0f;
    ls.stage_prefix(tp_start, rp_start);
    if (t <= 4 * WA) roff[t] = st5_roff(WA, t - 2 * WA);
    if (t == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init_n(full + k, 32);
            mbar_init_n(empty + k, ncw);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    for (int j = t; j < ls.nrp; j += blockDim.x) {
        int r1, r2;
        ls.rp_decode(rp_start, j, &r1, &r2);
        rp[j] = make_short2((short)r1, (short)r2);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // zeroed stages
    __syncthreads();
    const int nrp = (int)ls.nrp;
    volatile int *abort_v = abort_flag;
    long long q = 0;  // stages used so far (producer and consumers count alike)
    if (producer) {
        const uint32_t pbytes = (uint32_t)S5.plane_f * 4u, wbytes = (uint32_t)S5.w_f * 4u;
        bool more = true;
        while (more && !*abort_v) {
            long long it = 0;
            if (lane == 0) it = (long long)atomicAdd(pair_ctr, 1ull);
            it = __shfl_sync(0xffffffffu, it, 0);
            more = it < ls.ntp;
            int a = 0, b = 0, own_cls = 0;
            long long T = -1;
            St3Partner P, Pn;
            int dt = -1;  // the end mark's stage when the queue is exhausted
            if (more) {
                ls.tp_decode_diff(it, &a, &b);
                T = tp_index(ls, tp_start, a, b);
                const int a0 = a % ls.Nb;
                own_cls = tp_index(ls, tp_start, a0, b - (a - a0));
                dt = st3_next<adjoint>(ls, tp_start, a, b, 0, nwin, Wt, own_cls, P);
            }
            while (dt < nwin) {
                const int nxt =
                    more ? st3_next<adjoint>(ls, tp_start, a, b, dt + 1, nwin, Wt, own_cls, Pn)
                         : nwin;
                const int st = (int)(q % S);
                const long long use = q / S;
                bool ok = true;
                if (use > 0) ok = mbar_wait_sleep(empty + st, (uint32_t)((use - 1) & 1), limit, 2000);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok || *abort_v) {
                    if (lane == 0 && !ok) {
                        atomicExch(status, PSF_ETIMEOUT);
                        *abort_v = 1;
                    }
                    more = false;
                    break;
                }
                // header: pair index times 2, plus 1 on the pair's last partner
                if (lane == 0) hdr[st] = more ? 2 * T + (nxt >= nwin ? 1 : 0) : -1;
                if (!more) {  // end mark: no copies
                    mbar_arrive(full + st);
                    ++q;
                    break;
                }
                float *plane = stages + (size_t)st * S5.stage_f, *w3 = plane + S5.plane_f;
                const int64_t psrc = P.prow / nrp;  // the partner pair's index
                const uint32_t tx = (P.sw ? 0u : pbytes) + (P.wsw ? 0u : wbytes);
                if (P.sw || P.wsw) {
                    // transposed orientation: plain loads and stores by the warp
                    if (P.sw)
                        for (int j = lane; j < nrp; j += 32) {
                            const short2 rr = rp[j];
                            plane[(rr.x - rr.y + Dm) * PRp + (rr.y + WA)] = __ldg(in + P.prow + j);
                        }
                    if (P.wsw) {
                        const int E = (2 * Wt + 1) * W2a;
                        const float *wc = w + (int64_t)P.cls * S5.nd * E * E;
                        const int ea0 = (P.dt1 + Wt) * W2a, eb0 = (P.dt2 + Wt) * W2a;
                        for (int i = lane; i < S5.nd * W2a; i += 32) {
                            const int d = i / W2a - Dm, u = i % W2a;  // u = L1
                            const float *s0 = wc + (int64_t)(-d + Dm) * E * E + eb0 * E + ea0 + u;
                            float *d0 = w3 + st5_wrow(d + Dm, WR) + u;
#pragma unroll
                            for (int L2 = 0; L2 < W2a; ++L2) {
                                const int e = u - L2;
                                d0[roff[e + 2 * WA] - (e > 0 ? e : 0)] = __ldg(s0 + L2 * E);
                            }
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                }
                if (lane == 0) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 ::"r"(smem_u32(full + st)), "r"(tx) : "memory");
                    if (!P.sw) bulk_g2s_keep(plane, pin + psrc * S5.plane_f, pbytes, full + st);
                    if (!P.wsw)
                        bulk_g2s_keep(w3, wpad + ((int64_t)P.cls * nwin + dt) * S5.w_f, wbytes,
                                      full + st);
                } else {
                    mbar_arrive(full + st);
                }
                ++q;
                P = Pn;
                dt = nxt;
            }
        }
        // copies still in flight complete before the CTA exits
        if (lane == 0)
            for (long long k = q > S ? q - S : 0; k < q; ++k)
                mbar_wait(full + (int)(k % S), (uint32_t)((k / S) & 1), BK_DRAIN_LIMIT);
        return;
    }
    int qg = 0, strip = 0;
    const bool active = st5_tile(ls, S5, t, &qg, &strip);
    const int dl0 = qg * M - Dm, r0 = strip * K;
    // forward: the weight row of partner column c = dl0 - 2 WA + cc is row
    // 4 qg + cc - 2 WA, at st5_wrow = wq + a constant of cc
    const int wq = qg * (4 * WR + 4);
    // adjoint: the weight row of each owned difference (clamped to the last
    // one for the padding column past Dm, whose sums are never stored)
    int wrow[M];
#pragma unroll
    for (int m = 0; m < M; ++m) wrow[m] = st5_wrow((dl0 + m < Dm ? dl0 + m : Dm) + Dm, WR);
    for (;;) {
        int st = (int)(q % S);
        if (!__all_sync(0xffffffffu,
                        mbar_wait_sleep(full + st, (uint32_t)((q / S) & 1), limit, 200))) {
            if (lane == 0) {
                atomicExch(status, PSF_ETIMEOUT);
                *abort_v = 1;
            }
            return;
        }
        const long long h0 = hdr[st];
        if (h0 < 0) return;  // end mark
        const int64_t T = h0 >> 1;
        float acc[M][K];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[m][k] = 0.0f;
        for (;;) {
            if (active) {
                const float *plane = stages + (size_t)st * S5.stage_f, *w3 = plane + S5.plane_f;
#pragma unroll
                for (int cc = 0; cc < M + 4 * WA; ++cc) {
                    const int c = dl0 - 2 * WA + cc;  // partner column (ring difference)
                    if (c < -Dm || c > Dm) continue;
                    float v[4 * NV4];
                    const float4 *pv =
                        reinterpret_cast<const float4 *>(plane + (c + Dm) * PRp + r0);
#pragma unroll
                    for (int u = 0; u < NV4; ++u) {
                        const float4 f = pv[u];
                        v[4 * u] = f.x;
                        v[4 * u + 1] = f.y;
                        v[4 * u + 2] = f.z;
                        v[4 * u + 3] = f.w;
                    }
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const int e = adjoint ? m + 2 * WA - cc : cc - 2 * WA - m;
                        if (e < -2 * WA || e > 2 * WA) continue;
                        const int n = st5_rlen(WA, e), lo1 = (e - WA > -WA ? e - WA : -WA);
                        const float4 *pw = reinterpret_cast<const float4 *>(
                            w3 + (adjoint ? wrow[m] : wq + st5_wrow(cc - 2 * WA, WR)) +
                            st5_roff(WA, e));
                        float wv[8];
                        const float4 w0 = pw[0];
                        wv[0] = w0.x;
                        wv[1] = w0.y;
                        wv[2] = w0.z;
                        wv[3] = w0.w;
                        if (n > 4) {
                            const float4 w1 = pw[1];
                            wv[4] = w1.x;
                            wv[5] = w1.y;
                            wv[6] = w1.z;
                            wv[7] = w1.w;
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (j >= n) continue;
                            const int o1 = lo1 + j;
                            const float wgt = wv[j];
#pragma unroll
                            for (int k = 0; k < K; ++k)
                                acc[m][k] =
                                    fmaf(wgt, v[adjoint ? k + o1 + WA : k - o1 + WA], acc[m][k]);
                        }
                    }
                }
            }
            const bool last = hdr[st] & 1;
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + st);
            ++q;
            if (last) break;
            st = (int)(q % S);
            const bool ok = __all_sync(
                0xffffffffu, mbar_wait_sleep(full + st, (uint32_t)((q / S) & 1), limit, 200));
            if (!ok || *abort_v) {
                if (lane == 0 && !ok) {
                    atomicExch(status, PSF_ETIMEOUT);
                    *abort_v = 1;
                }
                return;
            }
        }
        if (active) {
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int ra = r0 + k, dl = dl0 + m, rb = ra + dl;
                    if (ra < NR && dl <= Dm && rb >= 0 && rb < NR)
                        out[T * nrp + rp_start[ra] + (rb - ls.rp_lo(ra))] = acc[m][k];
                }
        }
    }
}

// S^T 1 for the sensitivity image A^T 1 = G^T (S^T 1).  With an all-ones
// input the adjoint stencil's value at source LOR g is the sum of g's window
// weights over the window entries whose measured LOR is in the set:
//   q[g] = sum_{partner dt in set} sum_{(o1,o2): target rings in set}
//          W_{class(g)}[d][(dt1,o1)][(dt2,o2)],   d = g's ring difference.
// The partner sums C[d][o1][o2] = sum_{dt in set} W[...] are formed once per
// class (their partners in the set are the same for every pair of the class),
// then each ring pair adds the C entries of its in-set targets (all of them,
// one precomputed sum per d, away from the ends of the rings and the largest
// ring differences): 31 x 49 x 49 per class + 1372 x 49 additions per pair at
// most, instead of the stencil's 1372 x 2401 products.
constexpr int SS_T = 128;

// Offset (floats, even) of the class partner masks after the class sums.
__host__ __device__ __forceinline__ int64_t sens_mask_off(int64_t ncls, int nsum) {
    return (ncls * nsum + 1) & ~int64_t(1);
}

// Partners of transaxial pair (a, b) in the set, one bit per window offset
// pair, into mask[2] (zeroed by the caller, then a CTA barrier); threads
// t < nwin take one offset each.  Membership depends only on the crystal
// difference b - a (the fan is symmetric under b - a -> Nt - (b - a)), so all
// pairs of a class share their mask.
__device__ __forceinline__ void sens_partner_mask(const LorSet &ls, const int32_t *tp_start,
                                                  int a, int b, int Wt, int nwin,
                                                  unsigned long long *mask) {
    const int dt = threadIdx.x;
    if (dt >= nwin) return;
    int pa = a + dt / (2 * Wt + 1) - Wt, pb = b + dt % (2 * Wt + 1) - Wt;
    pa += pa < 0 ? ls.Nt : (pa >= ls.Nt ? -ls.Nt : 0);
    pb += pb < 0 ? ls.Nt : (pb >= ls.Nt ? -ls.Nt : 0);
    if (pa != pb && tp_member(ls, pa < pb ? pa : pb, pa < pb ? pb : pa))
        atomicOr(mask + (dt >> 6), 1ull << (dt & 63));
}

// Per spread class c: C_c[d][o1][o2] summed over the class's transaxial
// partners in the set (the partner sums of every pair of the class).
__global__ void __launch_bounds__(SS_T) sens_class_kernel(LorSet ls, int Wt, int Wa,
                                                          const float *__restrict__ w,
                                                          float *__restrict__ csum) {
    extern __shared__ __align__(16) unsigned char sc_raw[];
    unsigned long long *mask = reinterpret_cast<unsigned long long *>(sc_raw);
    int32_t *tp_start = reinterpret_cast<int32_t *>(mask + 2);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a, nd = 2 * ls.Dm + 1;
    const int nwin = (2 * Wt + 1) * (2 * Wt + 1), nsum = nd * W2a * W2a;
    ls.stage_prefix(tp_start, rp_start);
    for (int64_t c = blockIdx.x; c < ls.ntp_cls; c += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < 2) mask[threadIdx.x] = 0ull;
        __syncthreads();
        int a0, b0;
        ls.tp_decode(tp_start, c, &a0, &b0);
        sens_partner_mask(ls, tp_start, a0, b0, Wt, nwin, mask);
        __syncthreads();
        const unsigned long long m0 = mask[0], m1 = mask[1];
        if (threadIdx.x < 2)
            reinterpret_cast<unsigned long long *>(csum + sens_mask_off(ls.ntp_cls, nsum))
                [2 * c + threadIdx.x] = mask[threadIdx.x];
        const float *wc = w + c * nd * E * E;
        const bool all = __popcll(m0) + __popcll(m1) == nwin;
        for (int i = threadIdx.x; i < nsum; i += SS_T) {
            const int d = i / (W2a * W2a), L1 = (i / W2a) % W2a, L2 = i % W2a;
            const float *wd = wc + (int64_t)d * E * E + L1 * E + L2;
            float acc = 0.0f;
            if (all) {
                for (int dt = 0; dt < nwin; ++dt) {
                    const int dt1 = dt / (2 * Wt + 1), dt2 = dt % (2 * Wt + 1);
                    acc += __ldg(wd + dt1 * W2a * E + dt2 * W2a);
                }
            } else {
                for (int dt = 0; dt < nwin; ++dt) {
                    if (!(((dt < 64 ? m0 >> dt : m1 >> (dt - 64)) & 1ull))) continue;
                    const int dt1 = dt / (2 * Wt + 1), dt2 = dt % (2 * Wt + 1);
                    acc += __ldg(wd + dt1 * W2a * E + dt2 * W2a);
                }
            }
            csum[c * nsum + i] = acc;
        }
    }
}

__global__ void __launch_bounds__(SS_T) sens_spread_kernel(LorSet ls, int Wt, int Wa,
                                                           const float *__restrict__ w,
                                                           const float *__restrict__ csum,
                                                           float *__restrict__ q) {
    extern __shared__ __align__(16) unsigned char raw[];
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a, nd = 2 * ls.Dm + 1;
    const int nwin = (2 * Wt + 1) * (2 * Wt + 1), NR = ls.NR, Dm = ls.Dm;
    const int nsum = nd * W2a * W2a;
    float *C = reinterpret_cast<float *>(raw);                     // [nd][W2a][W2a]
    float *Ct = C + nd * W2a * W2a;                                // [nd] sums of C[d]
    short2 *rp = reinterpret_cast<short2 *>(Ct + nd);              // [nrp]
    int32_t *tp_start = reinterpret_cast<int32_t *>(rp + ls.nrp);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    unsigned long long *mask = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(rp_start + ls.NR + 1) + 7) & ~uintptr_t(7));
    const int t = threadIdx.x;
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    for (int j = t; j < ls.nrp; j += SS_T) {
        int r1, r2;
        ls.rp_decode(rp_start, j, &r1, &r2);
        rp[j] = make_short2((short)r1, (short)r2);
    }
    const int nrp = (int)ls.nrp;
    for (int64_t T = blockIdx.x; T < ls.ntp; T += gridDim.x) {
        __syncthreads();
        int a, b;
        ls.tp_decode(tp_start, T, &a, &b);
        if (t < 4) mask[t] = 0ull;
        __syncthreads();
        const int a0 = a % ls.Nb;
        const int64_t cls = tp_index(ls, tp_start, a0, b - (a - a0));
        sens_partner_mask(ls, tp_start, a, b, Wt, nwin, mask);
        __syncthreads();
        const unsigned long long m0 = mask[0], m1 = mask[1];
        const unsigned long long *cmask =
            reinterpret_cast<const unsigned long long *>(csum + sens_mask_off(ls.ntp_cls, nsum)) +
            2 * cls;
        if (m0 == cmask[0] && m1 == cmask[1]) {
            // the class's partners: its sums (the same additions in the same
            // order)
            for (int i = t; i < nsum; i += SS_T) C[i] = __ldg(csum + cls * nsum + i);
        } else {
            const float *wc = w + cls * nd * E * E;
            for (int i = t; i < nsum; i += SS_T) {
                const int d = i / (W2a * W2a), L1 = (i / W2a) % W2a, L2 = i % W2a;
                const float *wd = wc + (int64_t)d * E * E + L1 * E + L2;
                float acc = 0.0f;
                for (int dt = 0; dt < nwin; ++dt) {
                    if (!(((dt < 64 ? m0 >> dt : m1 >> (dt - 64)) & 1ull))) continue;
                    const int dt1 = dt / (2 * Wt + 1), dt2 = dt % (2 * Wt + 1);
                    acc += __ldg(wd + dt1 * W2a * E + dt2 * W2a);
                }
                C[i] = acc;
            }
        }
        __syncthreads();
        for (int d = t; d < nd; d += SS_T) {  // whole-window sums, in the loop's order
            const float *Cd = C + d * W2a * W2a;
            float acc = 0.0f;
            for (int i = 0; i < W2a * W2a; ++i) acc += Cd[i];
            Ct[d] = acc;
        }
        __syncthreads();
        for (int j = t; j < nrp; j += SS_T) {
            const short2 rr = rp[j];
            const int ra = rr.x, rb = rr.y, d = rb - ra;
            if (ra >= Wa && ra + Wa < NR && rb >= Wa && rb + Wa < NR &&
                (d < 0 ? -d : d) + 2 * Wa <= Dm) {  // every target in the set
                q[T * nrp + j] = Ct[d + Dm];
                continue;
            }
            const float *Cd = C + (d + Dm) * W2a * W2a;
            float acc = 0.0f;
            for (int L1 = 0; L1 < W2a; ++L1) {
                const int ta = ra + L1 - Wa;
                if (ta < 0 || ta >= NR) continue;
                for (int L2 = 0; L2 < W2a; ++L2) {
                    const int tb = rb + L2 - Wa;
                    if (tb < 0 || tb >= NR || tb - ta > Dm || ta - tb > Dm) continue;
                    acc += Cd[L1 * W2a + L2];
                }
            }
            q[T * nrp + j] = acc;
        }
    }
}

// Top-N spreads (psf_matrix_set_spread_topn): S and S^T with each class's
// kept window entries as sparse taps.  Forward: every source LOR g adds
// w_k p[g] to the measured LOR that kept entry k of its class lands on
// (several sources meet in one target: FP32 atomics, so the order of the
// additions, and the last bits of a sum, vary between runs); adjoint:
// q[g] = sum_k w_k r[m_k], a gather in rank order (in == NULL: r = 1, the
// sensitivity's S^T 1, with no reads).  A window entry lands on
// the crystal pair (a + dt1, ra + da1), (b + dt2, rb + da2), transaxial
// indices wrapping around the ring; pairs outside the set, off the rings or
// of one crystal with itself are dropped, as in the dense stencil.
//
// The same pass over the taps also builds the transpose of S (the sources of
// every measured LOR, psf_matrix_build_sparse_adjoint): TS_COUNT counts each
// target's sources, TS_FILL writes (source, weight) into the target's list at
// a slot taken from a per-target cursor (the order inside a list depends on
// the atomics).  With it, S^T of an input with at most 1/16 nonzero entries
// is a scatter from those entries; the gather then returns at once.
constexpr int TS_T = 256, TS_G = 8;
enum { TS_FWD = 0, TS_ADJ = 1, TS_COUNT = 2, TS_FILL = 3 };

struct TsTr {
    unsigned long long *cnt;      // TS_COUNT: [n] sources per target
    const int64_t *ptr;           // TS_FILL: [n + 1] list offsets
    int32_t *cur;                 // TS_FILL: [n] cursors (zeroed)
    int32_t *src;                 // TS_FILL: sources
    float *w;                     // TS_FILL: weights
    const unsigned long long *nz;  // TS_ADJ: nonzero input count (NULL: always gather)
};

__host__ __device__ inline bool ts_sparse(unsigned long long nz, int64_t n) {
    return nz <= (unsigned long long)(n >> 4);
}

template <int MODE>
__global__ void __launch_bounds__(TS_T, 4) topn_s_kernel(LorSet ls, int Wt, int Wa, int N,
                                                      const int32_t *__restrict__ tidx,
                                                      const float *__restrict__ tw,
                                                      const __nv_bfloat16 *__restrict__ twh,
                                                      const float *__restrict__ tsc,
                                                      const float *__restrict__ in,
                                                      float *__restrict__ out, TsTr tr) {
    constexpr bool adjoint = MODE == TS_ADJ;
    extern __shared__ __align__(16) unsigned char raw[];
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a, Nt = ls.Nt, NR = ls.NR;
    char4 *dec = reinterpret_cast<char4 *>(raw);  // [E*E] window index -> (dt1, da1, dt2, da2)
    int32_t *tp_start = reinterpret_cast<int32_t *>(dec + E * E);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    short2 *rp = reinterpret_cast<short2 *>(rp_start + ls.NR + 1);
    const int t = threadIdx.x;
    for (int e = t; e < E * E; e += TS_T) {
        const int e1 = e / E, e2 = e - e1 * E;
        dec[e] = make_char4((signed char)(e1 / W2a - Wt), (signed char)(e1 % W2a - Wa),
                            (signed char)(e2 / W2a - Wt), (signed char)(e2 % W2a - Wa));
    }
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    for (int j = t; j < ls.nrp; j += TS_T) {
        int r1, r2;
        ls.rp_decode(rp_start, j, &r1, &r2);
        rp[j] = make_short2((short)r1, (short)r2);
    }
    __syncthreads();
    const int64_t n = ls.ntp * ls.nrp;
    if (adjoint && tr.nz && ts_sparse(*tr.nz, n)) return;  // the scatter has it
    for (int64_t g = (int64_t)blockIdx.x * TS_T + t; g < n; g += (int64_t)gridDim.x * TS_T) {
        const int64_t T = g / ls.nrp;
        const int j = (int)(g - T * ls.nrp);
        float pg = 0.0f;
        if (MODE == TS_FWD) {
            pg = in[g];
            if (pg == 0.0f) continue;
        }
        int a, b;
        ls.tp_decode(tp_start, T, &a, &b);
        const short2 r2 = rp[j];
        const int ra = r2.x, rb = r2.y;
        const int64_t cls = ls.class_of(tp_start, a, b, ra, rb);
        const int32_t *ik = tidx + cls * N;
        const float *wk = tw ? tw + cls * N : nullptr;
        const __nv_bfloat16 *wh = twh ? twh + cls * N : nullptr;
        const float wsc = twh ? __ldg(tsc + cls) : 1.0f;
        float acc = 0.0f;
        // taps in groups of TS_G: the targets first, then their reads or
        // atomics, so a group's memory operations are in flight together
        for (int k0 = 0; k0 < N; k0 += TS_G) {
            int64_t m[TS_G];
            float wv[TS_G];
#pragma unroll
            for (int u = 0; u < TS_G; ++u) {
                m[u] = -1;
                wv[u] = 0.0f;
                const int k = k0 + u;
                if (k >= N) continue;
                const float w = wh ? __bfloat162float(wh[k]) * wsc : __ldg(wk + k);
                if (w == 0.0f) continue;
                const char4 o = dec[__ldg(ik + k)];
                const int qa = ra + o.y, qb = rb + o.w;
                if (qa < 0 || qa >= NR || qb < 0 || qb >= NR) continue;
                int pa = a + o.x, pb = b + o.z;
                pa += pa < 0 ? Nt : (pa >= Nt ? -Nt : 0);
                pb += pb < 0 ? Nt : (pb >= Nt ? -Nt : 0);
                const bool sw = pa > pb;
                const int A = sw ? pb : pa, B = sw ? pa : pb, RA = sw ? qb : qa, RB = sw ? qa : qb;
                if (!ls.member(A, B, RA, RB)) continue;
                m[u] = ls.row_of(tp_start, rp_start, A, B, RA, RB);
                wv[u] = w;
            }
            if (adjoint) {
                float v[TS_G];
#pragma unroll
                for (int u = 0; u < TS_G; ++u)
                    v[u] = m[u] >= 0 ? (in ? __ldg(in + m[u]) : 1.0f) : 0.0f;
#pragma unroll
                for (int u = 0; u < TS_G; ++u) acc = fmaf(wv[u], v[u], acc);
            } else if (MODE == TS_FWD) {
#pragma unroll
                for (int u = 0; u < TS_G; ++u)
                    if (m[u] >= 0) atomicAdd(out + m[u], wv[u] * pg);
            } else if (MODE == TS_COUNT) {
#pragma unroll
                for (int u = 0; u < TS_G; ++u)
                    if (m[u] >= 0) atomicAdd(tr.cnt + m[u], 1ull);
            } else {
#pragma unroll
                for (int u = 0; u < TS_G; ++u)
                    if (m[u] >= 0) {
                        const int64_t e = tr.ptr[m[u]] + atomicAdd(tr.cur + m[u], 1);
                        tr.src[e] = (int32_t)g;
                        tr.w[e] = wv[u];
                    }
            }
        }
        if (adjoint) out[g] = acc;
    }
}

// S^T of a sparse input through the transpose: out = 0, then every listed
// nonzero input entry adds w * in[m] to each of its sources.  Both kernels
// return at once when the input is not sparse (the gather runs instead).
__global__ void ts_zero_kernel(float *__restrict__ out, int64_t n,
                               const unsigned long long *nz) {
    if (!ts_sparse(*nz, n)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = 0.0f;
}

__global__ void ts_scatter_kernel(const int32_t *__restrict__ list, const unsigned long long *nz,
                                  int64_t n, const int64_t *__restrict__ ptr,
                                  const int32_t *__restrict__ src, const float *__restrict__ w,
                                  const float *__restrict__ in, float *__restrict__ out) {
    const unsigned long long cnt = *nz;
    if (!ts_sparse(cnt, n)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t mm = list[i];
        const float v = in[mm];
        for (int64_t e = ptr[mm]; e < ptr[mm + 1]; ++e) atomicAdd(out + src[e], w[e] * v);
    }
}

static int topn_s(const psf_matrix *m, const float *in, float *out, bool adjoint,
                  cudaStream_t st) {
    const size_t shm = sizeof(char4) * (size_t)m->E * m->E + sizeof(int32_t) * (m->ls.Nt + m->ls.NR + 2) +
                       sizeof(short2) * m->ls.nrp + 16;
    if (shm > 200 * 1024) return PSF_EINVAL;
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t n = m->ls.ntp * m->ls.nrp;
    const int64_t need = (n + TS_T - 1) / TS_T;
    const int grid = (int)(need < (int64_t)sms * 8 ? need : (int64_t)sms * 8);
    if (adjoint) {
        TsTr tr{};
        if (in && m->tr_ptr) {  // sparse inputs through the transpose
            PSF_TRY(cudaMemsetAsync(m->tr_nz, 0, sizeof(unsigned long long), st));
            list_nonzero(in, n, m->tr_list, m->tr_nz, st);
            PSF_LAUNCHED();
            {
                PSF_TIMED("ts_zero_kernel", st);
                ts_zero_kernel<<<grid_for(n, 256), 256, 0, st>>>(out, n, m->tr_nz);
            }
            PSF_LAUNCHED();
            {
                PSF_TIMED("ts_scatter_kernel", st);
                ts_scatter_kernel<<<grid_for(n >> 4, 256), 256, 0, st>>>(
                    m->tr_list, m->tr_nz, n, m->tr_ptr, m->tr_src, m->tr_w, in, out);
            }
            PSF_LAUNCHED();
            tr.nz = m->tr_nz;
        }
        PSF_TRY(cudaFuncSetAttribute(topn_s_kernel<TS_ADJ>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        PSF_TIMED("topn_s_kernel<adjoint>", st);
        topn_s_kernel<TS_ADJ><<<grid, TS_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->topn, m->tidx,
                                                        m->tw, m->twh, m->tsc, in, out, tr);
    } else {
        PSF_TRY(cudaMemsetAsync(out, 0, sizeof(float) * n, st));
        PSF_TRY(cudaFuncSetAttribute(topn_s_kernel<TS_FWD>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        PSF_TIMED("topn_s_kernel<forward>", st);
        topn_s_kernel<TS_FWD><<<grid, TS_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->topn, m->tidx,
                                                        m->tw, m->twh, m->tsc, in, out, TsTr{});
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

static size_t sens_smem_bytes(const LorSet &ls, int Wa) {
    const int W2a = 2 * Wa + 1, nd = 2 * ls.Dm + 1;
    return sizeof(float) * (nd * W2a * W2a + nd) + sizeof(short2) * ls.nrp +
           sizeof(int32_t) * (ls.Nt + ls.NR + 2) + 8 + 4 * sizeof(unsigned long long) + 16;
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

// Resident CTAs of a work-queue kernel at `threads` per CTA (whole grid).
template <typename K>
static int wq_grid(K kernel, int threads, int *grid) {
    int dev = 0, sms = 148, per_sm = 0;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PSF_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0));
    *grid = sms * (per_sm > 0 ? per_sm : 1);
    return PSF_OK;
}

// Grid and shared memory of the bulk-staged kernels: the resident CTAs.
template <typename K>
static int bk_launch_shape(K kernel, int64_t nch, int *grid, size_t *shm) {
    *shm = (sizeof(int32_t) + sizeof(float)) * 2 * BK_CAP + 2 * sizeof(uint64_t);
    PSF_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*shm));
    int dev = 0, sms = 148, per_sm = 0;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PSF_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, BK_T, *shm));
    const int64_t g = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    *grid = (int)(nch < g ? nch : g);
    return PSF_OK;
}

// The chunk table of the bulk-staged forms (FP32 rows, 16-byte aligned
// column and value arrays, at least one entry); PSF_EINVAL when they do not
// apply.  Synchronises on the first call.
static int bk_table(psf_matrix *m, cudaStream_t st) {
    if (m->bk_first) return PSF_OK;
    if (m->dtype != PSF_F32 || m->n_rows == 0) return PSF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(m->col) & 15) || (reinterpret_cast<uintptr_t>(m->val) & 15))
        return PSF_EINVAL;
    int64_t nnz = 0;
    PSF_TRY(cudaMemcpyAsync(&nnz, m->row_ptr + m->n_rows, sizeof(int64_t), cudaMemcpyDeviceToHost,
                            st));
    PSF_TRY(cudaStreamSynchronize(st));
    if (nnz <= 0) return PSF_EINVAL;
    const int64_t nch = (nnz + BK_CAP - 1) / BK_CAP;
    int64_t *fr = nullptr;
    PSF_TRY(cudaMalloc(&fr, sizeof(int64_t) * nch));
    {
        PSF_TIMED("bk_first_row_kernel", st);
        bk_first_row_kernel<<<(int)((nch + 255) / 256), 256, 0, st>>>(m->row_ptr, m->n_rows, nch,
                                                                      fr);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        cudaFree(fr);
        return PSF_ECUDA;
    }
    m->bk_first = fr;
    m->bk_nch = nch;
    m->bk_nnz = nnz;
    return PSF_OK;
}

static int rows_fwd_with(const psf_matrix *m, const float *x, float *y, int chunk, int threads,
                         cudaStream_t st) {
    if (chunk == -2) {  // bulk-staged chunks
        if (!m->bk_first) return PSF_EINVAL;
        int grid = 0;
        size_t shm = 0;
        int rc = bk_launch_shape(csr_fwd_bulk_kernel, m->bk_nch, &grid, &shm);
        if (rc) return rc;
        {
            PSF_TIMED("csr_fwd_bulk_kernel", st);
            csr_fwd_bulk_kernel<<<grid, BK_T, shm, st>>>(m->n_rows, m->bk_nnz, m->bk_nch,
                                                         m->bk_first, m->row_ptr, m->col,
                                                         (const float *)m->val, x, y, m->status,
                                                         (long long)wait_limit());
        }
        PSF_LAUNCHED();
        return PSF_OK;
    }
    if (chunk < 0) {  // streaming tiles (FP32 rows without a scale)
        if (m->dtype != PSF_F32) return PSF_EINVAL;
        int dev = 0, sms = 148;
        PSF_TRY(cudaGetDevice(&dev));
        PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int64_t ntile = (m->n_rows + CS_ROWS - 1) / CS_ROWS;
        const int grid = (int)(ntile < (int64_t)sms * 8 ? ntile : (int64_t)sms * 8);
        {
            PSF_TIMED("csr_fwd_stream_kernel", st);
            csr_fwd_stream_kernel<<<grid, CS_T, 0, st>>>(m->n_rows, m->row_ptr, m->col,
                                                         (const float *)m->val, x, y);
        }
        PSF_LAUNCHED();
        return PSF_OK;
    }
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        if (chunk > 0) {
            int grid = 0;
            int rc = wq_grid(csr_fwd_wq_kernel<VT>, threads, &grid);
            if (rc) return rc;
            PSF_TRY(cudaMemsetAsync(m->queue, 0, sizeof(unsigned long long), st));
            {
                PSF_TIMED("csr_fwd_wq_kernel", st);
                csr_fwd_wq_kernel<VT><<<grid, threads, 0, st>>>(
                    m->n_rows, m->row_ptr, m->col, (const VT *)m->val, m->row_scale, x, y,
                    m->queue, chunk);
            }
        } else {
            const int grid = grid_for(m->n_rows * 32, PJ_T);
            PSF_TIMED("csr_fwd_kernel", st);
            csr_fwd_kernel<VT><<<grid, PJ_T, 0, st>>>(m->n_rows, m->row_ptr, m->col,
                                                       (const VT *)m->val, m->row_scale, x, y);
        }
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

static int rows_back_with(const psf_matrix *m, const float *y, float *x, int chunk, int threads,
                          cudaStream_t st) {
    PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
    if (chunk == -2) {  // bulk-staged chunks
        if (!m->bk_first) return PSF_EINVAL;
        int grid = 0;
        size_t shm = 0;
        int rc = bk_launch_shape(csr_back_bulk_kernel<false>, m->bk_nch, &grid, &shm);
        if (rc) return rc;
        {
            PSF_TIMED("csr_back_bulk_kernel", st);
            csr_back_bulk_kernel<false><<<grid, BK_T, shm, st>>>(
                m->n_rows, m->bk_nnz, m->bk_nch, m->bk_first, m->row_ptr, m->col,
                (const float *)m->val, y, nullptr, x, nullptr, m->status,
                (long long)wait_limit());
        }
        PSF_LAUNCHED();
        return PSF_OK;
    }
    if (chunk < 0) chunk = 0;  // the streaming form is forward only
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        if (chunk > 0) {
            int grid = 0;
            int rc = wq_grid(csr_back_wq_kernel<VT>, threads, &grid);
            if (rc) return rc;
            PSF_TRY(cudaMemsetAsync(m->queue + 1, 0, sizeof(unsigned long long), st));
            {
                PSF_TIMED("csr_back_wq_kernel", st);
                csr_back_wq_kernel<VT><<<grid, threads, 0, st>>>(
                    m->n_rows, m->row_ptr, m->col, (const VT *)m->val, m->row_scale, y, x,
                    m->queue + 1, chunk);
            }
        } else {
            const int grid = grid_for(m->n_rows * 32, PJ_T);
            PSF_TIMED("csr_back_kernel", st);
            csr_back_kernel<VT><<<grid, PJ_T, 0, st>>>(m->n_rows, m->row_ptr, m->col,
                                                        (const VT *)m->val, m->row_scale, y, x);
        }
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

static int rows_fwd(const psf_matrix *m, const float *x, float *y, cudaStream_t st) {
    if (m->otf)
        return otf_rows_fwd(m->otf_sc, m->otf_im, m->otf_ls, nullptr, nullptr, x, y, m->status,
                            st);
    return rows_fwd_with(m, x, y, m->fwd_chunk, m->fwd_threads, st);
}

static int rows_back(const psf_matrix *m, const float *y, float *x, cudaStream_t st) {
    if (m->otf) {
        PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
        return otf_rows_back(m->otf_sc, m->otf_im, m->otf_ls, nullptr, nullptr, y, x, m->status,
                             st);
    }
    return rows_back_with(m, y, x, m->wq_chunk, m->wq_threads, st);
}

static int rows_back_pair(const psf_matrix *m, const float *qa, const float *qb, int form,
                          cudaStream_t st);

// S (adjoint == false) or S^T on LOR-space vectors of a factored plan.
template <bool adjoint, int WA>
static int launch_stencil2(const psf_matrix *m, const float *in, float *out, int grid,
                           cudaStream_t st) {
    const size_t shm = stencil2_smem_bytes(m->ls, WA);
    PSF_TRY(cudaFuncSetAttribute(stencil2_kernel<adjoint, WA, ST2_K>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    {
        PSF_TIMED(adjoint ? "stencil2_kernel<adjoint>" : "stencil2_kernel<forward>", st);
        stencil2_kernel<adjoint, WA, ST2_K><<<grid, ST_T, shm, st>>>(m->ls, m->Wt, m->cls, in, out);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

template <bool adjoint, int WA>
static int launch_stencil4(const psf_matrix *m, const float *in, float *out, cudaStream_t st) {
    const St4Shape s4 = st4_shape(m->ls, WA);
    const size_t shm = stencil4_smem_bytes(m->ls, WA);
    PSF_TRY(cudaFuncSetAttribute(stencil4_kernel<adjoint, WA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    int dev = 0, sms = 148, per_sm = 0;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PSF_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stencil4_kernel<adjoint, WA>,
                                                          s4.threads, shm));
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(m->ls.ntp < cap ? m->ls.ntp : cap);
    {
        PSF_TIMED(adjoint ? "stencil4_kernel<adjoint>" : "stencil4_kernel<forward>", st);
        stencil4_kernel<adjoint, WA><<<grid, s4.threads, shm, st>>>(m->ls, m->Wt, m->cls, in,
                                                                    out);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

template <bool adjoint, int WA>
static int launch_stencil3(const psf_matrix *m, const float *in, float *out, int grid,
                           cudaStream_t st) {
    const size_t shm = stencil3_smem_bytes(m->ls, WA);
    PSF_TRY(cudaFuncSetAttribute(stencil3_kernel<adjoint, WA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    {
        PSF_TIMED(adjoint ? "stencil3_kernel<adjoint>" : "stencil3_kernel<forward>", st);
        stencil3_kernel<adjoint, WA><<<grid, ST3_T, shm, st>>>(m->ls, m->Wt, m->cls, in, out);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

static bool stencil4_ok(const LorSet &ls, int Wa);

static bool stencil5_ok(const LorSet &ls, int Wt, int Wa) {
    const St5Shape s5 = st5_shape(ls, Wa);
    const int64_t E = (2 * (int64_t)Wt + 1) * (2 * Wa + 1);
    return stencil4_ok(ls, Wa) && s5.cthreads <= 128 &&
           stencil5_smem_bytes(ls, Wa) <= 72 * 1024 && E * E * 4 <= 48 * 1024;
}

// Form 5: pack the input into planes, re-lay the class spreads out if they
// changed since psf_matrix_set_spread, then the pipelined stencil.
template <bool adjoint, int WA>
static int launch_stencil5(const psf_matrix *mc, const float *in, float *out, cudaStream_t st) {
    psf_matrix *m = const_cast<psf_matrix *>(mc);  // the plan's own scratch
    const St5Shape s5 = st5_shape(m->ls, WA);
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (m->wpad_dirty) {
        PSF_TIMED("st5_wpad_kernel", st);
        st5_wpad_kernel<<<sms * 8, 256, sizeof(float) * m->E * m->E + 16 * sizeof(int), st>>>(
            m->ls, m->Wt, WA, s5.wrun, s5.w_f, m->cls, m->wpad);
        m->wpad_dirty = false;
    }
    PSF_LAUNCHED();
    {
        PSF_TIMED("st5_pack_kernel", st);
        st5_pack_kernel<<<sms * 8, 256,
                          sizeof(int32_t) * (m->ls.Nt + m->ls.NR + 2) + sizeof(float) * m->ls.nrp,
                          st>>>(m->ls, s5.PRp, s5.plane_f, WA, in, m->pin);
    }
    PSF_LAUNCHED();
    const size_t shm = stencil5_smem_bytes(m->ls, WA);
    PSF_TRY(cudaFuncSetAttribute(stencil5_kernel<adjoint, WA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    int per_sm = 0;
    PSF_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stencil5_kernel<adjoint, WA>,
                                                          s5.cthreads + 32, shm));
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(m->ls.ntp < cap ? m->ls.ntp : cap);
    PSF_TRY(cudaMemsetAsync(m->queue + 3, 0, sizeof(unsigned long long), st));  // pair counter
    {
        PSF_TIMED(adjoint ? "stencil5_kernel<adjoint>" : "stencil5_kernel<forward>", st);
        stencil5_kernel<adjoint, WA><<<grid, s5.cthreads + 32, shm, st>>>(
            m->ls, m->Wt, m->cls, m->wpad, in, m->pin, out, m->queue + 3, m->status,
            (long long)wait_limit());
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

static bool stencil4_ok(const LorSet &ls, int Wa) {
    const St4Shape s4 = st4_shape(ls, Wa);
    return Wa <= 3 && s4.nstrip <= 32 && s4.threads <= 256 &&
           stencil4_smem_bytes(ls, Wa) <= 110 * 1024;
}

// The plain and register-blocked stencil forms: one CTA holds all ring pairs of
// a transaxial pair.
static bool plain_stencil_ok(const LorSet &ls, int Wa) {
    return ls.nrp <= ST_T * ST_OUT && stencil_smem_bytes(ls, Wa) <= 200 * 1024 &&
           stencil2_smem_bytes(ls, Wa) <= 200 * 1024;
}

static bool stencil3_ok(const LorSet &ls, int Wa) {
    const St3Shape s3 = st3_shape(ls, Wa);
    return Wa <= 3 && s3.items <= ST3_T && stencil3_smem_bytes(ls, Wa) <= 110 * 1024;
}

static int stencil(const psf_matrix *m, const float *in, float *out, bool adjoint,
                   cudaStream_t st) {
    if (m->topn > 0) return topn_s(m, in, out, adjoint, st);
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int form = m->st_form[adjoint ? 1 : 0];
    if (form == 5 && m->wpad && m->pin && stencil5_ok(m->ls, m->Wt, m->Wa)) {
        switch (m->Wa * 2 + (adjoint ? 1 : 0)) {
            case 0: return launch_stencil5<false, 0>(m, in, out, st);
            case 1: return launch_stencil5<true, 0>(m, in, out, st);
            case 2: return launch_stencil5<false, 1>(m, in, out, st);
            case 3: return launch_stencil5<true, 1>(m, in, out, st);
            case 4: return launch_stencil5<false, 2>(m, in, out, st);
            case 5: return launch_stencil5<true, 2>(m, in, out, st);
            case 6: return launch_stencil5<false, 3>(m, in, out, st);
            case 7: return launch_stencil5<true, 3>(m, in, out, st);
            default: break;
        }
    }
    const bool ok4 = stencil4_ok(m->ls, m->Wa), ok3 = stencil3_ok(m->ls, m->Wa);
    const bool use4 = form != 1 && form != 2 && ok4 && (form != 3 || !ok3);
    const bool use3 = form != 1 && form != 2 && !use4 && ok3;
    if (use4) {
        switch (m->Wa * 2 + (adjoint ? 1 : 0)) {
            case 0: return launch_stencil4<false, 0>(m, in, out, st);
            case 1: return launch_stencil4<true, 0>(m, in, out, st);
            case 2: return launch_stencil4<false, 1>(m, in, out, st);
            case 3: return launch_stencil4<true, 1>(m, in, out, st);
            case 4: return launch_stencil4<false, 2>(m, in, out, st);
            case 5: return launch_stencil4<true, 2>(m, in, out, st);
            case 6: return launch_stencil4<false, 3>(m, in, out, st);
            case 7: return launch_stencil4<true, 3>(m, in, out, st);
            default: break;
        }
    }
    if (use3) {
        const int64_t g3 = m->ls.ntp < (int64_t)sms * 4 ? m->ls.ntp : (int64_t)sms * 4;
        switch (m->Wa * 2 + (adjoint ? 1 : 0)) {
            case 0: return launch_stencil3<false, 0>(m, in, out, (int)g3, st);
            case 1: return launch_stencil3<true, 0>(m, in, out, (int)g3, st);
            case 2: return launch_stencil3<false, 1>(m, in, out, (int)g3, st);
            case 3: return launch_stencil3<true, 1>(m, in, out, (int)g3, st);
            case 4: return launch_stencil3<false, 2>(m, in, out, (int)g3, st);
            case 5: return launch_stencil3<true, 2>(m, in, out, (int)g3, st);
            case 6: return launch_stencil3<false, 3>(m, in, out, (int)g3, st);
            case 7: return launch_stencil3<true, 3>(m, in, out, (int)g3, st);
            default: break;
        }
    }
    int64_t grid = m->ls.ntp < (int64_t)sms * 8 ? m->ls.ntp : (int64_t)sms * 8;
    if (!plain_stencil_ok(m->ls, m->Wa)) return PSF_EINVAL;  // sets beyond the plain forms' size
    if (form != 1)
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
        {
            PSF_TIMED("stencil_kernel<adjoint>", st);
            stencil_kernel<true><<<(int)grid, ST_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->cls, in, out);
        }
    } else {
        PSF_TRY(cudaFuncSetAttribute(stencil_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        {
            PSF_TIMED("stencil_kernel<forward>", st);
            stencil_kernel<false><<<(int)grid, ST_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->cls, in, out);
        }
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

}  // namespace psf

using namespace psf;

extern "C" int psf_matrix_create(psf_matrix **out, int64_t n_rows, int64_t n_cols,
                                 const int64_t *row_ptr, const int32_t *col, const void *val,
                                 int32_t dtype, const float *row_scale, void *stream) {
    PSF_RANGE("psf_matrix_create");
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
    m->wq_chunk = 0;
    m->wq_threads = 0;
    m->fwd_chunk = 0;
    m->fwd_threads = 0;
    m->queue = nullptr;
    m->st_form[0] = m->st_form[1] = 0;
    m->img2 = nullptr;
    m->csum = nullptr;
    m->csum_n = 0;
    m->topn = 0;
    m->tidx = nullptr;
    m->tw = nullptr;
    m->bk_first = nullptr;
    m->bk_nch = m->bk_nnz = 0;
    m->pair_form = 0;
    m->status = nullptr;
    m->tr_ptr = nullptr;
    m->tr_src = nullptr;
    m->tr_w = nullptr;
    m->tr_list = nullptr;
    m->tr_nz = nullptr;
    // row counters [2], the status word and the stencil's pair counter, one
    // allocation
    if (cudaMalloc(&m->queue, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        delete m;
        return PSF_ECUDA;
    }
    m->status = reinterpret_cast<int *>(m->queue + 2);
    if (cudaMemset(m->status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(m->queue);
        delete m;
        return PSF_ECUDA;
    }
    if (cudaMalloc(&m->img2, sizeof(float2) * n_cols) != cudaSuccess) {
        cudaFree(m->queue);
        delete m;
        return PSF_ECUDA;
    }
    if (n_rows > 0) {
        if (cudaMalloc(&m->p, sizeof(float) * n_rows) != cudaSuccess ||
            cudaMalloc(&m->q, sizeof(float) * n_rows) != cudaSuccess) {
            cudaFree(m->p);
            cudaFree(m->queue);
            cudaFree(m->img2);
            delete m;
            return PSF_ECUDA;
        }
    }
    *out = m;
    return PSF_OK;
}

extern "C" int psf_matrix_create_otf(psf_matrix **out, const psf_scanner *scanner,
                                     const psf_image *image, const psf_lor_set *set,
                                     void *stream) {
    PSF_RANGE("psf_matrix_create_otf");
    if (!out || !scanner || !image || !set) return PSF_EINVAL;
    Scan sc;
    Img im;
    LorSet ls;
    int rc = make_scan(scanner, &sc);
    if (!rc) rc = make_img(image, &im);
    if (!rc) rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    const int64_t n = ls.ntp * ls.nrp, nv = (int64_t)im.nx * im.ny * im.nz;
    if (n == 0 || n > INT32_MAX || nv > INT32_MAX) return PSF_EINVAL;
    // the plan's scratch and status as for stored rows; no row arrays
    static const int64_t dummy_ptr = 0;
    rc = psf_matrix_create(out, n, nv, &dummy_ptr, reinterpret_cast<const int32_t *>(&dummy_ptr),
                           &dummy_ptr, PSF_F32, nullptr, stream);
    if (rc) return rc;
    psf_matrix *m = *out;
    m->row_ptr = nullptr;
    m->col = nullptr;
    m->val = nullptr;
    m->otf = true;
    m->otf_sc = sc;
    m->otf_im = im;
    m->otf_ls = ls;
    return PSF_OK;
}

namespace psf {
// A new spread makes the transpose of the previous one stale.
static void drop_transpose(psf_matrix *m) {
    cudaFree(m->tr_ptr);
    cudaFree(m->tr_src);
    cudaFree(m->tr_w);
    cudaFree(m->tr_list);
    m->tr_ptr = nullptr;
    m->tr_src = nullptr;
    m->tr_w = nullptr;
    m->tr_list = nullptr;
    m->tr_nz = nullptr;
}
}  // namespace psf

extern "C" int psf_matrix_set_spread(psf_matrix *m, const psf_scanner *scanner,
                                     const psf_lor_set *set, int32_t half_t, int32_t half_a,
                                     const float *class_spread) {
    PSF_RANGE("psf_matrix_set_spread");
    if (!m || !class_spread || half_t < 0 || half_a < 0) return PSF_EINVAL;
    LorSet ls;
    int rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    if (ls.ntp * ls.nrp != m->n_rows) return PSF_EINVAL;
    if (!(plain_stencil_ok(ls, half_a) || stencil4_ok(ls, half_a)) || ls.NR > 32000)
        return PSF_EINVAL;
    // the class partner sums, then (8-byte aligned) each class's partner mask
    // (2 x 64 bits)
    const int64_t need =
        ls.ntp_cls * ((2 * ls.Dm + 1) * (2 * half_a + 1) * (2 * half_a + 1) + 4) + 1;
    if (need > m->csum_n) {  // grows only: a plan reused over calls allocates once
        cudaFree(m->csum);
        m->csum = nullptr;
        m->csum_n = 0;
        PSF_TRY(cudaMalloc(&m->csum, sizeof(float) * need));
        m->csum_n = need;
    }
    if (stencil5_ok(ls, half_t, half_a)) {  // form 5's packed input and weight slices
        const St5Shape s5 = st5_shape(ls, half_a);
        const int64_t np = ls.ntp * s5.plane_f;
        const int64_t nw = ls.ntp_cls * (2 * half_t + 1) * (2 * half_t + 1) * s5.w_f;
        if (np != m->pin_n) {
            cudaFree(m->pin);
            m->pin = nullptr;
            m->pin_n = 0;
            PSF_TRY(cudaMalloc(&m->pin, sizeof(float) * np));
            m->pin_n = np;
        }
        if (nw > m->wpad_n) {
            cudaFree(m->wpad);
            m->wpad = nullptr;
            m->wpad_n = 0;
            PSF_TRY(cudaMalloc(&m->wpad, sizeof(float) * nw));
            m->wpad_n = nw;
        }
    }
    m->wpad_dirty = true;
    drop_transpose(m);
    m->factored = true;
    m->ls = ls;
    m->Wt = half_t;
    m->Wa = half_a;
    m->E = (2 * half_t + 1) * (2 * half_a + 1);
    m->cls = class_spread;
    m->topn = 0;
    m->tidx = nullptr;
    m->tw = nullptr;
    m->twh = nullptr;
    m->tsc = nullptr;
    return PSF_OK;
}

extern "C" int psf_matrix_set_spread_topn(psf_matrix *m, const psf_scanner *scanner,
                                          const psf_lor_set *set, int32_t half_t, int32_t half_a,
                                          int32_t n_keep, const int32_t *idx, const float *w) {
    PSF_RANGE("psf_matrix_set_spread_topn");
    if (!m || !idx || !w || half_t < 0 || half_a < 0 || half_t > 127 || half_a > 127)
        return PSF_EINVAL;
    const int64_t E = (2 * (int64_t)half_t + 1) * (2 * (int64_t)half_a + 1);
    if (n_keep < 1 || n_keep > E * E) return PSF_EINVAL;
    LorSet ls;
    int rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    if (ls.ntp * ls.nrp != m->n_rows || ls.NR > 32000 || half_t >= ls.Nt) return PSF_EINVAL;
    drop_transpose(m);
    m->factored = true;
    m->ls = ls;
    m->Wt = half_t;
    m->Wa = half_a;
    m->E = (int)E;
    m->cls = nullptr;
    m->topn = n_keep;
    m->tidx = idx;
    m->tw = w;
    m->twh = nullptr;
    m->tsc = nullptr;
    return PSF_OK;
}

extern "C" int psf_matrix_set_spread_topn_bf16(psf_matrix *m, const psf_scanner *scanner,
                                               const psf_lor_set *set, int32_t half_t,
                                               int32_t half_a, int32_t n_keep,
                                               const int32_t *idx, const void *w16,
                                               const float *scale) {
    PSF_RANGE("psf_matrix_set_spread_topn_bf16");
    if (!w16 || !scale) return PSF_EINVAL;
    // validation and plan state as for FP32 weights, then the weights' form
    const int rc = psf_matrix_set_spread_topn(m, scanner, set, half_t, half_a, n_keep, idx,
                                              reinterpret_cast<const float *>(w16));
    if (rc) return rc;
    m->tw = nullptr;
    m->twh = static_cast<const __nv_bfloat16 *>(w16);
    m->tsc = scale;
    return PSF_OK;
}

extern "C" int psf_matrix_build_sparse_adjoint(psf_matrix *m, void *stream) {
    PSF_RANGE("psf_matrix_build_sparse_adjoint");
    if (!m || m->topn <= 0) return PSF_EINVAL;
    if (m->tr_ptr) return PSF_OK;
    const int64_t n = m->n_rows;
    if (n == 0) return PSF_OK;
    if (n > INT32_MAX) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    const size_t shm = sizeof(char4) * (size_t)m->E * m->E +
                       sizeof(int32_t) * (m->ls.Nt + m->ls.NR + 2) + sizeof(short2) * m->ls.nrp + 16;
    if (shm > 200 * 1024) return PSF_EINVAL;
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t need = (n + TS_T - 1) / TS_T;
    const int grid = (int)(need < (int64_t)sms * 8 ? need : (int64_t)sms * 8);
    int64_t *ptr = nullptr, *tiles = nullptr;
    int32_t *cur = nullptr, *src = nullptr, *list = nullptr;
    float *w = nullptr;
    int rc = PSF_OK;
    auto fail = [&](int code) {
        cudaFree(ptr);
        cudaFree(tiles);
        cudaFree(cur);
        cudaFree(src);
        cudaFree(w);
        cudaFree(list);
        return code;
    };
    if (cudaMalloc(&ptr, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&tiles, sizeof(int64_t) * scan_tile_count(n)) != cudaSuccess ||
        cudaMalloc(&cur, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&list, sizeof(int32_t) * n + 2 * sizeof(unsigned long long)) != cudaSuccess)
        return fail(PSF_ECUDA);
    if (cudaMemsetAsync(ptr, 0, sizeof(int64_t) * (n + 1), st) != cudaSuccess ||
        cudaMemsetAsync(cur, 0, sizeof(int32_t) * n, st) != cudaSuccess ||
        cudaFuncSetAttribute(topn_s_kernel<TS_COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)shm) != cudaSuccess ||
        cudaFuncSetAttribute(topn_s_kernel<TS_FILL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)shm) != cudaSuccess)
        return fail(PSF_ECUDA);
    TsTr tr{};
    tr.cnt = reinterpret_cast<unsigned long long *>(ptr + 1);
    {
        PSF_TIMED("topn_s_kernel<count>", st);
        topn_s_kernel<TS_COUNT><<<grid, TS_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->topn, m->tidx,
                                                          m->tw, m->twh, m->tsc, nullptr, nullptr, tr);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(PSF_ECUDA);
    rc = inclusive_scan(ptr + 1, n, tiles, st);
    if (rc) return fail(rc);
    int64_t total = 0;
    if (cudaMemcpyAsync(&total, ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(PSF_ECUDA);
    if (cudaMalloc(&src, sizeof(int32_t) * (total + 1)) != cudaSuccess ||
        cudaMalloc(&w, sizeof(float) * (total + 1)) != cudaSuccess)
        return fail(PSF_ECUDA);
    tr = TsTr{};
    tr.ptr = ptr;
    tr.cur = cur;
    tr.src = src;
    tr.w = w;
    {
        PSF_TIMED("topn_s_kernel<fill>", st);
        topn_s_kernel<TS_FILL><<<grid, TS_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->topn, m->tidx,
                                                         m->tw, m->twh, m->tsc, nullptr, nullptr, tr);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return fail(PSF_ECUDA);
    cudaFree(cur);
    cudaFree(tiles);
    m->tr_ptr = ptr;
    m->tr_src = src;
    m->tr_w = w;
    m->tr_list = list;
    m->tr_nz = reinterpret_cast<unsigned long long *>(list + n + (n & 1));
    return PSF_OK;
}

extern "C" int psf_matrix_destroy(psf_matrix *m) {
    PSF_RANGE("psf_matrix_destroy");
    if (!m) return PSF_EINVAL;
    cudaFree(m->p);
    cudaFree(m->q);
    cudaFree(m->queue);
    cudaFree(m->img2);
    cudaFree(m->csum);
    cudaFree(m->bk_first);
    cudaFree(m->tr_ptr);
    cudaFree(m->tr_src);
    cudaFree(m->tr_w);
    cudaFree(m->tr_list);  // the nonzero count shares this allocation
    cudaFree(m->pin);
    cudaFree(m->wpad);
    delete m;
    return PSF_OK;
}

extern "C" int psf_forward(const psf_matrix *m, const float *x, float *y, void *stream) {
    PSF_RANGE("psf_forward");
    if (!m || !x) return PSF_EINVAL;
    if (m->n_rows == 0) return PSF_OK;  // y has no entries (may be NULL)
    if (!y) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (!m->factored) return rows_fwd(m, x, y, st);
    int rc = rows_fwd(m, x, m->p, st);
    if (rc) return rc;
    return stencil(m, m->p, y, false, st);
}

namespace psf {

// y = G x on the rows with mask != 0 only (the others 0); list: int32
// scratch of n_rows entries.
static int rows_fwd_masked(const psf_matrix *m, const float *x, const float *mask, float *y,
                           int32_t *list, cudaStream_t st) {
    PSF_TRY(cudaMemsetAsync(m->queue, 0, sizeof(unsigned long long), st));
    list_nonzero(mask, m->n_rows, list, m->queue, st);
    PSF_LAUNCHED();
    PSF_TRY(cudaMemsetAsync(y, 0, sizeof(float) * m->n_rows, st));
    if (m->otf)
        return otf_rows_fwd(m->otf_sc, m->otf_im, m->otf_ls, list, m->queue, x, y, m->status, st);
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        int dev = 0, sms = 148;
        PSF_TRY(cudaGetDevice(&dev));
        PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        {
            PSF_TIMED("csr_fwd_list_kernel", st);
            csr_fwd_list_kernel<VT><<<sms * 8, PJ_T, 0, st>>>(list, m->queue, m->row_ptr, m->col,
                                                              (const VT *)m->val, m->row_scale,
                                                              x, y);
        }
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

}  // namespace psf

extern "C" int psf_forward_masked(const psf_matrix *m, const float *x, const float *mask,
                                  float *y, void *stream) {
    PSF_RANGE("psf_forward_masked");
    if (!m || !x) return PSF_EINVAL;
    if (m->n_rows == 0) return PSF_OK;  // mask and y have no entries (may be NULL)
    if (!mask || !y) return PSF_EINVAL;
    if (m->n_rows > INT32_MAX) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (!m->factored) return rows_fwd_masked(m, x, mask, y, reinterpret_cast<int32_t *>(m->p), st);
    // sources feeding a masked measured LOR: S^T of the (non-negative) mask
    int rc = stencil(m, mask, m->q, true, st);
    if (rc) return rc;
    rc = rows_fwd_masked(m, x, m->q, m->p, reinterpret_cast<int32_t *>(y), st);
    if (rc) return rc;
    rc = stencil(m, m->p, y, false, st);
    if (rc) return rc;
    {
        PSF_TIMED("keep_masked_kernel", st);
        keep_masked_kernel<<<grid_for(m->n_rows, 256), 256, 0, st>>>(mask, y, m->n_rows);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

namespace psf {

// x = A^T y for plans with the transpose of a top-N S (built for sparse
// inputs): the rows with y != 0 are listed into the transpose's list buffer;
// at most n/4 of them go through the list kernel, more through the work queue
// (each kernel returns at once when the other one applies).
static int rows_back_listed(const psf_matrix *m, const float *y, float *x, cudaStream_t st) {
    PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
    PSF_TRY(cudaMemsetAsync(m->tr_nz, 0, sizeof(unsigned long long), st));
    list_nonzero(y, m->n_rows, m->tr_list, m->tr_nz, st);
    PSF_LAUNCHED();
    if (m->otf)
        return otf_rows_back(m->otf_sc, m->otf_im, m->otf_ls, m->tr_list, m->tr_nz, y, x,
                             m->status, st);
    const int chunk = m->wq_chunk > 0 ? m->wq_chunk : 64;
    const int threads = m->wq_chunk > 0 ? m->wq_threads : 256;
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        int dev = 0, sms = 148;
        PSF_TRY(cudaGetDevice(&dev));
        PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        {
            PSF_TIMED("csr_back_list_kernel", st);
            csr_back_list_kernel<VT><<<sms * 8, PJ_T, 0, st>>>(
                m->tr_list, m->tr_nz, m->n_rows, m->row_ptr, m->col, (const VT *)m->val,
                m->row_scale, y, x);
        }
        PSF_LAUNCHED();
        int grid = 0;
        int rc = wq_grid(csr_back_wq_kernel<VT>, threads, &grid);
        if (rc) return rc;
        PSF_TRY(cudaMemsetAsync(m->queue + 1, 0, sizeof(unsigned long long), st));
        {
            PSF_TIMED("csr_back_wq_kernel", st);
            csr_back_wq_kernel<VT><<<grid, threads, 0, st>>>(
                m->n_rows, m->row_ptr, m->col, (const VT *)m->val, m->row_scale, y, x,
                m->queue + 1, chunk, m->tr_nz);
        }
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

}  // namespace psf

extern "C" int psf_back(const psf_matrix *m, const float *y, float *x, void *stream) {
    PSF_RANGE("psf_back");
    if (!m || !x) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (m->n_rows == 0) {  // y has no entries (may be NULL)
        PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
        return PSF_OK;
    }
    if (!y) return PSF_EINVAL;
    if (!m->factored) return rows_back(m, y, x, st);
    int rc = stencil(m, y, m->q, true, st);
    if (rc) return rc;
    if (m->tr_ptr) return rows_back_listed(m, m->q, x, st);
    return rows_back(m, m->q, x, st);
}

extern "C" int psf_matrix_autotune(psf_matrix *m, int32_t *chunk_out, int32_t *threads_out,
                                   void *stream) {
    PSF_RANGE("psf_matrix_autotune");
    if (!m) return PSF_EINVAL;
    if (m->otf) return PSF_EINVAL;  // traced rows: no launch choices to time
    cudaStream_t st = as_stream(stream);
    if (m->n_rows == 0) {
        m->wq_chunk = m->wq_threads = m->fwd_chunk = m->fwd_threads = 0;
        m->pair_form = 0;
    } else {
        // candidates per direction: the grid-stride kernels (chunk 0), the work
        // queue at every (rows per take, threads per CTA) pair and, forward with
        // FP32 rows, the streaming tiles (chunk -1); each timed with CUDA events
        // on all-ones vectors (one warm-up, best of two), the fastest kept
        static const int chunks[] = {-2, -1, 0, 1, 2, 4, 8, 16, 32, 64, 128};
        const bool bulk = bk_table(m, st) == PSF_OK;
        static const int threads[] = {128, 256, 512};
        float *x = nullptr;
        PSF_TRY(cudaMallocAsync(&x, sizeof(float) * m->n_cols, st));
        float *y = m->p;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int rc = PSF_OK;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            rc = PSF_ECUDA;
        if (!rc) {
            fill_kernel<<<grid_for(m->n_cols, 256), 256, 0, st>>>(x, 1.0f, m->n_cols);
            fill_kernel<<<grid_for(m->n_rows, 256), 256, 0, st>>>(y, 1.0f, m->n_rows);
            if (cudaGetLastError() != cudaSuccess) rc = PSF_ECUDA;
        }
        for (int dir = 0; dir < 2 && !rc; ++dir) {
            float best = 1e30f;
            int bc = 0, bt = 0;
            for (int c : chunks) {
                if (c < 0 && (dir == 1 || m->dtype != PSF_F32)) continue;
                if (c == -2 && !bulk) continue;
                for (int t : threads) {
                    if (rc) break;
                    if (c <= 0 && t != PJ_T) continue;
                    for (int rep = 0; rep < 3 && !rc; ++rep) {
                        if (cudaEventRecord(e0, st) != cudaSuccess) rc = PSF_ECUDA;
                        if (!rc)
                            rc = dir == 0 ? rows_fwd_with(m, x, y, c, t, st)
                                          : rows_back_with(m, y, x, c, t, st);
                        float ms = 0.0f;
                        if (!rc && (cudaEventRecord(e1, st) != cudaSuccess ||
                                    cudaEventSynchronize(e1) != cudaSuccess ||
                                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                            rc = PSF_ECUDA;
                        if (!rc && rep > 0 && ms < best) {
                            best = ms;
                            bc = c;
                            bt = c > 0 ? t : 0;
                        }
                    }
                }
            }
            if (dir == 0) {
                m->fwd_chunk = bc;
                m->fwd_threads = bt;
            } else {
                m->wq_chunk = bc;
                m->wq_threads = bt;
            }
        }
        // the pair back-projection of psf_back_sens: the back launch or the
        // bulk-staged kernel (the single back keeps the row-skipping launches:
        // a bulk-staged pass streams every chunk whatever y holds)
        m->pair_form = 0;
        PatchGrid pg;
        int psms = 0;
        size_t pshm = 0;
        const bool patch = patch_grid(m, &pg, &psms, &pshm);
        if ((bulk || patch) && !rc) {
            const int forms[3] = {0, -2, -3};
            float best[3] = {1e30f, 1e30f, 1e30f};
            for (int f = 0; f < 3 && !rc; ++f) {
                if ((f == 1 && !bulk) || (f == 2 && !patch)) continue;
                for (int rep = 0; rep < 3 && !rc; ++rep) {
                    float ms = 0.0f;
                    if (cudaEventRecord(e0, st) != cudaSuccess) rc = PSF_ECUDA;
                    if (!rc) rc = rows_back_pair(m, y, y, forms[f], st);
                    if (!rc && (cudaEventRecord(e1, st) != cudaSuccess ||
                                cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                        rc = PSF_ECUDA;
                    if (!rc && rep > 0 && ms < best[f]) best[f] = ms;
                }
            }
            int bf = 0;
            for (int f = 1; f < 3; ++f)
                if (best[f] < best[bf]) bf = f;
            if (!rc) m->pair_form = bf == 0 ? 1 : forms[bf];
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFreeAsync(x, st);
        if (rc) return rc;
        if (m->factored && m->topn == 0 && stencil3_ok(m->ls, m->Wa) &&
            stencil4_ok(m->ls, m->Wa)) {
            // stencil form per direction: both timed on all-ones LOR vectors
            cudaEvent_t f0 = nullptr, f1 = nullptr;
            if (cudaEventCreate(&f0) != cudaSuccess || cudaEventCreate(&f1) != cudaSuccess)
                rc = PSF_ECUDA;
            for (int dir = 0; dir < 2 && !rc; ++dir) {
                float best_ms = 1e30f;
                int best_form = 0;
                const int last = m->wpad && m->pin && stencil5_ok(m->ls, m->Wt, m->Wa) ? 5 : 4;
                for (int form = 3; form <= last && !rc; ++form) {
                    m->st_form[dir] = form;
                    for (int rep = 0; rep < 2 && !rc; ++rep) {
                        float ms = 0.0f;
                        if (cudaEventRecord(f0, st) != cudaSuccess) rc = PSF_ECUDA;
                        if (!rc) rc = stencil(m, m->p, m->q, dir == 1, st);
                        if (!rc && (cudaEventRecord(f1, st) != cudaSuccess ||
                                    cudaEventSynchronize(f1) != cudaSuccess ||
                                    cudaEventElapsedTime(&ms, f0, f1) != cudaSuccess))
                            rc = PSF_ECUDA;
                        if (!rc && rep > 0 && ms < best_ms) {
                            best_ms = ms;
                            best_form = form;
                        }
                    }
                }
                m->st_form[dir] = best_form;
            }
            if (f0) cudaEventDestroy(f0);
            if (f1) cudaEventDestroy(f1);
            if (rc) return rc;
        }
    }
    if (chunk_out) {
        chunk_out[0] = m->fwd_chunk;
        chunk_out[1] = m->wq_chunk;
    }
    if (threads_out) {
        threads_out[0] = m->fwd_threads;
        threads_out[1] = m->wq_threads;
    }
    return PSF_OK;
}

extern "C" int psf_matrix_set_image(psf_matrix *m, const psf_image *image) {
    PSF_RANGE("psf_matrix_set_image");
    if (!m || !image) return PSF_EINVAL;
    Img im;
    int rc = make_img(image, &im);
    if (rc) return rc;
    const int64_t nxy = (int64_t)im.nx * im.ny, nv = nxy * im.nz;
    if (nv != m->n_cols || im.nx > 65535 || nv >= (1ll << 30)) return PSF_EINVAL;
    const DivMagic a = div_magic((unsigned)nxy, (unsigned long long)nv),
                   b = div_magic((unsigned)im.nx, (unsigned long long)nxy);
    if (nv <= (1ll << 26)) {  // the theorem, checked over the grid's range
        for (int64_t n = 0; n < nv; ++n)
            if (a.div((unsigned)n) != (unsigned)(n / nxy)) return PSF_EDEBUG;
        for (int64_t n = 0; n < nxy; ++n)
            if (b.div((unsigned)n) != (unsigned)(n / im.nx)) return PSF_EDEBUG;
    }
    m->img_nx = im.nx;
    m->img_ny = im.ny;
    m->img_nz = im.nz;
    m->dv_xy_m = a.m;
    m->dv_xy_k = a.k;
    m->dv_x_m = b.m;
    m->dv_x_k = b.k;
    return PSF_OK;
}

extern "C" int psf_matrix_set_stencil_form(psf_matrix *m, int32_t form) {
    PSF_RANGE("psf_matrix_set_stencil_form");
    if (!m || form < 0 || form > 5) return PSF_EINVAL;
    m->st_form[0] = m->st_form[1] = form;
    return PSF_OK;
}

extern "C" int psf_matrix_set_launch(psf_matrix *m, int32_t chunk, int32_t threads) {
    PSF_RANGE("psf_matrix_set_launch");
    if (m && m->otf) return PSF_EINVAL;
    if (!m || chunk < -2 || chunk > (1 << 20)) return PSF_EINVAL;
    if (chunk > 0 && (threads < 32 || threads > 1024 || threads % 32)) return PSF_EINVAL;
    if (chunk < 0 && m->dtype != PSF_F32) return PSF_EINVAL;
    if (chunk == -2) {
        if (m->n_rows == 0) return PSF_EINVAL;
        const int rc = bk_table(m, nullptr);
        if (rc) return rc;
    }
    m->fwd_chunk = chunk;
    m->fwd_threads = chunk > 0 ? threads : 0;
    m->wq_chunk = chunk > 0 || chunk == -2 ? chunk : 0;
    m->wq_threads = chunk > 0 ? threads : 0;
    m->pair_form = chunk == -2 ? -2 : 0;
    return PSF_OK;
}

namespace psf {

// S^T 1 of a factored plan into out [n_rows]: the per-class partner sums, then
// the per-pair window sums.
static int sens_spread(const psf_matrix *m, float *out, cudaStream_t st) {
    if (m->topn > 0) return topn_s(m, nullptr, out, true, st);  // S^T 1: no input reads
    const int nwin = (2 * m->Wt + 1) * (2 * m->Wt + 1);
    const size_t shm = sens_smem_bytes(m->ls, m->Wa);
    if (nwin > 128 || shm > 200 * 1024 || !m->csum) return PSF_EINVAL;
    PSF_TRY(cudaFuncSetAttribute(sens_spread_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shm));
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cgrid = m->ls.ntp_cls < (int64_t)sms * 8 ? m->ls.ntp_cls : (int64_t)sms * 8;
    {
        PSF_TIMED("sens_class_kernel", st);
        sens_class_kernel<<<(int)cgrid, SS_T,
                            2 * sizeof(unsigned long long) + sizeof(int32_t) * (m->ls.Nt + m->ls.NR + 2),
                            st>>>(m->ls, m->Wt, m->Wa, m->cls, m->csum);
    }
    PSF_LAUNCHED();
    const int64_t grid = m->ls.ntp < (int64_t)sms * 8 ? m->ls.ntp : (int64_t)sms * 8;
    {
        PSF_TIMED("sens_spread_kernel", st);
        sens_spread_kernel<<<(int)grid, SS_T, shm, st>>>(m->ls, m->Wt, m->Wa, m->cls, m->csum,
                                                         out);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

}  // namespace psf

extern "C" int psf_sensitivity(const psf_matrix *m, float *x, void *stream) {
    PSF_RANGE("psf_sensitivity");
    if (!m || !x) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (m->n_rows == 0) {
        PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
        return PSF_OK;
    }
    if (!m->factored) {  // stored rows: A^T of an all-ones vector
        {
            PSF_TIMED("fill_kernel", st);
            fill_kernel<<<grid_for(m->n_rows, 256), 256, 0, st>>>(m->p, 1.0f, m->n_rows);
        }
        PSF_LAUNCHED();
        return rows_back(m, m->p, x, st);
    }
    const int rc = sens_spread(m, m->q, st);
    if (rc) return rc;
    return rows_back(m, m->q, x, st);
}

// x = A^T y and sens = A^T 1 with one pass over the stored rows.
extern "C" int psf_back_sens(const psf_matrix *m, const float *y, float *x, float *sens,
                             void *stream) {
    PSF_RANGE("psf_back_sens");
    if (!m || !x || !sens) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (m->n_rows == 0) {  // y has no entries (may be NULL)
        PSF_TRY(cudaMemsetAsync(x, 0, sizeof(float) * m->n_cols, st));
        PSF_TRY(cudaMemsetAsync(sens, 0, sizeof(float) * m->n_cols, st));
        return PSF_OK;
    }
    if (!y) return PSF_EINVAL;
    const float *qa, *qb;  // LOR-space inputs of G^T: S^T 1 and S^T y (or 1 and y)
    if (m->factored) {
        int rc = sens_spread(m, m->p, st);
        if (rc) return rc;
        rc = stencil(m, y, m->q, true, st);
        if (rc) return rc;
        qa = m->p;
        qb = m->q;
    } else {
        {
            PSF_TIMED("fill_kernel", st);
            fill_kernel<<<grid_for(m->n_rows, 256), 256, 0, st>>>(m->p, 1.0f, m->n_rows);
        }
        PSF_LAUNCHED();
        qa = m->p;
        qb = y;
    }
    if (m->otf) {  // two traced passes: A^T 1 then A^T y
        int rc = rows_back(m, qa, sens, st);
        return rc ? rc : rows_back(m, qb, x, st);
    }
    // pair form 0: the per-pair shared-memory kernel where the plan allows it,
    // else the back projection's launch (form 1: that launch, kept by the
    // autotuner)
    int form = m->pair_form;
    if (form == 0) {
        PatchGrid g;
        int sms = 0;
        size_t shm = 0;
        form = patch_grid(m, &g, &sms, &shm) ? -3 : 0;
    } else if (form == 1) {
        form = 0;
    }
    int rc = rows_back_pair(m, qa, qb, form, st);
    if (rc) return rc;
    {
        PSF_TIMED("split_pair_kernel", st);
        split_pair_kernel<<<grid_for(m->n_cols, 256), 256, 0, st>>>(m->img2, sens, x, m->n_cols);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

namespace psf {

// The launch of the per-pair shared-memory form: its grid (one CTA per SM),
// the cells a pair may hold, and whether the plan allows it (a factored plan
// over the full set with its image declared).
static bool patch_grid(const psf_matrix *m, PatchGrid *g, int *sms_out, size_t *shm_out) {
    if (!m->factored || m->topn > 0 || m->otf || m->img_nz <= 0 || m->n_rows == 0) return false;
    if (m->n_rows != m->ls.ntp * m->ls.nrp) return false;
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
        return false;
    g->nx = m->img_nx;
    g->ny = m->img_ny;
    g->nz = m->img_nz;
    g->nxy = m->img_nx * m->img_ny;
    g->dxy.m = m->dv_xy_m;
    g->dxy.k = m->dv_xy_k;
    g->dx.m = m->dv_x_m;
    g->dx.k = m->dv_x_k;
    const int rm = m->ls.NR / 2;  // the direct-plane row of the middle ring lists the cells
    int64_t jm = 0;
    for (int r = 0; r < rm; ++r) jm += m->ls.rp_count(r);
    g->jm = (int)(jm + (rm - m->ls.rp_lo(rm)));
    // + the kernel's static shared memory
    const size_t fixed = sizeof(int2) * (size_t)g->ny + sizeof(int) * 4 * (size_t)g->ny +
                         sizeof(int) * ((size_t)m->ls.nrp + 1) + sizeof(float2) * m->ls.nrp + 512;
    if ((size_t)optin <= fixed) return false;
    int cap = (int)(((size_t)optin - fixed) / (sizeof(float2) * g->nz + sizeof(int)));
    cap = cap / 4 * 4;
    cap = cap < 32767 ? cap : 32764;  // a cell index and a run length in 16 bits
    if (cap < 32) return false;
    g->cap = cap;
    *sms_out = sms;
    *shm_out = patch_smem_bytes(*g, (int)m->ls.nrp);
    return true;
}

static int rows_back_patch(const psf_matrix *m, const float *qa, const float *qb,
                           cudaStream_t st) {
    PatchGrid g;
    int sms = 0;
    size_t shm = 0;
    if (!patch_grid(m, &g, &sms, &shm)) return PSF_EINVAL;
    PSF_TRY(cudaMemsetAsync(m->queue + 3, 0, sizeof(unsigned long long), st));  // pair counter
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        PSF_TRY(cudaFuncSetAttribute(csr_back_patch_kernel<VT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        {
            PSF_TIMED("csr_back_patch_kernel", st);
            csr_back_patch_kernel<VT><<<sms, PP_T, shm, st>>>(
                m->ls.ntp, (int)m->ls.nrp, m->row_ptr, m->col, (const VT *)m->val,
                m->row_scale, qa, qb, m->img2, m->queue + 3, g);
        }
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

// img2 = A^T (qa, qb) as an interleaved pair: form -3 the per-pair
// shared-memory kernel, -2 the bulk-staged kernel, else the pair kernel at
// the back projection's launch.
static int rows_back_pair(const psf_matrix *m, const float *qa, const float *qb, int form,
                          cudaStream_t st) {
    PSF_TRY(cudaMemsetAsync(m->img2, 0, sizeof(float2) * m->n_cols, st));
    if (m->otf) return PSF_EINVAL;  // psf_back_sens traces twice instead
    if (form == -3) return rows_back_patch(m, qa, qb, st);
    if (form == -2) {
        if (!m->bk_first) return PSF_EINVAL;
        int grid = 0;
        size_t shm = 0;
        int rc = bk_launch_shape(csr_back_bulk_kernel<true>, m->bk_nch, &grid, &shm);
        if (rc) return rc;
        {
            PSF_TIMED("csr_back_bulk_kernel<pair>", st);
            csr_back_bulk_kernel<true><<<grid, BK_T, shm, st>>>(
                m->n_rows, m->bk_nnz, m->bk_nch, m->bk_first, m->row_ptr, m->col,
                (const float *)m->val, qa, qb, nullptr, m->img2, m->status,
                (long long)wait_limit());
        }
        PSF_LAUNCHED();
        return PSF_OK;
    }
    const int chunk = m->wq_chunk > 0 ? m->wq_chunk : 0;
    const int threads = chunk > 0 ? m->wq_threads : PJ_T;
    return dispatch_dtype(m->dtype, [&](auto tag) -> int {
        using VT = std::remove_const_t<std::remove_pointer_t<decltype(tag)>>;
        int grid = grid_for(m->n_rows * 32, PJ_T);
        if (chunk > 0) {
            int r = wq_grid(csr_back_pair_kernel<VT>, threads, &grid);
            if (r) return r;
            PSF_TRY(cudaMemsetAsync(m->queue + 1, 0, sizeof(unsigned long long), st));
        }
        {
            PSF_TIMED("csr_back_pair_kernel", st);
            csr_back_pair_kernel<VT><<<grid, threads, 0, st>>>(
                m->n_rows, m->row_ptr, m->col, (const VT *)m->val, m->row_scale, qa, qb, m->img2,
                chunk > 0 ? m->queue + 1 : nullptr, chunk);
        }
        PSF_LAUNCHED();
        return PSF_OK;
    });
}

}  // namespace psf

extern "C" int psf_matrix_check(const psf_matrix *m, void *stream) {
    PSF_RANGE("psf_matrix_check");
    if (!m) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    int h = 0;
    PSF_TRY(cudaMemcpyAsync(&h, m->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSF_TRY(cudaStreamSynchronize(st));
    if (h) PSF_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), st));
    return h;
}
