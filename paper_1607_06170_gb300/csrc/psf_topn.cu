// Top-N truncation of LOR spreads (Sec. 4.3, Table 3): the window entries of
// each LOR ranked by weight, the first N kept and rescaled to the window's
// total.  Ranking rule (a reading; the paper only says "descending order"):
// a negative weight ranks as 0; equal weights rank the smaller offset
// |dt1|+|da1|+|dt2|+|da2| first, then the lower window index e1*E + e2.
#include <cuda_bf16.h>

#include "psf_common.cuh"

namespace psf {

constexpr int TN_T = 128;    // threads per LOR
constexpr int TN_EPT = 19;   // window entries per thread: E*E <= 2432 (a 7 x 7 x 7 x 7 window)
constexpr int TN_MAX = 64;   // largest N

// Unique 64-bit rank key, larger = earlier: the weight's bits (non-negative
// floats order as their bit patterns), then the complement of the tie rank.
__device__ __forceinline__ unsigned long long tn_key(float w, unsigned tie) {
    const unsigned wb = w > 0.0f ? __float_as_uint(w) : 0u;
    return ((unsigned long long)wb << 32) | (0xffffffffu - tie);
}

__device__ __forceinline__ unsigned long long tn_max(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// One CTA per LOR.  Each round takes the largest key below the previous
// round's (keys are unique), so N rounds give the first N in rank order.
__global__ void __launch_bounds__(TN_T) topn_kernel(const float *__restrict__ spread, int64_t n,
                                                    int Wt, int Wa, int N,
                                                    int32_t *__restrict__ idx,
                                                    float *__restrict__ wout) {
    __shared__ unsigned long long red[TN_T / 32];
    __shared__ double dred[TN_T / 32];
    __shared__ float sel[TN_MAX];
    const int W2a = 2 * Wa + 1, E = (2 * Wt + 1) * W2a, EE = E * E;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned F = 0xffffffffu;
    for (int64_t g = blockIdx.x; g < n; g += gridDim.x) {
        const float *wg = spread + g * EE;
        unsigned long long key[TN_EPT];
        double part = 0.0;
#pragma unroll
        for (int i = 0; i < TN_EPT; ++i) {
            const int e = t + i * TN_T;
            key[i] = 0ull;  // padding: below every real key
            if (e < EE) {
                const float w = wg[e];
                part += (double)w;
                const int e1 = e / E, e2 = e - e1 * E;
                const int dist = abs(e1 / W2a - Wt) + abs(e1 % W2a - Wa) + abs(e2 / W2a - Wt) +
                                 abs(e2 % W2a - Wa);
                key[i] = tn_key(w, (unsigned)(dist * EE + e));
            }
        }
        part = warp_sum_d(part);
        __syncthreads();  // the previous LOR's readers of dred / sel are done
        if (lane == 0) dred[warp] = part;
        __syncthreads();
        double all = 0.0;
#pragma unroll
        for (int w = 0; w < TN_T / 32; ++w) all += dred[w];
        unsigned long long prev = ~0ull;
        double kept = 0.0;
        for (int k = 0; k < N; ++k) {
            unsigned long long best = 0ull;
#pragma unroll
            for (int i = 0; i < TN_EPT; ++i)
                if (key[i] < prev) best = tn_max(best, key[i]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) best = tn_max(best, __shfl_xor_sync(F, best, o));
            if (lane == 0) red[warp] = best;
            __syncthreads();
            best = red[0];
#pragma unroll
            for (int w = 1; w < TN_T / 32; ++w) best = tn_max(best, red[w]);
            __syncthreads();  // red is rewritten next round
            prev = best;
            const int e = (int)((0xffffffffu - (unsigned)best) % (unsigned)EE);
            const float w = wg[e];
            kept += (double)w;
            if (t == 0) {
                sel[k] = w;
                idx[g * N + k] = e;
            }
        }
        const double scale = kept != 0.0 ? all / kept : 1.0;
        __syncthreads();  // sel is complete
        for (int k = t; k < N; k += TN_T) wout[g * N + k] = (float)((double)sel[k] * scale);
    }
}

}  // namespace psf

using namespace psf;

extern "C" int psf_spread_topn(const float *spread, int64_t n_lors, int32_t half_t,
                               int32_t half_a, int32_t n_keep, int32_t *idx, float *w,
                               void *stream) {
    PSF_RANGE("psf_spread_topn");
    if (n_lors < 0 || half_t < 0 || half_a < 0) return PSF_EINVAL;
    const int64_t E = (2 * (int64_t)half_t + 1) * (2 * (int64_t)half_a + 1);
    if (E * E > (int64_t)TN_T * TN_EPT) return PSF_EINVAL;
    if (n_keep < 1 || n_keep > TN_MAX || n_keep > E * E) return PSF_EINVAL;
    if (n_lors == 0) return PSF_OK;
    if (!spread || !idx || !w) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    int dev = 0, sms = 148;
    PSF_TRY(cudaGetDevice(&dev));
    PSF_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t grid = n_lors < (int64_t)sms * 16 ? n_lors : (int64_t)sms * 16;
    {
        PSF_TIMED("topn_kernel", st);
        topn_kernel<<<(int)grid, TN_T, 0, st>>>(spread, n_lors, half_t, half_a, n_keep, idx, w);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

namespace psf {

// Top-N weights -> BF16 codes with one FP32 scale per spread: scale = the
// largest |w| of the spread's kept weights (1 when they are all 0), code =
// w / scale rounded to the nearest BF16 (ties to even).  One warp per spread.
__global__ void topn_bf16_kernel(const float *__restrict__ w, int64_t n, int N,
                                 __nv_bfloat16 *__restrict__ w16, float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n;
         g += warps) {
        float mx = 0.0f;
        for (int k = lane; k < N; k += 32) mx = fmaxf(mx, fabsf(w[g * N + k]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = mx > 0.0f ? mx : 1.0f;
        for (int k = lane; k < N; k += 32) w16[g * N + k] = __float2bfloat16_rn(__fdiv_rn(w[g * N + k], sc));
        if (lane == 0) scale[g] = sc;
    }
}

}  // namespace psf

extern "C" int psf_spread_topn_bf16(const float *w, int64_t n_spreads, int32_t n_keep,
                                    void *w16, float *scale, void *stream) {
    PSF_RANGE("psf_spread_topn_bf16");
    if (n_spreads < 0 || n_keep < 1 || n_keep > TN_MAX) return PSF_EINVAL;
    if (n_spreads == 0) return PSF_OK;
    if (!w || !w16 || !scale) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    const int64_t blocks = (n_spreads + 7) / 8;
    const int grid = (int)(blocks < 65535 * 16 ? blocks : 65535 * 16);
    {
        PSF_TIMED("topn_bf16_kernel", st);
        topn_bf16_kernel<<<grid, 256, 0, st>>>(w, n_spreads, n_keep,
                                               static_cast<__nv_bfloat16 *>(w16), scale);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}
