// Shared definitions of the GB300 P-SPIR library: derived scanner constants,
// argument validation, error plumbing and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdint>

#include "psf.h"

namespace psf {

// Last CUDA error seen by an entry point (for psf_strerror on PSF_ECUDA).
void set_cuda_error(cudaError_t e);

#define PSF_TRY(call)                                \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) {                     \
            ::psf::set_cuda_error(e_);               \
            return PSF_ECUDA;                        \
        }                                            \
    } while (0)

#define PSF_LAUNCHED()                               \
    do {                                             \
        cudaError_t e_ = cudaGetLastError();         \
        if (e_ != cudaSuccess) {                     \
            ::psf::set_cuda_error(e_);               \
            return PSF_ECUDA;                        \
        }                                            \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Kernel timing (psf_timing_enable): a scope around one launch records an
// event before and one after it on the launching stream while timing is on.
bool timing_on();
cudaEvent_t timing_start(cudaStream_t st);
void timing_stop(const char *name, cudaStream_t st, cudaEvent_t start);

struct KTimer {
    const char *name;
    cudaStream_t st;
    cudaEvent_t ev;
    KTimer(const char *n, cudaStream_t s) : name(n), st(s), ev(nullptr) {
        if (timing_on()) ev = timing_start(s);
    }
    ~KTimer() {
        if (ev) timing_stop(name, st, ev);
    }
    KTimer(const KTimer &) = delete;
    KTimer &operator=(const KTimer &) = delete;
};
#define PSF_TIMED(name, st) ::psf::KTimer psf_ktimer_(name, st)

// NVTX range around an entry point (shown by Nsight tools; inert otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *n) { nvtxRangePushA(n); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define PSF_RANGE(name) ::psf::NvtxRange psf_nvtx_range_(name)

// Cycle limit of the bounded device waits (psf_set_wait_limit): a wait that
// has not seen its event after this many SM clock cycles gives up and records
// PSF_ETIMEOUT; a negative limit makes the waits give up at once (a test of
// the timeout path).
int64_t wait_limit();

// Scanner constants as the kernels use them (passed by value).
struct Scan {
    int R, Nb, Nt, NR;          // blocks, crystals/block, crystals/ring, rings
    float wt, wa, depth;        // crystal width (transaxial / axial), depth
    float gt, ga, pt, pa;       // intra-block gaps and pitches
    float mu, radius;
    float half_w;               // half the transaxial block width
    float sigma;                // corner gap AB = BC of the gap construction
    float z0;                   // axial centre of ring 0 (rings on a uniform pitch)
    float two_pi_R;             // angle between neighbouring block normals
    float sin_two_pi_R;
    double radius64, pt64, pa64, z064;
};

// Table layout constants.
struct Tab {
    int Kt, Ka, Pt, Pa, Mt, Ma;
    float dt, da;               // node spacing (radians)
    float inv_dt, inv_da;
};

struct Img {
    int nx, ny, nz;
    double dx, dy, dz, ox, oy, oz;
    double idx, idy, idz;  // 1 / voxel size
};

// Validation + derivation (host).  Return PSF_OK or PSF_EINVAL.
int make_scan(const psf_scanner *s, Scan *out);
int make_tab(const psf_table_desc *d, const Scan &sc, Tab *out, bool check_reach);
int make_img(const psf_image *im, Img *out);

struct LorSet;

// Rows traced on the fly (a plan without stored rows, psf_matrix_create_otf):
// for the rows of a structured set listed in list[0 .. *count) -- or every row
// when list is NULL -- y[row] = G_row . x (overwrites the listed entries of y),
// or x += y[row] G_row (FP32 atomics; rows with y == 0 are skipped).  The
// chords are the per-LOR tracer's, so they equal the stored rows bit for bit.
// A tracer lookup that did not settle records PSF_EDEBUG in *status.
int otf_rows_fwd(const Scan &sc, const Img &im, const LorSet &ls, const int32_t *list,
                 const unsigned long long *count, const float *x, float *y, int *status,
                 cudaStream_t st);
int otf_rows_back(const Scan &sc, const Img &im, const LorSet &ls, const int32_t *list,
                  const unsigned long long *count, const float *y, float *x, int *status,
                  cudaStream_t st);

// Grid for a grid-stride loop over n items: at most 8 CTAs per SM.
int grid_for(int64_t n, int block);

// In-place inclusive scan of an int64 array on `st` (three launches);
// tile_sums needs scan_tile_count(n) slots.
int64_t scan_tile_count(int64_t n);
int inclusive_scan(int64_t *x, int64_t n, int64_t *tile_sums, cudaStream_t st);

__host__ __device__ inline int64_t table_entry(const Tab &t, int kt, int ka, int iu, int iv) {
    return (((int64_t)kt * t.Ka + ka) * t.Pt + iu) * t.Pa + iv;
}

// Conversions with the device intrinsics' rounding, usable from host code.
__host__ __device__ __forceinline__ int f2i_rd(float x) {
#ifdef __CUDA_ARCH__
    return __float2int_rd(x);
#else
    return (int)floorf(x);
#endif
}

__host__ __device__ __forceinline__ long long d2ll_rn(double x) {
#ifdef __CUDA_ARCH__
    return __double2ll_rn(x);
#else
    return llrint(x);
#endif
}

template <typename T>
__host__ __device__ __forceinline__ T ldg(const T *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// Nearest angle node (nodes at k * spacing, clamped to the last node).
__host__ __device__ __forceinline__ int angle_node(float ang, float inv_step, int K) {
    int k = f2i_rd(fmaf(ang, inv_step, 0.5f));
    return k < K - 1 ? k : K - 1;
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace psf
