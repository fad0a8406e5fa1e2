// List-mode data (the paper's next step, Sec. 5): events are crystal pairs,
// mapped to the rows of a structured LOR set and accumulated per subset into
// LOR-space counts, so that an OSEM sub-iteration over a subset of events,
//   x <- x * sum_{e in subset} A_e^T / (A_e x) / (A^T 1 / n_subsets),
// runs on the set's projector as x * A^T(c / A x) / A^T 1 with
// c = n_subsets * (events of the subset per LOR).
#include "psf_common.cuh"
#include "psf_lorset.cuh"

namespace psf {

constexpr int LM_T = 256;

// Row of each event's crystal pair in the set (either order of the two
// crystals), -1 when the pair is not in the set.
__global__ void __launch_bounds__(LM_T) event_rows_kernel(LorSet ls, const int32_t *__restrict__ ev,
                                                          int64_t n, int64_t *__restrict__ rows) {
    extern __shared__ int32_t lm_pre[];  // tp_start [Nt + 1], rp_start [NR + 1]
    int32_t *tp_start = lm_pre, *rp_start = lm_pre + ls.Nt + 1;
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    const int nc = ls.Nt * ls.NR;
    for (int64_t i = (int64_t)blockIdx.x * LM_T + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * LM_T) {
        const int id1 = ev[2 * i], id2 = ev[2 * i + 1];
        int64_t r = -1;
        if (id1 >= 0 && id2 >= 0 && id1 < nc && id2 < nc) {
            const int r1 = id1 / ls.Nt, c1 = id1 - r1 * ls.Nt;
            const int r2 = id2 / ls.Nt, c2 = id2 - r2 * ls.Nt;
            const bool sw = c1 > c2;
            const int a = sw ? c2 : c1, b = sw ? c1 : c2, ra = sw ? r2 : r1, rb = sw ? r1 : r2;
            if (ls.member(a, b, ra, rb)) r = ls.row_of(tp_start, rp_start, a, b, ra, rb);
        }
        rows[i] = r;
    }
}

__global__ void __launch_bounds__(LM_T) histogram_kernel(const int64_t *__restrict__ rows, int64_t n,
                                                         float weight, float *__restrict__ counts,
                                                         int64_t n_rows) {
    for (int64_t i = (int64_t)blockIdx.x * LM_T + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * LM_T) {
        const int64_t r = rows[i];
        if (r >= 0 && r < n_rows) atomicAdd(counts + r, weight);
    }
}

// Sinogram view and bin of every transaxial pair of the set (the histogram
// organisation of Sec. 4, Table 1), ideal-ring convention: u = a + b,
// view = (u mod Nt) / 2, bin = sg (b - a - Nt/2) + F, sg = +1 if u < Nt else -1.
__global__ void __launch_bounds__(LM_T) sino_bins_kernel(LorSet ls, int32_t *__restrict__ view,
                                                         int32_t *__restrict__ bin) {
    extern __shared__ int32_t sb_pre[];  // tp_start [Nt + 1], rp_start [NR + 1]
    ls.stage_prefix(sb_pre, sb_pre + ls.Nt + 1);
    __syncthreads();
    for (int64_t T = (int64_t)blockIdx.x * LM_T + threadIdx.x; T < ls.ntp;
         T += (int64_t)gridDim.x * LM_T) {
        int a, b;
        ls.tp_decode(sb_pre, T, &a, &b);
        const int u = a + b, d = b - a;
        view[T] = (u % ls.Nt) / 2;
        bin[T] = (u < ls.Nt ? 1 : -1) * (d - ls.Nt / 2) + ls.F;
    }
}

}  // namespace psf

using namespace psf;

extern "C" int psf_sino_bins(const psf_scanner *scanner, const psf_lor_set *set, int32_t *view,
                             int32_t *bin, void *stream) {
    PSF_RANGE("psf_sino_bins");
    LorSet ls;
    int rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    if (ls.Nt % 2 || ls.F > ls.Nt / 2 - 1) return PSF_EINVAL;
    if (ls.ntp == 0) return PSF_OK;
    if (!view || !bin) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    const size_t shm = sizeof(int32_t) * (ls.Nt + ls.NR + 2);
    {
        PSF_TIMED("sino_bins_kernel", st);
        sino_bins_kernel<<<grid_for(ls.ntp, LM_T), LM_T, shm, st>>>(ls, view, bin);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

extern "C" int psf_event_rows(const psf_scanner *scanner, const psf_lor_set *set,
                              const int32_t *events, int64_t n_events, int64_t *rows,
                              void *stream) {
    PSF_RANGE("psf_event_rows");
    LorSet ls;
    int rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    if (n_events < 0) return PSF_EINVAL;
    if (n_events == 0) return PSF_OK;
    if (!events || !rows) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    const size_t shm = sizeof(int32_t) * (ls.Nt + ls.NR + 2);
    {
        PSF_TIMED("event_rows_kernel", st);
        event_rows_kernel<<<grid_for(n_events, LM_T), LM_T, shm, st>>>(ls, events, n_events, rows);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

extern "C" int psf_histogram(const int64_t *rows, int64_t n_events, float weight, float *counts,
                             int64_t n_rows, void *stream) {
    PSF_RANGE("psf_histogram");
    if (n_events < 0 || n_rows < 0) return PSF_EINVAL;
    if (n_rows > 0 && !counts) return PSF_EINVAL;
    if (n_events > 0 && !rows) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    if (n_rows > 0) PSF_TRY(cudaMemsetAsync(counts, 0, sizeof(float) * n_rows, st));
    if (n_events == 0 || n_rows == 0) return PSF_OK;
    {
        PSF_TIMED("histogram_kernel", st);
        histogram_kernel<<<grid_for(n_events, LM_T), LM_T, 0, st>>>(rows, n_events, weight, counts,
                                                                     n_rows);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}
