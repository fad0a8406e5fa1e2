// K1: the P-SPIR response table (Sec. 2.1.1, Eq. 1) with the FP64 counting-
// rate prefix sums of the normalisation (Sec. 2.1.3, Eq. 6-7).
//
// One warp per table entry (angle node pair, entry sub-position).  The lanes
// clip the ray against the stored crystal boxes in parallel, stage the entry
// depth and path length of every box in shared memory, and each lane then
// sums the material met before its box across the warp's staging area.
// Values are FP32; the per-entry counting-rate sums are FP64 warp scans.
#include "psf_common.cuh"

namespace psf {

__global__ void __launch_bounds__(128) response_kernel(Scan sc, Tab tb, float *__restrict__ table,
                                                       double *__restrict__ eta) {
    extern __shared__ float sh[];
    const int MM = tb.Mt * tb.Ma;
    const int warps = blockDim.x >> 5;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *zin = sh + w * 3 * MM;
    float *len = zin + MM;
    float *tv = len + MM;
    const int64_t n_entries = (int64_t)tb.Kt * tb.Ka * tb.Pt * tb.Pa;
    for (int64_t e = (int64_t)blockIdx.x * warps + w; e < n_entries;
         e += (int64_t)gridDim.x * warps) {
        int iv = (int)(e % tb.Pa);
        int iu = (int)((e / tb.Pa) % tb.Pt);
        int ka = (int)((e / ((int64_t)tb.Pa * tb.Pt)) % tb.Ka);
        int kt = (int)(e / ((int64_t)tb.Pa * tb.Pt * tb.Ka));
        float at = kt * tb.dt, th = ka * tb.da;
        float tx = tanf(at);
        float ty = tanf(th) / cosf(at);
        float x0 = (iu + 0.5f) / tb.Pt * sc.wt;
        float y0 = (iv + 0.5f) / tb.Pa * sc.wa;
        float ds = sqrtf(1.0f + tx * tx + ty * ty);
        // clip every stored crystal box (kx, ky) against the ray
        for (int b = lane; b < MM; b += 32) {
            int kx = b / tb.Ma, ky = b - kx * tb.Ma;
            float lo = 0.0f, hi = sc.depth;
            float ax = kx * sc.pt, bx = ax + sc.wt;
            float ay = ky * sc.pa, by = ay + sc.wa;
            if (tx > 0.0f) {
                lo = fmaxf(lo, (ax - x0) / tx);
                hi = fminf(hi, (bx - x0) / tx);
            } else if (!(x0 >= ax && x0 <= bx)) {
                hi = -1.0f;
            }
            if (ty > 0.0f) {
                lo = fmaxf(lo, (ay - y0) / ty);
                hi = fminf(hi, (by - y0) / ty);
            } else if (!(y0 >= ay && y0 <= by)) {
                hi = -1.0f;
            }
            zin[b] = lo;
            len[b] = hi > lo ? (hi - lo) * ds : 0.0f;
        }
        __syncwarp();
        // first-interaction probability: exp(-mu L_before) (1 - exp(-mu L))
        float *out = table + e * MM;
        for (int b = lane; b < MM; b += 32) {
            float L = len[b], z = zin[b];
            float before = 0.0f;
            for (int j = 0; j < MM; ++j) {
                float lj = len[j];
                before += (lj > 0.0f && zin[j] < z) ? lj : 0.0f;
            }
            float T = L > 0.0f ? expf(-sc.mu * before) * -expm1f(-sc.mu * L) : 0.0f;
            tv[b] = T;
            out[b] = T;
        }
        __syncwarp();
        // FP64 prefix over dx of the dz-summed table (counting rate, Eq. 6)
        double *eo = eta + e * (tb.Mt + 1);
        double carry = 0.0;
        if (lane == 0) eo[0] = 0.0;
        for (int base = 0; base < tb.Mt; base += 32) {
            int dx = base + lane;
            double col = 0.0;
            if (dx < tb.Mt)
                for (int dz = 0; dz < tb.Ma; ++dz) col += (double)tv[dx * tb.Ma + dz];
            double inc = col;
            for (int o = 1; o < 32; o <<= 1) {
                double t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            if (dx < tb.Mt) eo[dx + 1] = carry + inc;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        __syncwarp();
    }
}

}  // namespace psf

using namespace psf;

extern "C" int psf_response_build(const psf_scanner *scanner, const psf_table_desc *desc,
                                  float *table, double *eta, void *stream) {
    PSF_RANGE("psf_response_build");
    Scan sc;
    Tab tb;
    int rc = make_scan(scanner, &sc);
    if (rc) return rc;
    rc = make_tab(desc, sc, &tb, true);
    if (rc) return rc;
    if (!table || !eta) return PSF_EINVAL;
    const int threads = 128, warps = threads / 32;
    size_t shm = sizeof(float) * 3 * tb.Mt * tb.Ma * warps;
    int64_t n = (int64_t)tb.Kt * tb.Ka * tb.Pt * tb.Pa;
    int64_t blocks = (n + warps - 1) / warps;
    if (blocks > 65535) blocks = 65535;
    if (shm > 48 * 1024)
        PSF_TRY(cudaFuncSetAttribute(response_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)shm));
    {
        PSF_TIMED("response_kernel", as_stream(stream));
        response_kernel<<<(int)blocks, threads, shm, as_stream(stream)>>>(sc, tb, table, eta);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}
