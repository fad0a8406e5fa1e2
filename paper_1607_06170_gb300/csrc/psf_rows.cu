// K4-K7: system-matrix rows in CSR.
//
// Geometric rows G (chord lengths of the segment joining two crystal
// front-face centres):  K4 counts each row with the exact-parameter tracer
// (per row of voxels, not per voxel), K5 scans the counts into row_ptr, K6
// traces again and writes the sorted columns and chords.
// PSF rows A = S G (Sec. 2.3) for small images:  K7 gathers, for each output
// LOR, every geometric LOR whose spread window lands on it, accumulates their
// weighted rows densely in shared memory in a fixed order, and compacts the
// non-zeros in ascending voxel order (count pass, scan, fill pass).
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "psf_common.cuh"
#include "psf_rows.cuh"

namespace psf {

constexpr int ROWS_THREADS = 128;

// Block trig (FP64) staged per CTA.
__device__ __forceinline__ void stage_blocks(const Scan &sc, double *cs) {
    for (int b = threadIdx.x; b < sc.R; b += blockDim.x) {
        double s, c;
        sincospi(2.0 * b / sc.R, &s, &c);
        cs[2 * b] = c;
        cs[2 * b + 1] = s;
    }
}

// Front-face centre of crystal id (mm, FP64).
__device__ __forceinline__ void face_centre(const Scan &sc, const double *cs, int id, double &x,
                                            double &y, double &z) {
    int ring = id / sc.Nt, c = id - ring * sc.Nt;
    int b = c / sc.Nb, i = c - b * sc.Nb;
    double cb = cs[2 * b], sb = cs[2 * b + 1];
    double s = (i - 0.5 * (sc.Nb - 1)) * sc.pt64;
    x = sc.radius64 * cb - s * sb;
    y = sc.radius64 * sb + s * cb;
    z = sc.z064 + ring * sc.pa64;
}

__device__ __forceinline__ void lor_ray(Ray &r, const Scan &sc, const Img &im, const double *cs,
                                        int id1, int id2) {
    const int nc = sc.Nt * sc.NR;
    if (id1 < 0 || id2 < 0 || id1 >= nc || id2 >= nc) {  // invalid ids: empty row
        r.empty = true;
        return;
    }
    double px, py, pz, qx, qy, qz;
    face_centre(sc, cs, id1, px, py, pz);
    face_centre(sc, cs, id2, qx, qy, qz);
    make_ray(r, im, px, py, pz, qx, qy, qz);
}

__global__ void __launch_bounds__(ROWS_THREADS) g_count_kernel(
    Scan sc, Img im, const int32_t *__restrict__ lors, int64_t n, int64_t *__restrict__ counts,
    int *__restrict__ status) {
    extern __shared__ double cs[];
    stage_blocks(sc, cs);
    __syncthreads();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        Ray r;
        lor_ray(r, sc, im, cs, lors[2 * k], lors[2 * k + 1]);
        int64_t cnt = 0;
        bool ok = trace_rows(r, [&](int, int, int x0, int x1, long long, long long) {
            cnt += x1 - x0 + 1;
        });
        if (!ok) atomicExch(status, PSF_EDEBUG);
        counts[k] = cnt;
    }
}

// K6: each lane of a warp traces one LOR with a resumable cursor and stages
// up to 32 of its voxels in shared memory; the warp then writes every lane's
// chunk with full 128-byte stores (one row segment per store instruction).
constexpr int FILL_WARPS = 8;
constexpr int FILL_PAD = 33;  // staging row stride (conflict-free lane-major writes)

__global__ void __launch_bounds__(FILL_WARPS * 32) g_fill_kernel(
    Scan sc, Img im, const int32_t *__restrict__ lors, int64_t n,
    const int64_t *__restrict__ row_ptr, int32_t *__restrict__ col, float *__restrict__ val,
    int *__restrict__ status) {
    extern __shared__ double cs[];
    stage_blocks(sc, cs);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *scol = reinterpret_cast<int32_t *>(cs + 2 * sc.R) + warp * 32 * FILL_PAD;
    float *sval = reinterpret_cast<float *>(reinterpret_cast<int32_t *>(cs + 2 * sc.R) +
                                            FILL_WARPS * 32 * FILL_PAD) +
                  warp * 32 * FILL_PAD;
    __syncthreads();
    const int nx = im.nx, nxy = im.nx * im.ny;
    for (int64_t base = ((int64_t)blockIdx.x * FILL_WARPS + warp) * 32; base < n;
         base += (int64_t)gridDim.x * FILL_WARPS * 32) {
        const int64_t k = base + lane;
        Ray r;
        VoxelCursor c;
        int64_t pos = 0, end = 0;
        float to_mm = 0.0f;
        c.done = true;
        c.ok = true;
        if (k < n) {
            lor_ray(r, sc, im, cs, lors[2 * k], lors[2 * k + 1]);
            cursor_start(r, c);
            pos = row_ptr[k];
            end = row_ptr[k + 1];
            to_mm = (float)(r.len_mm / FX);
        }
        bool bad = false;
        while (__any_sync(0xffffffffu, !c.done)) {
            int cnt = 0;
            while (cnt < 32 && !c.done) {
                int iz, iy, ix;
                long long ch;
                cursor_take(r, c, iz, iy, ix, ch);
                scol[lane * FILL_PAD + cnt] = iz * nxy + iy * nx + ix;
                sval[lane * FILL_PAD + cnt] = (float)ch * to_mm;
                ++cnt;
            }
            if (pos + cnt > end) {  // never for a consistent count pass; stay in the row
                bad = true;
                cnt = (int)(end - pos > 0 ? end - pos : 0);
            }
            __syncwarp();
            for (int j = 0; j < 32; ++j) {
                const int cj = __shfl_sync(0xffffffffu, cnt, j);
                const int64_t pj = __shfl_sync(0xffffffffu, pos, j);
                if (lane < cj) {
                    col[pj + lane] = scol[j * FILL_PAD + lane];
                    val[pj + lane] = sval[j * FILL_PAD + lane];
                }
            }
            pos += cnt;
            __syncwarp();
        }
        if (k < n && (!c.ok || bad || pos != end)) atomicExch(status, PSF_EDEBUG);
    }
}

// ---------------------------------------------------------------- K5 scan
constexpr int SCAN_T = 256, SCAN_V = 8, SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < (int)(blockDim.x >> 5)) sh[lane] = s;
    }
    __syncthreads();
    int64_t r = v + (w > 0 ? sh[w - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) scan_tiles_kernel(const int64_t *__restrict__ x,
                                                            int64_t n,
                                                            int64_t *__restrict__ tile_sums) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
    int64_t s = 0;
    for (int j = 0; j < SCAN_V; ++j)
        if (base + j < n) s += x[base + j];
    int64_t inc = block_incl_scan(s, sh);
    if (threadIdx.x == blockDim.x - 1) tile_sums[blockIdx.x] = inc;
}

__global__ void __launch_bounds__(SCAN_T) scan_sums_kernel(int64_t *__restrict__ sums,
                                                           int64_t nt) {
    __shared__ int64_t sh[32];
    __shared__ int64_t last;
    int64_t carry = 0;
    for (int64_t b = 0; b < nt; b += SCAN_T) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < nt ? sums[i] : 0;
        int64_t inc = block_incl_scan(v, sh);
        if (i < nt) sums[i] = carry + inc - v;  // exclusive
        if (threadIdx.x == blockDim.x - 1) last = inc;
        __syncthreads();
        carry += last;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_T) scan_apply_kernel(int64_t *__restrict__ x, int64_t n,
                                                            const int64_t *__restrict__ offs) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
    int64_t v[SCAN_V];
    int64_t s = 0;
    for (int j = 0; j < SCAN_V; ++j) {
        v[j] = base + j < n ? x[base + j] : 0;
        s += v[j];
    }
    int64_t inc = block_incl_scan(s, sh);
    int64_t run = offs[blockIdx.x] + inc - s;
    for (int j = 0; j < SCAN_V; ++j) {
        run += v[j];
        if (base + j < n) x[base + j] = run;
    }
}

// In-place inclusive scan of x[0..n) (int64); tile_sums has ceil(n/TILE) slots.
static int inclusive_scan(int64_t *x, int64_t n, int64_t *tile_sums, cudaStream_t st) {
    if (n <= 0) return PSF_OK;
    int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    scan_tiles_kernel<<<(unsigned)nt, SCAN_T, 0, st>>>(x, n, tile_sums);
    PSF_LAUNCHED();
    scan_sums_kernel<<<1, SCAN_T, 0, st>>>(tile_sums, nt);
    PSF_LAUNCHED();
    scan_apply_kernel<<<(unsigned)nt, SCAN_T, 0, st>>>(x, n, tile_sums);
    PSF_LAUNCHED();
    return PSF_OK;
}

// ---------------------------------------------------------------- K7 merge
__global__ void pair_map_kernel(const int32_t *__restrict__ lors, int64_t n, int64_t nc,
                                int32_t *__restrict__ map) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = lors[2 * k], b = lors[2 * k + 1];
        if (a >= 0 && b >= 0 && a < nc && b < nc) map[a * nc + b] = (int32_t)k;
    }
}

template <typename VT>
__device__ __forceinline__ VT to_val(float v);
template <>
__device__ __forceinline__ float to_val<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_val<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half to_val<__half>(float v) { return __float2half_rn(v); }

constexpr int MERGE_T = 256;

// pass 0: counts[m] = nnz of row m;  pass 1: write row m.
template <typename VT>
__global__ void __launch_bounds__(MERGE_T) merge_kernel(
    int pass, Scan sc, int64_t nvox, const int32_t *__restrict__ lors, int64_t n,
    const int32_t *__restrict__ map, const int64_t *__restrict__ gptr,
    const int32_t *__restrict__ gcol, const float *__restrict__ gval,
    const float *__restrict__ w, int Wt, int Wa, int64_t *__restrict__ counts_or_ptr,
    int32_t *__restrict__ col, VT *__restrict__ val, float *__restrict__ row_scale) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int E = (2 * Wt + 1) * (2 * Wa + 1), W2a = 2 * Wa + 1;
    const int NC = 2 * E * E;
    float *acc = (float *)smraw;                         // [nvox]
    int32_t *src = (int32_t *)(acc + nvox);              // [NC] source row or -1
    float *sw = (float *)(src + NC);                     // [NC] weight
    int *red = (int *)(sw + NC);                         // [MERGE_T/32 + 2]
    float *redf = (float *)(red + MERGE_T / 32 + 2);     // [MERGE_T/32]
    const int64_t nc = (int64_t)sc.Nt * sc.NR;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int64_t m = blockIdx.x; m < n; m += gridDim.x) {
        for (int64_t v = t; v < nvox; v += MERGE_T) acc[v] = 0.0f;
        const int X = lors[2 * m], Y = lors[2 * m + 1];
        const int rX = X / sc.Nt, tX = X - rX * sc.Nt;
        const int rY = Y / sc.Nt, tY = Y - rY * sc.Nt;
        for (int c = t; c < NC; c += MERGE_T) {
            int cs = c / (E * E), e = c - cs * E * E;
            int e1 = e / E, e2 = e - e1 * E;
            int dt1 = e1 / W2a - Wt, da1 = e1 % W2a - Wa;
            int dt2 = e2 / W2a - Wt, da2 = e2 % W2a - Wa;
            // case 0: source end1 lands on X, end2 on Y; case 1: end1 on Y, end2 on X
            int t1 = cs ? tY : tX, r1 = cs ? rY : rX;
            int t2 = cs ? tX : tY, r2 = cs ? rX : rY;
            int g1t = ((t1 - dt1) % sc.Nt + sc.Nt) % sc.Nt, g1r = r1 - da1;
            int g2t = ((t2 - dt2) % sc.Nt + sc.Nt) % sc.Nt, g2r = r2 - da2;
            int32_t row = -1;
            float wv = 0.0f;
            if (g1r >= 0 && g1r < sc.NR && g2r >= 0 && g2r < sc.NR) {
                int64_t g1 = (int64_t)g1r * sc.Nt + g1t, g2 = (int64_t)g2r * sc.Nt + g2t;
                if (g1 != g2) {
                    row = map[g1 * nc + g2];
                    if (row >= 0) {
                        wv = w[(int64_t)row * E * E + e];
                        if (!(wv > 0.0f) || gptr[row + 1] == gptr[row]) row = -1;
                    }
                }
            }
            src[c] = row;
            sw[c] = wv;
        }
        __syncthreads();
        // accumulate the sources in candidate order (deterministic)
        for (int c = 0; c < NC; ++c) {
            int32_t row = src[c];
            if (row < 0) continue;
            float wv = sw[c];
            for (int64_t j = gptr[row] + t; j < gptr[row + 1]; j += MERGE_T)
                acc[gcol[j]] += wv * gval[j];
            __syncthreads();
        }
        // compact non-zeros in ascending voxel order
        int64_t per = (nvox + MERGE_T - 1) / MERGE_T;
        int64_t v0 = t * per, v1 = v0 + per < nvox ? v0 + per : nvox;
        int cnt = 0;
        float mx = 0.0f;
        for (int64_t v = v0; v < v1; ++v) {
            float a = acc[v];
            cnt += a > 0.0f;
            mx = fmaxf(mx, a);
        }
        int inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int tt = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += tt;
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 31) red[warp] = inc;
        if (lane == 0) redf[warp] = mx;
        __syncthreads();
        int before = 0, total = 0;
        float rmax = 0.0f;
        for (int w2 = 0; w2 < MERGE_T / 32; ++w2) {
            if (w2 < warp) before += red[w2];
            total += red[w2];
            rmax = fmaxf(rmax, redf[w2]);
        }
        if (pass == 0) {
            if (t == 0) counts_or_ptr[m] = total;
        } else {
            int64_t pos = counts_or_ptr[m] + before + inc - cnt;
            float scale = 1.0f, inv = 1.0f;
            if (row_scale) {
                scale = rmax > 0.0f ? rmax : 1.0f;
                inv = 1.0f / scale;
                if (t == 0) row_scale[m] = scale;
            }
            for (int64_t v = v0; v < v1; ++v) {
                float a = acc[v];
                if (a > 0.0f) {
                    col[pos] = (int32_t)v;
                    val[pos] = to_val<VT>(row_scale ? a * inv : a);
                    ++pos;
                }
            }
        }
        __syncthreads();
    }
}

static int sm_count() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Geometric rows into (row_ptr, col, val); col == NULL: counts + scan only.
static int geom_rows(const Scan &sc, const Img &im, const int32_t *lors, int64_t n,
                     int64_t *row_ptr, int32_t *col, float *val, int64_t capacity,
                     int64_t *nnz_out, int64_t *tile_sums, int *status, cudaStream_t st) {
    const size_t shm = sizeof(double) * 2 * sc.R;
    const int grid = sm_count() * 16;
    PSF_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
    g_count_kernel<<<grid, ROWS_THREADS, shm, st>>>(sc, im, lors, n, row_ptr + 1, status);
    PSF_LAUNCHED();
    int rc = inclusive_scan(row_ptr + 1, n, tile_sums, st);
    if (rc) return rc;
    int64_t nnz = 0;
    int h_status = 0;
    PSF_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PSF_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSF_TRY(cudaStreamSynchronize(st));
    *nnz_out = nnz;
    if (h_status) return h_status;
    if (!col) return PSF_OK;
    if (nnz > capacity) return PSF_ECAPACITY;
    const size_t fshm = shm + sizeof(int32_t) * 2 * FILL_WARPS * 32 * FILL_PAD;
    PSF_TRY(cudaFuncSetAttribute(g_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fshm));
    int64_t fgrid = (n + FILL_WARPS * 32 - 1) / (FILL_WARPS * 32);
    if (fgrid > (int64_t)sm_count() * 3) fgrid = (int64_t)sm_count() * 3;
    g_fill_kernel<<<(int)fgrid, FILL_WARPS * 32, fshm, st>>>(sc, im, lors, n, row_ptr, col, val,
                                                            status);
    PSF_LAUNCHED();
    PSF_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSF_TRY(cudaStreamSynchronize(st));
    return h_status;
}

}  // namespace psf

using namespace psf;

extern "C" int psf_sysmat_rows(const psf_scanner *scanner, const psf_image *image,
                               const int32_t *lors, int64_t n_lors, const float *spread,
                               int32_t half_t, int32_t half_a, int32_t dtype, int64_t *row_ptr,
                               int32_t *col, void *val, float *row_scale, int64_t capacity,
                               int64_t *nnz_out, void *stream) {
    Scan sc;
    Img im;
    int rc = make_scan(scanner, &sc);
    if (rc) return rc;
    rc = make_img(image, &im);
    if (rc) return rc;
    if (!nnz_out || !row_ptr || n_lors < 0) return PSF_EINVAL;
    if (dtype < PSF_F32 || dtype > PSF_F16) return PSF_EINVAL;
    if ((dtype == PSF_F32) != (row_scale == nullptr)) return PSF_EINVAL;
    if (col && !val) return PSF_EINVAL;
    if (n_lors > 0 && !lors) return PSF_EINVAL;
    cudaStream_t st = as_stream(stream);
    const int64_t nvox = (int64_t)im.nx * im.ny * im.nz;
    const int64_t ntiles = (n_lors + SCAN_TILE - 1) / SCAN_TILE + 1;
    *nnz_out = 0;
    if (!spread) {
        if (dtype != PSF_F32) return PSF_EINVAL;  // geometric rows are stored in FP32
        if (n_lors == 0) {
            PSF_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
            return PSF_OK;
        }
        void *scratch = nullptr;
        size_t bytes = sizeof(int64_t) * ntiles + 256;
        PSF_TRY(cudaMallocAsync(&scratch, bytes, st));
        int *status = (int *)((char *)scratch + sizeof(int64_t) * ntiles);
        cudaMemsetAsync(status, 0, sizeof(int), st);
        rc = geom_rows(sc, im, lors, n_lors, row_ptr, col, (float *)val, capacity, nnz_out,
                       (int64_t *)scratch, status, st);
        cudaFreeAsync(scratch, st);
        return rc;
    }
    // PSF rows A = S G, merged densely per output row
    if (half_t < 0 || half_a < 0) return PSF_EINVAL;
    const int E = (2 * half_t + 1) * (2 * half_a + 1);
    const int64_t nc = (int64_t)sc.Nt * sc.NR;
    if (nvox > 49152 || E * E > 2401 || nc > 4096) return PSF_EINVAL;
    if (n_lors == 0) {
        PSF_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
        return PSF_OK;
    }
    // scratch: G (ptr, col, val), pair map, scan tiles, status
    int64_t gnnz = 0;
    int64_t *gptr = nullptr;
    void *misc = nullptr;
    size_t misc_bytes = sizeof(int64_t) * ntiles + sizeof(int32_t) * nc * nc + 256;
    PSF_TRY(cudaMallocAsync(&gptr, sizeof(int64_t) * (n_lors + 1), st));
    PSF_TRY(cudaMallocAsync(&misc, misc_bytes, st));
    int64_t *tiles = (int64_t *)misc;
    int32_t *map = (int32_t *)(tiles + ntiles);
    int *status = (int *)(map + nc * nc);
    cudaMemsetAsync(status, 0, sizeof(int), st);
    int32_t *gcol = nullptr;
    float *gval = nullptr;
    rc = geom_rows(sc, im, lors, n_lors, gptr, nullptr, nullptr, 0, &gnnz, tiles, status, st);
    if (!rc) {
        if (cudaMallocAsync(&gcol, sizeof(int32_t) * (gnnz + 1), st) != cudaSuccess ||
            cudaMallocAsync(&gval, sizeof(float) * (gnnz + 1), st) != cudaSuccess)
            rc = PSF_ECUDA;
    }
    if (!rc)
        rc = geom_rows(sc, im, lors, n_lors, gptr, gcol, gval, gnnz, &gnnz, tiles, status, st);
    if (!rc) {
        cudaMemsetAsync(map, 0xff, sizeof(int32_t) * nc * nc, st);
        pair_map_kernel<<<grid_for(n_lors, 256), 256, 0, st>>>(lors, n_lors, nc, map);
        size_t shm = sizeof(float) * nvox + (sizeof(int32_t) + sizeof(float)) * 2 * E * E +
                     sizeof(int) * (MERGE_T / 32 + 2) + sizeof(float) * (MERGE_T / 32) + 16;
        int grid = sm_count() * 4;
        auto launch = [&](int pass, auto *vptr) -> int {
            using VT = std::remove_pointer_t<decltype(vptr)>;
            PSF_TRY(cudaFuncSetAttribute(merge_kernel<VT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
            merge_kernel<VT><<<grid, MERGE_T, shm, st>>>(
                pass, sc, nvox, lors, n_lors, map, gptr, gcol, gval, spread, half_t, half_a,
                pass == 0 ? row_ptr + 1 : row_ptr, col, vptr, row_scale);
            PSF_LAUNCHED();
            return PSF_OK;
        };
        cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st);
        rc = launch(0, (float *)nullptr);
        if (!rc) rc = inclusive_scan(row_ptr + 1, n_lors, tiles, st);
        int64_t nnz = 0;
        if (!rc) {
            if (cudaMemcpyAsync(&nnz, row_ptr + n_lors, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = PSF_ECUDA;
            *nnz_out = nnz;
        }
        if (!rc && col) {
            if (nnz > capacity) {
                rc = PSF_ECAPACITY;
            } else if (dtype == PSF_F32) {
                rc = launch(1, (float *)val);
            } else if (dtype == PSF_BF16) {
                rc = launch(1, (__nv_bfloat16 *)val);
            } else {
                rc = launch(1, (__half *)val);
            }
        }
    }
    if (gcol) cudaFreeAsync(gcol, st);
    if (gval) cudaFreeAsync(gval, st);
    cudaFreeAsync(gptr, st);
    cudaFreeAsync(misc, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = PSF_ECUDA;
    return rc;
}
