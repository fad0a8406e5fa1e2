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
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "psf_common.cuh"
#include "psf_lorset.cuh"
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
__host__ __device__ __forceinline__ void face_centre(const Scan &sc, const double *cs, int id, double &x,
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
            to_mm = r.len_mm * (float)(1.0 / FX);
        }
        bool bad = false;
        while (__any_sync(0xffffffffu, !c.done)) {
            int cnt = 0;
            while (cnt < 32 && !c.done) {
                int iz, iy, ix;
                long long ch;
                cursor_take(r, c, iz, iy, ix, ch);
                scol[lane * FILL_PAD + cnt] = iz * nxy + iy * nx + ix;
                sval[lane * FILL_PAD + cnt] = units_to_f(ch) * to_mm;
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

// ------------------------------------------- rows traced on the fly
// One thread per row (the per-LOR tracer is sequential along the ray); the
// row of the set is decoded into its crystal pair, traced, and each voxel's
// chord is used at once instead of being stored.
template <bool BACK>
__global__ void __launch_bounds__(ROWS_THREADS) otf_rows_kernel(
    Scan sc, Img im, LorSet ls, const int32_t *__restrict__ list,
    const unsigned long long *__restrict__ count, const float *__restrict__ in,
    float *__restrict__ out, int *__restrict__ status) {
    extern __shared__ double cs[];
    int32_t *tp_start = reinterpret_cast<int32_t *>(cs + 2 * sc.R);
    int32_t *rp_start = tp_start + ls.Nt + 1;
    stage_blocks(sc, cs);
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    const int64_t nl = list ? (int64_t)*count : ls.ntp * ls.nrp;
    const int nx = im.nx, nxy = im.nx * im.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = list ? list[i] : i;
        const float yr = BACK ? in[row] : 0.0f;
        if (BACK && yr == 0.0f) continue;
        const int64_t T = row / ls.nrp;
        int a, b, ra, rb;
        ls.tp_decode(tp_start, T, &a, &b);
        ls.rp_decode(rp_start, row - T * ls.nrp, &ra, &rb);
        Ray r;
        lor_ray(r, sc, im, cs, ra * ls.Nt + a, rb * ls.Nt + b);
        const float to_mm = r.len_mm * (float)(1.0 / FX);
        float acc = 0.0f;
        const bool ok = trace_rows(r, [&](int iz, int iy, int x0, int x1, long long lo,
                                          long long hi) {
            const int base = iz * nxy + iy * nx;
            for (int ix = x0; ix <= x1; ++ix) {
                const float ch = units_to_f(chord_in_row(r.ax[0], ix, lo, hi)) * to_mm;
                if (BACK)
                    atomicAdd(out + base + ix, ch * yr);
                else
                    acc = fmaf(ch, __ldg(in + base + ix), acc);
            }
        });
        if (!ok) atomicExch(status, PSF_EDEBUG);
        if (!BACK) out[row] = acc;
    }
}

static int sm_count();

template <bool BACK>
static int otf_launch(const Scan &sc, const Img &im, const LorSet &ls, const int32_t *list,
                      const unsigned long long *count, const float *in, float *out, int *status,
                      cudaStream_t st) {
    const size_t shm = sizeof(double) * 2 * sc.R + sizeof(int32_t) * (ls.Nt + ls.NR + 2);
    {
        PSF_TIMED(BACK ? "otf_rows_kernel<back>" : "otf_rows_kernel<forward>", st);
        otf_rows_kernel<BACK><<<sm_count() * 16, ROWS_THREADS, shm, st>>>(sc, im, ls, list, count,
                                                                          in, out, status);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

int otf_rows_fwd(const Scan &sc, const Img &im, const LorSet &ls, const int32_t *list,
                 const unsigned long long *count, const float *x, float *y, int *status,
                 cudaStream_t st) {
    return otf_launch<false>(sc, im, ls, list, count, x, y, status, st);
}

int otf_rows_back(const Scan &sc, const Img &im, const LorSet &ls, const int32_t *list,
                  const unsigned long long *count, const float *y, float *x, int *status,
                  cudaStream_t st) {
    return otf_launch<true>(sc, im, ls, list, count, y, x, status, st);
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

int64_t scan_tile_count(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// In-place inclusive scan of x[0..n) (int64); tile_sums has ceil(n/TILE) slots.
int inclusive_scan(int64_t *x, int64_t n, int64_t *tile_sums, cudaStream_t st) {
    if (n <= 0) return PSF_OK;
    int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    {
        PSF_TIMED("scan_tiles_kernel", st);
        scan_tiles_kernel<<<(unsigned)nt, SCAN_T, 0, st>>>(x, n, tile_sums);
    }
    PSF_LAUNCHED();
    {
        PSF_TIMED("scan_sums_kernel", st);
        scan_sums_kernel<<<1, SCAN_T, 0, st>>>(tile_sums, nt);
    }
    PSF_LAUNCHED();
    {
        PSF_TIMED("scan_apply_kernel", st);
        scan_apply_kernel<<<(unsigned)nt, SCAN_T, 0, st>>>(x, n, tile_sums);
    }
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
    {
        PSF_TIMED("g_count_kernel", st);
        g_count_kernel<<<grid, ROWS_THREADS, shm, st>>>(sc, im, lors, n, row_ptr + 1, status);
    }
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
    {
        PSF_TIMED("g_fill_kernel", st);
        g_fill_kernel<<<(int)fgrid, FILL_WARPS * 32, fshm, st>>>(sc, im, lors, n, row_ptr, col, val,
                                                                status);
    }
    PSF_LAUNCHED();
    PSF_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSF_TRY(cudaStreamSynchronize(st));
    return h_status;
}

// ------------------------------------------------- rows of a structured set
// One CTA per transaxial pair.  Its segment's transaxial projection is the
// same for every ring pair, and so are the fixed-point parameters of its x
// and y plane crossings.  One thread builds the ordered list of 2D cells
// (x, y voxel and parameter interval, contiguous and non-empty) once; every
// ring pair then cuts the list at its own z-plane crossings.  A voxel's
// parameter interval is the intersection of its three slabs, exactly as in
// the per-LOR tracer, so the rows are the same numbers.
constexpr int SET_T = 256;
constexpr int SET_MAXC = 1024;  // 2D cells per transaxial pair (nx + ny + 1 <= 1024)
constexpr int SET_MAXF = 64;    // short cells checked one by one against each ring pair

struct Cells2D {
    long long *bnd;  // [n + 1] parameter boundaries
    short *ix, *iy;  // [n] voxel of each cell
    short *run;      // [n] run (constant iy) of each cell
    short *rstart;   // [nruns + 1] first cell of each run
    short *flag;     // [nflag] cells shorter than twice the transaxial chord threshold
    short *tie;      // [ny crossings + 1] parallel build: prefix of x/y plane ties
    int *hdr;        // n, nruns, nflag, ok; parallel build: crossings and first voxels
    Axis *X, *Y;
    long long *clip;  // amin2, amax2
    double *xy;       // endpoints (x1, y1, x2, y2)
};

// Shared-memory layout, widest fields first so every field is naturally
// aligned (the 8-byte fields sit at multiples of 8 from a 16-aligned base, the
// int header at a multiple of 8, the shorts after it).
__host__ __device__ __forceinline__ unsigned char *cells_layout(Cells2D &c, unsigned char *p) {
    c.bnd = reinterpret_cast<long long *>(p);
    p += sizeof(long long) * (SET_MAXC + 1);
    c.clip = reinterpret_cast<long long *>(p);  // amin, amax, short-cell threshold, -
    p += sizeof(long long) * 4;
    c.xy = reinterpret_cast<double *>(p);
    p += sizeof(double) * 4;
    c.X = reinterpret_cast<Axis *>(p);
    p += sizeof(Axis);
    c.Y = reinterpret_cast<Axis *>(p);
    p += sizeof(Axis);
    c.hdr = reinterpret_cast<int *>(p);
    p += sizeof(int) * 16;
    c.ix = reinterpret_cast<short *>(p);
    p += sizeof(short) * SET_MAXC;
    c.iy = reinterpret_cast<short *>(p);
    p += sizeof(short) * SET_MAXC;
    c.run = reinterpret_cast<short *>(p);
    p += sizeof(short) * SET_MAXC;
    c.rstart = reinterpret_cast<short *>(p);
    p += sizeof(short) * (SET_MAXC + 1);
    c.flag = reinterpret_cast<short *>(p);
    p += sizeof(short) * SET_MAXF;
    c.tie = reinterpret_cast<short *>(p);
    p += sizeof(short) * (SET_MAXC + 1);
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
}

static size_t cells_bytes() {
    return sizeof(long long) * (SET_MAXC + 5) + sizeof(double) * 4 + 2 * sizeof(Axis) +
           sizeof(short) * (5 * SET_MAXC + 2 + SET_MAXF) + sizeof(int) * 16 + 32;
}

// Segment of transaxial pair (a, b) in the transaxial plane: endpoints,
// x/y axes, clipped parameter interval [amin, amax) and the short-cell
// threshold.  Returns false when the segment misses the grid.
__host__ __device__ bool cells_setup(const Scan &sc, const Img &im, const double *cs, int a,
                                     int b, Cells2D &c, long long &amin, long long &amax) {
    double px, py, pz, qx, qy, qz;
    face_centre(sc, cs, a, px, py, pz);
    face_centre(sc, cs, b, qx, qy, qz);
    c.xy[0] = px;
    c.xy[1] = py;
    c.xy[2] = qx;
    c.xy[3] = qy;
    bool empty = false;
    Axis &X = *c.X, &Y = *c.Y;
    make_axis(X, (px - im.ox) * im.idx, (qx - im.ox) * im.idx, im.nx, empty);
    make_axis(Y, (py - im.oy) * im.idy, (qy - im.oy) * im.idy, im.ny, empty);
    amin = 0;
    amax = (long long)FX;
    for (int k = 0; k < 2; ++k) {
        const Axis &A = k ? Y : X;
        if (A.kind == 0) continue;
        long long p = plane_alpha(A, 0), q = plane_alpha(A, A.n);
        long long lo = p < q ? p : q, hi = p < q ? q : p;
        amin = lo > amin ? lo : amin;
        amax = hi < amax ? hi : amax;
    }
    c.clip[0] = amin;
    c.clip[1] = amax;
    c.clip[2] = 0;
    if (empty || amax <= amin) return false;
    const float lx = (float)(qx - px), ly = (float)(qy - py);
    const float len2 = sqrtf(lx * lx + ly * ly);
    // the 3D threshold is at most the transaxial one (3D segments are longer)
    c.clip[2] = 2 * (long long)ceilf((float)MIN_CHORD_MM / len2 * (float)FX);
    return true;
}

// One thread: the 2D cells of transaxial pair (a, b) by walking the x and y
// plane crossings in ray order (the reference for the parallel build).
__host__ __device__ void build_cells(const Scan &sc, const Img &im, const double *cs, int a, int b,
                            Cells2D &c) {
    long long amin, amax;
    const bool live = cells_setup(sc, im, cs, a, b, c, amin, amax);
    const Axis &X = *c.X, &Y = *c.Y;
    int n = 0, nruns = 0, nflag = 0;
    bool ok = true;
    if (live) {
        int cx, cy;
        ok &= voxel_at(X, amin, cx);
        ok &= voxel_at(Y, amin, cy);
        long long cur = amin;
        c.bnd[0] = amin;
        const long long thr2 = c.clip[2];
        for (int it = 0; it < im.nx + im.ny + 4 && n < SET_MAXC; ++it) {
            long long lo, ex_, ey_;
            if (X.kind == 0) ex_ = FX_BIG; else slab(X, cx, lo, ex_);
            if (Y.kind == 0) ey_ = FX_BIG; else slab(Y, cy, lo, ey_);
            long long nxt = ex_ < ey_ ? ex_ : ey_;
            nxt = nxt < amax ? nxt : amax;
            if (nxt > cur) {
                c.ix[n] = (short)(cx < 0 ? 0 : (cx >= im.nx ? im.nx - 1 : cx));
                c.iy[n] = (short)(cy < 0 ? 0 : (cy >= im.ny ? im.ny - 1 : cy));
                if (n == 0 || c.iy[n] != c.iy[n - 1]) c.rstart[nruns++] = (short)n;
                c.run[n] = (short)(nruns - 1);
                if (nxt - cur < thr2) {
                    if (nflag < SET_MAXF) c.flag[nflag] = (short)n;
                    ++nflag;
                }
                ++n;
                c.bnd[n] = nxt;
            }
            if (nxt >= amax) break;
            if (ex_ == nxt) cx += X.inc ? 1 : -1;
            if (ey_ == nxt) cy += Y.inc ? 1 : -1;
            cur = nxt;
        }
        if (n >= SET_MAXC && c.bnd[n] < amax) ok = false;
    }
    c.rstart[nruns] = (short)n;
    c.hdr[0] = n;
    c.hdr[1] = nruns;
    c.hdr[2] = nflag;
    c.hdr[3] = ok;
    c.hdr[13] = float_bits(n > 0 ? (float)n / (float)(c.bnd[n] - c.bnd[0]) : 0.0f);
}

// Parameter of the i-th plane crossing (i >= 1) along the segment of an axis
// whose voxel at the start of the clipped interval is k0.
__host__ __device__ __forceinline__ long long crossing(const Axis &A, int k0, int i) {
    return plane_alpha(A, A.inc ? k0 + i : k0 + 1 - i);
}

#ifdef __CUDACC__
// Every thread of the CTA: the same cells as build_cells, built in parallel.
// The boundaries are the distinct x and y plane crossings inside the clipped
// interval in ray order.  Each crossing finds its rank in that order by
// counting the other axis's crossings before it (an exact voxel lookup at
// the parameter just below it), and a crossing where an x and a y plane meet
// (a tie) is counted once, through a prefix count of the tied y crossings.
// A cell's voxel is the voxel at its start, its run the number of y
// crossings before it.  Ends with a CTA barrier.
__device__ void build_cells_par(const Scan &sc, const Img &im, const double *cs, int a, int b,
                                Cells2D &c) {
    int *H = c.hdr;
    const Axis &X = *c.X, &Y = *c.Y;
    if (threadIdx.x == 0) {
        long long amin, amax;
        const bool live = cells_setup(sc, im, cs, a, b, c, amin, amax);
        int kx0 = 0, ky0 = 0, kx1 = 0, ky1 = 0;
        bool ok = true;
        if (live) {
            ok &= voxel_at(X, amin, kx0);
            ok &= voxel_at(X, amax - 1, kx1);
            ok &= voxel_at(Y, amin, ky0);
            ok &= voxel_at(Y, amax - 1, ky1);
        }
        const int nxc = live ? abs(kx1 - kx0) : 0, nyc = live ? abs(ky1 - ky0) : 0;
        H[0] = live ? 1 + nxc + nyc : 0;  // before ties
        H[2] = 0;
        H[3] = ok && 1 + nxc + nyc <= SET_MAXC;
        H[8] = kx0;
        H[9] = ky0;
        H[10] = nxc;
        H[11] = nyc;
        H[12] = live && H[3];
    }
    __syncthreads();
    const int kx0 = H[8], ky0 = H[9], nxc = H[10], nyc = H[11];
    const bool live = H[12];
    const int t = threadIdx.x, nt = blockDim.x;
    if (live) {
        // 1. tie flags of the y crossings
        for (int j = t + 1; j <= nyc; j += nt) {
            const long long P = crossing(Y, ky0, j);
            int v1 = 0, v0 = 0;
            voxel_at(X, P, v1);
            voxel_at(X, P - 1, v0);
            c.tie[j] = v1 != v0;
        }
    }
    __syncthreads();
    if (live && t < 32) {  // 2. inclusive prefix: tie[m] = tied crossings among y 1..m
        int carry = 0;
        for (int base = 1; base <= nyc; base += 32) {
            const int j = base + t;
            const int v = j <= nyc ? c.tie[j] : 0;
            int inc = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (t >= o) inc += u;
            }
            if (j <= nyc) c.tie[j] = (short)(carry + inc);
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (t == 0) c.tie[0] = 0;
    }
    __syncthreads();
    if (live) {  // 3. ranks -> boundaries, run starts
        for (int i = t + 1; i <= nxc; i += nt) {
            const long long P = crossing(X, kx0, i);
            int vy = 0;
            voxel_at(Y, P - 1, vy);
            const int ylt = abs(vy - ky0);
            c.bnd[(i - 1) + ylt - c.tie[ylt] + 1] = P;
        }
        for (int j = t + 1; j <= nyc; j += nt) {
            const long long P = crossing(Y, ky0, j);
            int vx = 0;
            voxel_at(X, P - 1, vx);
            const int r = (j - 1) + abs(vx - kx0) - c.tie[j - 1] + 1;
            c.bnd[r] = P;  // a tie writes the same value as its x crossing
            c.rstart[j] = (short)r;
        }
        if (t == 0) {
            const int n = 1 + nxc + nyc - c.tie[nyc];
            c.bnd[0] = c.clip[0];
            c.bnd[n] = c.clip[1];
            c.rstart[0] = 0;
            c.rstart[nyc + 1] = (short)n;
            H[0] = n;
            H[1] = nyc + 1;
            H[13] = __float_as_int((float)n / (float)(c.clip[1] - c.clip[0]));
        }
    } else if (t == 0) {
        H[0] = 0;
        H[1] = 0;
        H[13] = 0;
        c.rstart[0] = 0;
    }
    __syncthreads();
    const int n = H[0];
    const long long thr2 = c.clip[2];
    for (int cc = t; cc < n; cc += nt) {  // 4. cells
        const long long s0 = c.bnd[cc];
        int cx = 0, cy = 0;
        voxel_at(X, s0, cx);
        voxel_at(Y, s0, cy);
        c.ix[cc] = (short)(cx < 0 ? 0 : (cx >= im.nx ? im.nx - 1 : cx));
        c.iy[cc] = (short)(cy < 0 ? 0 : (cy >= im.ny ? im.ny - 1 : cy));
        c.run[cc] = (short)abs(cy - ky0);
        if (c.bnd[cc + 1] - s0 < thr2) {
            const int f = atomicAdd(&H[2], 1);
            if (f < SET_MAXF) c.flag[f] = (short)cc;
        }
    }
    __syncthreads();
}
#endif

// First cell whose interval ends after al / last cell that starts before al.
__host__ __device__ __forceinline__ int first_cell_after(const long long *bnd, int n, long long al) {
    int lo = 0, hi = n - 1;  // smallest c with bnd[c+1] > al
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (bnd[mid + 1] > al) hi = mid; else lo = mid + 1;
    }
    return lo;
}
__host__ __device__ __forceinline__ int last_cell_before(const long long *bnd, int n, long long al) {
    int lo = 0, hi = n - 1;  // largest c with bnd[c] < al
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (bnd[mid] < al) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ __forceinline__ long long piece(const long long *bnd, int cc, long long zl,
                                           long long zh) {
    long long lo = bnd[cc] > zl ? bnd[cc] : zl, hi = bnd[cc + 1] < zh ? bnd[cc + 1] : zh;
    return hi - lo;
}

}  // namespace psf

#include "psf_rows_set.cuh"

namespace psf {

// Per CTA: the cells of its current transaxial pair, block trig, set prefix
// tables, the cells again in voxel order (their packed x/y voxel, chord and
// chord as a float), and each warp's work area.
struct SetSmem {
    Cells2D c;
    double *cs;
    long long *s_len;   // [SET_MAXC] chord (units) of the cell at each voxel-order position
    int2 *s_xyl;        // [SET_MAXC] iy * nx + ix, chord as a float (bits, rounded once)
    int32_t *tp_start, *rp_start;
    int *next;          // next ring-pair group of the current transaxial pair
    unsigned long long *lmax;  // longest cell chord of the current pair (units)
    SetWarp *w;         // [SET_T / 32]
};

__device__ __forceinline__ void set_smem_layout(SetSmem &m, unsigned char *raw, const Scan &sc,
                                                const LorSet &ls) {
    m.cs = reinterpret_cast<double *>(cells_layout(m.c, raw));
    m.s_len = reinterpret_cast<long long *>(m.cs + 2 * sc.R);
    m.s_xyl = reinterpret_cast<int2 *>(m.s_len + SET_MAXC);
    m.tp_start = reinterpret_cast<int32_t *>(m.s_xyl + SET_MAXC);
    m.rp_start = m.tp_start + ls.Nt + 1;
    m.next = m.rp_start + ls.NR + 1;
    m.lmax = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(m.next + 1) + 7) & ~uintptr_t(7));
    m.w = reinterpret_cast<SetWarp *>(
        (reinterpret_cast<uintptr_t>(m.lmax + 1) + 15) & ~uintptr_t(15));
}

// The count kernel's layout: the pair's cells, block trig and prefix tables
// as above, without the voxel-order copies, and per warp only its rows and
// their counts.
struct CountWarp {
    int cnt[32];
    SlabRow row[32];
};

__device__ __forceinline__ CountWarp *count_smem_layout(SetSmem &m, unsigned char *raw,
                                                        const Scan &sc, const LorSet &ls) {
    m.cs = reinterpret_cast<double *>(cells_layout(m.c, raw));
    m.s_len = nullptr;
    m.s_xyl = nullptr;
    m.tp_start = reinterpret_cast<int32_t *>(m.cs + 2 * sc.R);
    m.rp_start = m.tp_start + ls.Nt + 1;
    m.next = m.rp_start + ls.NR + 1;
    m.lmax = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(m.next + 1) + 7) & ~uintptr_t(7));
    m.w = nullptr;
    return reinterpret_cast<CountWarp *>(
        (reinterpret_cast<uintptr_t>(m.lmax + 1) + 15) & ~uintptr_t(15));
}

static size_t count_smem(const Scan &sc, const LorSet &ls) {
    return cells_bytes() + sizeof(double) * 2 * sc.R + sizeof(int32_t) * (ls.Nt + ls.NR + 2) +
           sizeof(int) * 4 + 32 + sizeof(CountWarp) * (SET_T / 32) + 64;
}

static size_t set_smem(const Scan &sc, const LorSet &ls) {
    return cells_bytes() + sizeof(double) * 2 * sc.R +
           (sizeof(long long) + sizeof(int2)) * SET_MAXC +
           sizeof(int32_t) * (ls.Nt + ls.NR + 2) + sizeof(int) * 4 + 32 +
           sizeof(SetWarp) * (SET_T / 32) + 64;
}

// Ring-pair table of a set: entry j is the z axis of ring pair j's segments.
__global__ void __launch_bounds__(256) zaxis_kernel(Scan sc, Img im, LorSet ls,
                                                    ZAx *__restrict__ zt) {
    extern __shared__ int32_t zpre[];  // [Nt + 1 + NR + 1]
    ls.stage_prefix(zpre, zpre + ls.Nt + 1);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ls.nrp) return;
    int ra, rb;
    ls.rp_decode(zpre + ls.Nt + 1, j, &ra, &rb);
    zaxis_of(sc, im, ra, rb, zt[j]);
}

// Cache of the 2D cells of every transaxial pair in device memory: the count
// kernel stores each pair's cells as it builds them and the fill reads them
// back instead of building them a second time (base == nullptr: no cache,
// both kernels build).  A slot holds the header block (clip, endpoints, axes,
// header words: contiguous in the shared-memory layout), the boundaries, the
// cells' voxels and runs, the run starts and the short-cell list, for at most
// maxc = nx + ny + 1 cells.
struct CellCache {
    unsigned char *base;
    int maxc;
    int64_t stride;  // bytes per pair, a multiple of 16
};

constexpr int CELL_HEAD = 32 + 32 + 2 * (int)sizeof(Axis) + 64;  // clip .. hdr
static_assert(CELL_HEAD % 16 == 0, "cell cache header block");

__host__ __device__ inline int64_t cell_slot_bytes(int maxc) {
    const int64_t b = (int64_t)sizeof(long long) * (maxc + 1);
    const int64_t sh = (int64_t)sizeof(short) * (4 * maxc + 1 + SET_MAXF);
    return CELL_HEAD + ((b + 15) & ~15LL) + ((sh + 15) & ~15LL);
}

// Store (or, with load, read back) the current cells of the CTA; every thread
// calls.  The counts come from the header (clamped to the slot).
__device__ __forceinline__ void cells_copy(Cells2D &c, const CellCache &cc, int64_t T, bool load) {
    unsigned char *slot = cc.base + T * cc.stride;
    int *head_g = reinterpret_cast<int *>(slot);
    int *head_s = reinterpret_cast<int *>(c.clip);
    const int t = threadIdx.x, nt = blockDim.x;
    if (load) {
        for (int i = t; i < CELL_HEAD / 4; i += nt) head_s[i] = head_g[i];
        __syncthreads();
    } else {
        for (int i = t; i < CELL_HEAD / 4; i += nt) head_g[i] = head_s[i];
    }
    const int n = min(c.hdr[0], cc.maxc), nr = min(c.hdr[1], cc.maxc),
              nf = min(c.hdr[2], SET_MAXF);
    long long *bnd = reinterpret_cast<long long *>(slot + CELL_HEAD);
    short *sh = reinterpret_cast<short *>(
        slot + CELL_HEAD + ((sizeof(long long) * (cc.maxc + 1) + 15) & ~(size_t)15));
    short *ix = sh, *iy = sh + cc.maxc, *run = sh + 2 * cc.maxc, *rs = sh + 3 * cc.maxc,
          *fl = sh + 4 * cc.maxc + 1;
    if (load) {
        for (int i = t; i <= n; i += nt) c.bnd[i] = bnd[i];
        for (int i = t; i < n; i += nt) {
            c.ix[i] = ix[i];
            c.iy[i] = iy[i];
            c.run[i] = run[i];
        }
        for (int i = t; i <= nr; i += nt) c.rstart[i] = rs[i];
        for (int i = t; i < nf; i += nt) c.flag[i] = fl[i];
    } else {
        for (int i = t; i <= n; i += nt) bnd[i] = c.bnd[i];
        for (int i = t; i < n; i += nt) {
            ix[i] = c.ix[i];
            iy[i] = c.iy[i];
            run[i] = c.run[i];
        }
        for (int i = t; i <= nr; i += nt) rs[i] = c.rstart[i];
        for (int i = t; i < nf; i += nt) fl[i] = c.flag[i];
    }
}

// Per transaxial pair: the CTA builds the 2D cells (or reads them from the
// cache the count kernel filled), then every thread helps write the
// voxel-order copies: each cell's packed x/y voxel and its chord as
// a float -- in parameter units, or (norm: the 16-bit value forms) divided by
// the pair's longest cell chord, so that every stored value lies in (0, 1].
// Returns after the CTA barrier.
__device__ __forceinline__ void set_pair_cells(SetSmem &m, const Scan &sc, const Img &im,
                                               const LorSet &ls, int64_t T, int *status,
                                               bool norm, bool voxel_order,
                                               const CellCache &cache, bool load) {
    __syncthreads();  // the previous pair's readers are done
    const Cells2D &c = m.c;
    if (load) {
        cells_copy(m.c, cache, T, true);
        __syncthreads();
    } else {
        int a, b;
        ls.tp_decode(m.tp_start, T, &a, &b);
        build_cells_par(sc, im, m.cs, a, b, m.c);
        if (cache.base) cells_copy(m.c, cache, T, false);
    }
    if (threadIdx.x == 0) {
        if (!c.hdr[3]) atomicExch(status, PSF_EDEBUG);
        *m.next = 0;
        *m.lmax = 1;
    }
    __syncthreads();
    if (!voxel_order) return;  // (the count kernel cuts the ray-order cells only)
    if (norm) {
        unsigned long long mx = 1;
        for (int cc = threadIdx.x; cc < c.hdr[0]; cc += SET_T) {
            const unsigned long long L = (unsigned long long)(c.bnd[cc + 1] - c.bnd[cc]);
            mx = L > mx ? L : mx;
        }
        atomicMax(m.lmax, mx);
        __syncthreads();
    }
    const float lmax = units_to_f((long long)*m.lmax);
    const bool xinc = c.X->kind == 0 || c.X->inc;
    const bool yinc = c.Y->kind == 0 || c.Y->inc;
    for (int cc = threadIdx.x; cc < c.hdr[0]; cc += SET_T) {
        const int p = sorted_pos(c, cc, xinc, yinc, c.hdr[0]);
        const long long L = c.bnd[cc + 1] - c.bnd[cc];
        m.s_len[p] = L;
        const float lf = norm ? __fdiv_rn(units_to_f(L), lmax) : units_to_f(L);
        m.s_xyl[p] = make_int2((int)c.iy[cc] * im.nx + c.ix[cc], float_bits(lf));
    }
    __syncthreads();
}

// Value of a cut end cell (La units): mm, or (norm) as a fraction of the
// pair's longest cell chord lmax, like the interior cells.
__device__ __forceinline__ float end_value(long long La, float to_mm, bool norm, float lmax) {
    return norm ? __fdiv_rn(units_to_f(La), lmax) : units_to_f(La) * to_mm;
}

// Store of a row value in the output format (round to nearest).
template <typename VT>
__device__ __forceinline__ void st_val(VT *p, float v);
template <>
__device__ __forceinline__ void st_val<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void st_val<__nv_bfloat16>(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ void st_val<__half>(__half *p, float v) { *p = __float2half_rn(v); }

// Next group of 32 ring pairs for this warp (groups handed out in order).
__device__ __forceinline__ int set_next_group(int *next) {
    int g = 0;
    if ((threadIdx.x & 31) == 0) g = atomicAdd(next, 1);
    return __shfl_sync(0xffffffffu, g, 0);
}

// K4 (set): a warp takes 32 ring pairs of the CTA's transaxial pair; its
// lanes cut the z slabs of all of them, 32 slabs at a time, and add each
// slab's stored voxels to its ring pair's count.
__global__ void __launch_bounds__(SET_T, 4) set_count_kernel(Scan sc, Img im, LorSet ls,
                                                             const ZAx *__restrict__ zt,
                                                             int64_t *__restrict__ counts,
                                                             int *__restrict__ status,
                                                             CellCache cache) {
    extern __shared__ __align__(16) unsigned char raw[];
    SetSmem m;
    CountWarp *cw = count_smem_layout(m, raw, sc, ls);
    stage_blocks(sc, m.cs);
    ls.stage_prefix(m.tp_start, m.rp_start);
    const Cells2D &c = m.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    CountWarp &W = cw[warp];
    const int nrp = (int)ls.nrp, ngroups = (nrp + 31) / 32;
    for (int64_t T = blockIdx.x; T < ls.ntp; T += gridDim.x) {
        set_pair_cells(m, sc, im, ls, T, status, false, false, cache, false);
        const CellsHead hd = cells_head(c);
        const float lx = (float)(c.xy[2] - c.xy[0]), ly = (float)(c.xy[3] - c.xy[1]);
        for (int g = set_next_group(m.next); g < ngroups; g = set_next_group(m.next)) {
            const int j = g * 32 + lane;
            RingPair rp;
            rp_setup(c, zt, j, nrp, im.nz, lx, ly, rp);
            W.cnt[lane] = 0;
            int incl = rp.nsl;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            slab_row_put(rp, incl - rp.nsl, W.row[lane]);
            __syncwarp();
            for (int base = 0; base < total; base += 32) {
                SlabOf so;
                slab_of(W.row, incl, base + lane, total, so);
                if (so.q >= 0) {
                    const SlabCells s = cut_cells(c, hd, so.zl, so.zh, so.minu);
                    if (s.count) atomicAdd(&W.cnt[so.q], s.count);
                }
            }
            __syncwarp();
            if (j < nrp) counts[T * nrp + j] = W.cnt[lane];
            __syncwarp();
        }
    }
}

// Left shift that gives 0 for shift counts of 32 and more (PTX shl.b32
// clamps the count; a C++ shift by 32 is undefined).
__device__ __forceinline__ unsigned shl_clamped(unsigned v, int n) {
    unsigned r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(n));
    return r;
}

// General emission of one round (any keep pattern): a keep decision per cell
// and a ballot compaction of the kept entries.  Used for the rare rounds where
// a short interior cell of some slab is dropped.  Returns the entries stored.
template <typename VT>
__device__ __forceinline__ int fill_round_general(const SetSmem &m, SetWarp &W, const SlabOf &so,
                                               const SlabCells &s, bool xinc, bool yinc,
                                               int nxy, bool norm, float lmax, long long pos,
                                               long long pend, int32_t *__restrict__ col,
                                               VT *__restrict__ val) {
    const Cells2D &c = m.c;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u, le = (2u << lane) - 1u;
    int lo[3], hi[3], ns = 0;
    if (so.q >= 0 && s.cb >= s.ca) {
        ns = slab_segments(c, s.ca, s.cb, xinc, yinc, lo, hi, c.hdr[0]);
        const long long La = piece(c.bnd, s.ca, so.zl, so.zh);
        const long long Lb = piece(c.bnd, s.cb, so.zl, so.zh);
        W.gen.sa[lane] = make_int4(so.iz * nxy, sorted_pos(c, s.ca, xinc, yinc, c.hdr[0]),
                                   sorted_pos(c, s.cb, xinc, yinc, c.hdr[0]),
                                   (La >= so.minu) | ((Lb >= so.minu) << 1));
        W.gen.sf[lane] = make_float4(end_value(La, so.to_mm, norm, lmax),
                                     end_value(Lb, so.to_mm, norm, lmax),
                                     norm ? 1.0f : so.to_mm, 0.0f);
        W.gen.sm[lane] = so.minu;
    }
    int len = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (k < ns) len += hi[k] - lo[k] + 1;
    int inc_len = len, inc_seg = ns;
    for (int o = 1; o < 32; o <<= 1) {
        const int a1 = __shfl_up_sync(0xffffffffu, inc_len, o);
        const int a2 = __shfl_up_sync(0xffffffffu, inc_seg, o);
        if (lane >= o) {
            inc_len += a1;
            inc_seg += a2;
        }
    }
    const int total = __shfl_sync(0xffffffffu, inc_len, 31);
    const int nseg = __shfl_sync(0xffffffffu, inc_seg, 31);
    int off = inc_len - len;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (k < ns) {
            W.gen.rs[inc_seg - ns + k] = make_int2(off, lo[k] | (lane << 16));
            off += hi[k] - lo[k] + 1;
        }
    __syncwarp();
    const long long pos0 = pos;
    int gbase = -1;  // range holding the entry before the chunk
    for (int e0 = 0; e0 < total; e0 += 32) {
        const int gq = gbase + 1 + lane;
        unsigned bit = 0u;
        if (gq < nseg) {
            const int st = W.gen.rs[gq].x - e0;
            if (st < 32) bit = 1u << st;
        }
        const unsigned B = __reduce_or_sync(0xffffffffu, bit);
        const int e = e0 + lane;
        bool keep = false;
        int colv = 0;
        float v = 0.0f;
        if (e < total) {
            const int gi = gbase + __popc(B & le);
            const int2 R = W.gen.rs[gi];
            const int p = (R.y & 0xffff) + (e - R.x), k = R.y >> 16;
            const int4 A = W.gen.sa[k];
            const float4 F = W.gen.sf[k];
            const int2 xl = m.s_xyl[p];
            // end cells take their cut chord and keep bit; interior cells
            // their 2D chord, kept unless shorter than the row's threshold
            const bool isa = p == A.y, isb = p == A.z;
            v = isa ? F.x : (isb ? F.y : __int_as_float(xl.y) * F.z);
            keep = isa ? (A.w & 1) : (isb ? ((A.w >> 1) & 1) : m.s_len[p] >= W.gen.sm[k]);
            colv = A.x + xl.x;
        }
        gbase += __popc(B);
        const unsigned msk = __ballot_sync(0xffffffffu, keep);
        const long long wpos = pos + __popc(msk & lt);
        if (keep && wpos < pend) {
            col[wpos] = colv;
            st_val(val + wpos, v);
        }
        pos += __popc(msk);
    }
    __syncwarp();
    return (int)(pos - pos0);
}

// K6 (set): the same walk.  Each round's slabs become at most three
// voxel-order ranges each (a slab's first and last ray-order cells, cut by the
// z planes, are always range endpoints, so a dropped end cell only trims its
// range; one range when the segment's x and y directions have the same sign,
// voxel order then being ray order or its reverse), laid end to end; the lanes
// then copy that flattened list 32 entries
// at a time onto consecutive slots -- column = slab base + the cell's packed
// x/y voxel, value = the cell's 2D chord x the row's mm per unit -- and the
// slab lanes finally overwrite the values of the kept end cells with their cut
// chords.  A round in which some slab drops a short interior cell takes the
// general per-cell path.  The 32 rows of a group are consecutive in the CSR,
// so the whole group is one contiguous output span.
template <typename VT>
__global__ void __launch_bounds__(SET_T, 3) set_fill_kernel(Scan sc, Img im, LorSet ls,
                                                            const ZAx *__restrict__ zt,
                                                            const int64_t *__restrict__ row_ptr,
                                                            int32_t *__restrict__ col,
                                                            VT *__restrict__ val,
                                                            float *__restrict__ row_scale,
                                                            int *__restrict__ status,
                                                            CellCache cache) {
    // FP32 values are chords in mm; the 16-bit forms store chord / row scale
    // with row scale = (pair's longest cell chord) x (row's mm per unit)
    constexpr bool norm = !std::is_same<VT, float>::value;
    extern __shared__ __align__(16) unsigned char raw[];
    SetSmem m;
    set_smem_layout(m, raw, sc, ls);
    stage_blocks(sc, m.cs);
    ls.stage_prefix(m.tp_start, m.rp_start);
    const Cells2D &c = m.c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SetWarp &W = m.w[warp];
    const unsigned le = (2u << lane) - 1u;
    const int nrp = (int)ls.nrp, ngroups = (nrp + 31) / 32;
    const int nxy = im.nx * im.ny;
    for (int64_t T = blockIdx.x; T < ls.ntp; T += gridDim.x) {
        set_pair_cells(m, sc, im, ls, T, status, norm, true, cache, cache.base != nullptr);
        const float lx = (float)(c.xy[2] - c.xy[0]), ly = (float)(c.xy[3] - c.xy[1]);
        const bool xinc = c.X->kind == 0 || c.X->inc;
        const bool yinc = c.Y->kind == 0 || c.Y->inc;
        const float lmax = units_to_f((long long)*m.lmax);
        for (int g = set_next_group(m.next); g < ngroups; g = set_next_group(m.next)) {
            const int j0 = g * 32, j = j0 + lane;
            const int nq = nrp - j0 < 32 ? nrp - j0 : 32;
            RingPair rp;
            rp_setup(c, zt, j, nrp, im.nz, lx, ly, rp);
            int incl = rp.nsl;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total_slabs = __shfl_sync(0xffffffffu, incl, 31);
            slab_row_put(rp, incl - rp.nsl, W.row[lane]);
            if (norm && j < nrp) row_scale[T * nrp + j] = lmax * rp.to_mm;
            long long pos = row_ptr[T * nrp + j0];
            const long long pend = row_ptr[T * nrp + j0 + nq];  // the group's span ends here
            __syncwarp();
            for (int base = 0; base < total_slabs; base += 32) {
                SlabOf so;
                slab_of(W.row, incl, base + lane, total_slabs, so);
                SlabCells s;
                s.ca = 0;
                s.cb = -1;
                s.inner = 0;
                // (the header words are re-read per slab here: holding them in
                // registers across the round costs the fill more in spills)
                if (so.q >= 0) s = cut_cells(c, cells_head(c), so.zl, so.zh, so.minu);
                if (__any_sync(0xffffffffu, s.inner > 0)) {
                    pos += fill_round_general(m, W, so, s, xinc, yinc, nxy, norm, lmax, pos,
                                              pend, col, val);
                    continue;
                }
                // 1. this round's slabs -> trimmed voxel-order ranges, flattened
                int lo[3], hi[3], nr = 0, pa = 0, pb = 0;
                bool ka = false, kb = false;
                float va = 0.0f, vb = 0.0f;
                if (s.cb >= s.ca) {
                    if (xinc == yinc) {  // voxel order is ray order or its reverse
                        const int nc1 = c.hdr[0] - 1;
                        pa = xinc ? s.ca : nc1 - s.ca;
                        pb = xinc ? s.cb : nc1 - s.cb;
                        nr = 1;
                        lo[0] = pa < pb ? pa : pb;
                        hi[0] = pa < pb ? pb : pa;
                    } else {
                        nr = slab_segments(c, s.ca, s.cb, xinc, yinc, lo, hi, c.hdr[0]);
                        pa = sorted_pos(c, s.ca, xinc, yinc, c.hdr[0]);
                        pb = sorted_pos(c, s.cb, xinc, yinc, c.hdr[0]);
                    }
                    const long long La = piece(c.bnd, s.ca, so.zl, so.zh);
                    const long long Lb = piece(c.bnd, s.cb, so.zl, so.zh);
                    ka = La >= so.minu;
                    kb = s.cb != s.ca && Lb >= so.minu;
                    const bool drop_b = s.cb != s.ca && !kb;
                    va = end_value(La, so.to_mm, norm, lmax);
                    vb = end_value(Lb, so.to_mm, norm, lmax);
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (k < nr) {
                            if (!ka) {
                                if (pa == lo[k]) ++lo[k];
                                else if (pa == hi[k]) --hi[k];
                            }
                            if (drop_b) {
                                if (pb == lo[k]) ++lo[k];
                                else if (pb == hi[k]) --hi[k];
                            }
                        }
                }
                int ns = 0, len = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (k < nr && hi[k] >= lo[k]) {
                        ++ns;
                        len += hi[k] - lo[k] + 1;
                    }
                // one scan of (entries << 7 | ranges): at most 96 ranges a round
                int inc = (len << 7) | ns;
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t;
                }
                const int tot = __shfl_sync(0xffffffffu, inc, 31);
                const int total = tot >> 7, nseg = tot & 127;
                int off = (inc >> 7) - len, wr = (inc & 127) - ns;
                int sa = -1, sb = -1;  // round slots of the kept end cells
                const int colbase = so.iz * nxy,
                          mm = __float_as_int(norm ? 1.0f : so.to_mm);  // value per stored chord
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (k < nr && hi[k] >= lo[k]) {
                        W.cp.start[wr] = off;
                        W.cp.rec[wr] = make_int4(lo[k] - off, colbase, mm, 0);
                        if (pa >= lo[k] && pa <= hi[k]) sa = off + pa - lo[k];
                        if (pb >= lo[k] && pb <= hi[k]) sb = off + pb - lo[k];
                        off += hi[k] - lo[k] + 1;
                        ++wr;
                    }
                W.cp.start[nseg + lane] = 0x7fffffff;  // no range starts past the last
                __syncwarp();
                // 2. every lane copies one cell per step; the ranges starting
                // inside each 32-entry chunk are found with one OR-reduction
                const long long room = pend - pos;
                const int lim = room < (long long)total ? (int)room : total;
                int32_t *cdst = col + pos;
                VT *vdst = val + pos;
                int gbase = -1;  // range holding the entry before the chunk
#pragma unroll 2
                for (int e0 = 0; e0 < total; e0 += 32) {
                    const unsigned B = __reduce_or_sync(
                        0xffffffffu, shl_clamped(1u, W.cp.start[gbase + 1 + lane] - e0));
                    const int e = e0 + lane;
                    if (e < lim) {
                        const int4 R = W.cp.rec[gbase + __popc(B & le)];
                        const int2 xl = m.s_xyl[e + R.x];
                        cdst[e] = R.y + xl.x;
                        st_val(vdst + e, __int_as_float(xl.y) * __int_as_float(R.z));
                    }
                    gbase += __popc(B);
                }
                __syncwarp();
                // 3. the cut chords of the kept end cells
                if (ka && sa < lim) st_val(vdst + sa, va);
                if (kb && sb < lim) st_val(vdst + sb, vb);
                pos += total;
                __syncwarp();
            }
            if (lane == 0 && pos != pend) atomicExch(status, PSF_EDEBUG);
        }
    }
}

}  // namespace psf

using namespace psf;

namespace psf {

// Validated arguments of the set row generator.
static int set_args(const psf_scanner *scanner, const psf_image *image, const psf_lor_set *set,
                    const int64_t *row_ptr, const int32_t *col, const void *val,
                    const int64_t *nnz_out, Scan &sc, Img &im, LorSet &ls) {
    int rc = make_scan(scanner, &sc);
    if (rc) return rc;
    rc = make_img(image, &im);
    if (rc) return rc;
    rc = make_lorset(scanner, set, &ls);
    if (rc) return rc;
    if (!row_ptr || !nnz_out || (col && !val)) return PSF_EINVAL;
    if (im.nx + im.ny + 1 > SET_MAXC || im.nx > 32767 || im.ny > 32767) return PSF_EINVAL;
    return PSF_OK;
}

// Scratch of the set row generator: scan tile sums, a status word and the
// ring-pair z-axis table.
static size_t set_scratch_bytes(const LorSet &ls, int64_t *ntiles_out) {
    const int64_t n = ls.ntp * ls.nrp;
    const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE + 1;
    *ntiles_out = ntiles;
    return sizeof(int64_t) * ntiles + 64 + sizeof(ZAx) * ls.nrp;
}

// The allocating entry points add the per-pair cell cache after the scratch
// (16-byte aligned).
static size_t set_cache_bytes(const LorSet &ls, const Img &im) {
    return 16 + (size_t)ls.ntp * (size_t)cell_slot_bytes(im.nx + im.ny + 1);
}

// Ring-pair table, count, scan, (size check,) fill.  row_ptr[0] is already 0.
template <typename VT>
static int set_fill_launch(const Scan &sc, const Img &im, const LorSet &ls, const ZAx *zt,
                           const int64_t *row_ptr, int32_t *col, void *val, float *row_scale,
                           int *status, int grid, size_t shm, const CellCache &cache,
                           cudaStream_t st) {
    PSF_TRY(cudaFuncSetAttribute(set_fill_kernel<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shm));
    {
        PSF_TIMED("set_fill_kernel", st);
        set_fill_kernel<VT><<<grid, SET_T, shm, st>>>(sc, im, ls, zt, row_ptr, col,
                                                      static_cast<VT *>(val), row_scale, status,
                                                      cache);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

// cached: the scratch is followed by set_cache_bytes of room for the cell
// cache (else both kernels build the cells).
static int set_pipeline(const Scan &sc, const Img &im, const LorSet &ls, int64_t *row_ptr,
                        int32_t *col, void *val, int64_t capacity, int64_t *nnz_out,
                        unsigned char *scratch, int64_t ntiles, cudaStream_t st, bool cached,
                        int32_t dtype = PSF_F32, float *row_scale = nullptr) {
    const int64_t n = ls.ntp * ls.nrp;
    int64_t *tiles = reinterpret_cast<int64_t *>(scratch);
    int *status = reinterpret_cast<int *>(tiles + ntiles);
    ZAx *zt = reinterpret_cast<ZAx *>(reinterpret_cast<unsigned char *>(status) + 64);
    CellCache cache{nullptr, im.nx + im.ny + 1, cell_slot_bytes(im.nx + im.ny + 1)};
    if (cached)
        cache.base = reinterpret_cast<unsigned char *>(
            (reinterpret_cast<uintptr_t>(zt + ls.nrp) + 15) & ~uintptr_t(15));
    PSF_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
    const size_t zshm = sizeof(int32_t) * (ls.Nt + ls.NR + 2);
    {
        PSF_TIMED("zaxis_kernel", st);
        zaxis_kernel<<<(int)((ls.nrp + 255) / 256), 256, zshm, st>>>(sc, im, ls, zt);
    }
    PSF_LAUNCHED();
    const int grid_max = sm_count() * 3;  // the fill's resident CTAs (launch bounds 3 per SM)
    const int grid = (int)(ls.ntp < grid_max ? ls.ntp : grid_max);
    const size_t shm = set_smem(sc, ls);  // the fill's
    {
        // the count kernel's own (smaller) layout and grid
        const size_t cshm = count_smem(sc, ls);
        PSF_TRY(cudaFuncSetAttribute(set_count_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cshm));
        int per_sm = 0;
        PSF_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, set_count_kernel, SET_T,
                                                              cshm));
        const int cmax = sm_count() * (per_sm > 0 ? per_sm : 1);
        const int cgrid = (int)(ls.ntp < cmax ? ls.ntp : cmax);
        PSF_TIMED("set_count_kernel", st);
        set_count_kernel<<<cgrid, SET_T, cshm, st>>>(sc, im, ls, zt, row_ptr + 1, status,
                                                     cache);
    }
    PSF_LAUNCHED();
    int rc = inclusive_scan(row_ptr + 1, n, tiles, st);
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
    rc = dtype == PSF_BF16
             ? set_fill_launch<__nv_bfloat16>(sc, im, ls, zt, row_ptr, col, val, row_scale,
                                              status, grid, shm, cache, st)
         : dtype == PSF_F16
             ? set_fill_launch<__half>(sc, im, ls, zt, row_ptr, col, val, row_scale, status,
                                       grid, shm, cache, st)
             : set_fill_launch<float>(sc, im, ls, zt, row_ptr, col, val, nullptr, status, grid,
                                      shm, cache, st);
    if (rc) return rc;
    PSF_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PSF_TRY(cudaStreamSynchronize(st));
    return h_status;
}

}  // namespace psf

namespace psf {
// Scratch of the allocating entry points: with room for the cell cache, or,
// when that much device memory is not available, without it (the count and
// fill kernels then both build the cells).
static int set_scratch_alloc(const LorSet &ls, const Img &im, cudaStream_t st, void **scratch,
                             int64_t *ntiles, bool *cached) {
    const size_t base = set_scratch_bytes(ls, ntiles);
    *cached = true;
    if (cudaMallocAsync(scratch, base + set_cache_bytes(ls, im), st) == cudaSuccess)
        return PSF_OK;
    (void)cudaGetLastError();  // the failed request leaves no sticky error
    *cached = false;
    PSF_TRY(cudaMallocAsync(scratch, base, st));
    return PSF_OK;
}
}  // namespace psf

extern "C" int psf_sysmat_rows_set(const psf_scanner *scanner, const psf_image *image,
                                   const psf_lor_set *set, int64_t *row_ptr, int32_t *col,
                                   float *val, int64_t capacity, int64_t *nnz_out, void *stream) {
    PSF_RANGE("psf_sysmat_rows_set");
    Scan sc;
    Img im;
    LorSet ls;
    int rc = set_args(scanner, image, set, row_ptr, col, val, nnz_out, sc, im, ls);
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    *nnz_out = 0;
    PSF_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
    if (ls.ntp * ls.nrp == 0) return PSF_OK;
    int64_t ntiles = 0;
    void *scratch = nullptr;
    bool cached = false;
    rc = set_scratch_alloc(ls, im, st, &scratch, &ntiles, &cached);
    if (rc) return rc;
    rc = set_pipeline(sc, im, ls, row_ptr, col, val, capacity, nnz_out,
                      static_cast<unsigned char *>(scratch), ntiles, st, cached);
    cudaFreeAsync(scratch, st);
    return rc;
}

extern "C" int psf_sysmat_rows_set_typed(const psf_scanner *scanner, const psf_image *image,
                                         const psf_lor_set *set, int32_t dtype,
                                         int64_t *row_ptr, int32_t *col, void *val,
                                         float *row_scale, int64_t capacity, int64_t *nnz_out,
                                         void *stream) {
    PSF_RANGE("psf_sysmat_rows_set_typed");
    if (dtype != PSF_F32 && dtype != PSF_BF16 && dtype != PSF_F16) return PSF_EINVAL;
    // F32: no scale; 16-bit forms: a scale per row, needed with the fill
    if (dtype == PSF_F32 ? row_scale != nullptr : (col != nullptr && row_scale == nullptr))
        return PSF_EINVAL;
    Scan sc;
    Img im;
    LorSet ls;
    int rc = set_args(scanner, image, set, row_ptr, col, val, nnz_out, sc, im, ls);
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    *nnz_out = 0;
    PSF_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
    if (ls.ntp * ls.nrp == 0) return PSF_OK;
    int64_t ntiles = 0;
    void *scratch = nullptr;
    bool cached = false;
    rc = set_scratch_alloc(ls, im, st, &scratch, &ntiles, &cached);
    if (rc) return rc;
    rc = set_pipeline(sc, im, ls, row_ptr, col, val, capacity, nnz_out,
                      static_cast<unsigned char *>(scratch), ntiles, st, cached, dtype,
                      row_scale);
    cudaFreeAsync(scratch, st);
    return rc;
}

extern "C" int psf_sysmat_rows(const psf_scanner *scanner, const psf_image *image,
                               const int32_t *lors, int64_t n_lors, const float *spread,
                               int32_t half_t, int32_t half_a, int32_t dtype, int64_t *row_ptr,
                               int32_t *col, void *val, float *row_scale, int64_t capacity,
                               int64_t *nnz_out, void *stream) {
    PSF_RANGE("psf_sysmat_rows");
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
        {
            PSF_TIMED("pair_map_kernel", st);
            pair_map_kernel<<<grid_for(n_lors, 256), 256, 0, st>>>(lors, n_lors, nc, map);
        }
        size_t shm = sizeof(float) * nvox + (sizeof(int32_t) + sizeof(float)) * 2 * E * E +
                     sizeof(int) * (MERGE_T / 32 + 2) + sizeof(float) * (MERGE_T / 32) + 16;
        int grid = sm_count() * 4;
        auto launch = [&](int pass, auto *vptr) -> int {
            using VT = std::remove_pointer_t<decltype(vptr)>;
            PSF_TRY(cudaFuncSetAttribute(merge_kernel<VT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
            {
                PSF_TIMED("merge_kernel", st);
                merge_kernel<VT><<<grid, MERGE_T, shm, st>>>(
                    pass, sc, nvox, lors, n_lors, map, gptr, gcol, gval, spread, half_t, half_a,
                    pass == 0 ? row_ptr + 1 : row_ptr, col, vptr, row_scale);
            }
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

// ------------------------------------------------ no-allocation entry point
// psf_sysmat_rows_set without any allocation: the scan's tile sums and the
// status word live in one fixed device array (see psf.h).  The array's device
// address is looked up once per device, on that device's first call.
#include <mutex>

namespace psf {
static __device__ __align__(256) unsigned char g_noalloc_scratch[PSF_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[1024];  // device address of the array, per device ordinal

static int noalloc_scratch(void **out) {
    int dev = 0;
    PSF_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 1024) return PSF_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        PSF_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));  // host name -> device address
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PSF_OK;
}
}  // namespace psf

extern "C" int psf_sysmat_rows_set_noalloc(const psf_scanner *scanner, const psf_image *image,
                                           const psf_lor_set *set, int64_t *row_ptr,
                                           int32_t *col, float *val, int64_t capacity,
                                           int64_t *nnz_out, void *stream) {
    PSF_RANGE("psf_sysmat_rows_set_noalloc");
    Scan sc;
    Img im;
    LorSet ls;
    int rc = set_args(scanner, image, set, row_ptr, col, val, nnz_out, sc, im, ls);
    if (rc) return rc;
    *nnz_out = 0;
    if (ls.ntp * ls.nrp > PSF_NOALLOC_MAX_ROWS) return PSF_ENOSCRATCH;
    int64_t ntiles = 0;
    if (set_scratch_bytes(ls, &ntiles) > (size_t)PSF_NOALLOC_SCRATCH_BYTES) return PSF_ENOSCRATCH;
    void *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = as_stream(stream);
    PSF_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
    if (ls.ntp * ls.nrp == 0) return PSF_OK;
    // tile sums and the ring-pair table are fully rewritten; set_pipeline
    // clears the status word an earlier call may have left set
    return set_pipeline(sc, im, ls, row_ptr, col, val, capacity, nnz_out,
                        static_cast<unsigned char *>(scratch), ntiles, st, false);
}
