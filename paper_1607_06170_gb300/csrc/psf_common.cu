// Validation of the C-ABI descriptions, error strings, structured LOR sets
// and the MLEM elementwise steps.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "psf_common.cuh"
#include "psf_lorset.cuh"

namespace psf {

static thread_local cudaError_t g_last_cuda = cudaSuccess;

void set_cuda_error(cudaError_t e) { g_last_cuda = e; }

int make_scan(const psf_scanner *s, Scan *o) {
    if (!s || !o) return PSF_EINVAL;
    if (s->n_blocks < 3 || s->nt_block < 1 || s->na_block < 1 || s->n_block_rings < 1)
        return PSF_EINVAL;
    if (!(s->xtal_w_t > 0) || !(s->xtal_w_a > 0) || !(s->depth > 0) || !(s->gap_t >= 0) ||
        !(s->gap_a >= 0) || !(s->radius > 0) || !(s->mu > 0) || !(s->block_gap_a >= 0))
        return PSF_EINVAL;
    if (s->n_block_rings > 1 && s->block_gap_a != s->gap_a) return PSF_EINVAL;
    int64_t nt = (int64_t)s->n_blocks * s->nt_block;
    int64_t nr = (int64_t)s->na_block * s->n_block_rings;
    if (nt * nr > INT32_MAX / 2) return PSF_EINVAL;
    double pt = s->xtal_w_t + s->gap_t, pa = s->xtal_w_a + s->gap_a;
    double half_w = 0.5 * (s->nt_block * s->xtal_w_t + (s->nt_block - 1) * s->gap_t);
    double sigma = s->radius * tan(M_PI / s->n_blocks) - half_w;
    if (!(sigma >= 0)) return PSF_EINVAL;  // neighbouring blocks would overlap
    o->R = s->n_blocks;
    o->Nb = s->nt_block;
    o->Nt = (int)nt;
    o->NR = (int)nr;
    o->wt = (float)s->xtal_w_t;
    o->wa = (float)s->xtal_w_a;
    o->depth = (float)s->depth;
    o->gt = (float)s->gap_t;
    o->ga = (float)s->gap_a;
    o->pt = (float)pt;
    o->pa = (float)pa;
    o->mu = (float)s->mu;
    o->radius = (float)s->radius;
    o->half_w = (float)half_w;
    o->sigma = (float)sigma;
    double z0 = -0.5 * (nr - 1) * pa;
    o->z0 = (float)z0;
    o->two_pi_R = (float)(2.0 * M_PI / s->n_blocks);
    o->sin_two_pi_R = (float)sin(2.0 * M_PI / s->n_blocks);
    o->radius64 = s->radius;
    o->pt64 = pt;
    o->pa64 = pa;
    o->z064 = z0;
    return PSF_OK;
}

int make_tab(const psf_table_desc *d, const Scan &sc, Tab *o, bool check_reach) {
    if (!d || !o) return PSF_EINVAL;
    if (d->n_ang_t < 1 || d->n_ang_a < 1 || d->n_sub_t < 1 || d->n_sub_a < 1 ||
        d->max_off_t < 1 || d->max_off_a < 1)
        return PSF_EINVAL;
    if (!(d->ang_max_t_deg > 0 && d->ang_max_t_deg <= 90) ||
        !(d->ang_max_a_deg > 0 && d->ang_max_a_deg <= 90))
        return PSF_EINVAL;
    if ((int64_t)d->n_ang_t * d->n_ang_a * d->n_sub_t * d->n_sub_a * d->max_off_t *
            d->max_off_a > (int64_t)1 << 28)
        return PSF_EINVAL;
    if (d->max_off_t * d->max_off_a > 1024 || d->max_off_t > 64) return PSF_EINVAL;
    double st = d->ang_max_t_deg / d->n_ang_t * M_PI / 180.0;
    double sa = d->ang_max_a_deg / d->n_ang_a * M_PI / 180.0;
    double at_last = (d->n_ang_t - 1) * st, aa_last = (d->n_ang_a - 1) * sa;
    if (at_last >= 0.5 * M_PI || aa_last >= 0.5 * M_PI) return PSF_EINVAL;
    if (check_reach) {
        // every crystal a ray of the last node can reach must have a slot
        double x0 = (d->n_sub_t - 0.5) / d->n_sub_t * sc.wt;
        double y0 = (d->n_sub_a - 0.5) / d->n_sub_a * sc.wa;
        double xr = x0 + sc.depth * tan(at_last);
        double yr = y0 + sc.depth * tan(aa_last) / cos(at_last);
        if ((int)floor(xr / sc.pt64) + 1 > d->max_off_t) return PSF_EINVAL;
        if ((int)floor(yr / sc.pa64) + 1 > d->max_off_a) return PSF_EINVAL;
    }
    o->Kt = d->n_ang_t;
    o->Ka = d->n_ang_a;
    o->Pt = d->n_sub_t;
    o->Pa = d->n_sub_a;
    o->Mt = d->max_off_t;
    o->Ma = d->max_off_a;
    o->dt = (float)st;
    o->da = (float)sa;
    o->inv_dt = (float)(1.0 / st);
    o->inv_da = (float)(1.0 / sa);
    return PSF_OK;
}

int make_img(const psf_image *im, Img *o) {
    if (!im || !o) return PSF_EINVAL;
    if (im->nx < 1 || im->ny < 1 || im->nz < 1) return PSF_EINVAL;
    if ((int64_t)im->nx * im->ny * im->nz > INT32_MAX) return PSF_EINVAL;
    if (!(im->dx > 0) || !(im->dy > 0) || !(im->dz > 0)) return PSF_EINVAL;
    o->nx = im->nx;
    o->ny = im->ny;
    o->nz = im->nz;
    o->dx = im->dx;
    o->dy = im->dy;
    o->dz = im->dz;
    o->ox = im->ox;
    o->oy = im->oy;
    o->oz = im->oz;
    o->idx = 1.0 / im->dx;
    o->idy = 1.0 / im->dy;
    o->idz = 1.0 / im->dz;
    return PSF_OK;
}

// ------------------------------------------------------------ LOR sets
int make_lorset(const psf_scanner *s, const psf_lor_set *set, LorSet *o) {
    Scan sc;
    int rc = make_scan(s, &sc);
    if (rc) return rc;
    if (!set || !o) return PSF_EINVAL;
    if (sc.Nt % 2 || sc.Nt > 8192 || sc.NR > 1024) return PSF_EINVAL;
    if (set->fan_half < 0 || set->fan_half > sc.Nt / 2 - 1) return PSF_EINVAL;
    if (set->max_ring_diff < 0 || set->max_ring_diff > sc.NR - 1) return PSF_EINVAL;
    o->Nt = sc.Nt;
    o->NR = sc.NR;
    o->Nb = sc.Nb;
    o->F = set->fan_half;
    o->Dm = set->max_ring_diff;
    int64_t ntp = 0, ntp_cls = 0;
    for (int a = 0; a < sc.Nt; ++a) {
        int c = o->tp_count(a);
        ntp += c;
        if (a < sc.Nb) ntp_cls += c;
    }
    int64_t nrp = 0;
    for (int r = 0; r < sc.NR; ++r) nrp += o->rp_count(r);
    o->ntp = ntp;
    o->nrp = nrp;
    o->ntp_cls = ntp_cls;
    return PSF_OK;
}

__global__ void lorset_list_kernel(LorSet ls, int32_t *lors, bool classes) {
    extern __shared__ int32_t sh[];
    int32_t *tp_start = sh;            // [Nt + 1]
    int32_t *rp_start = sh + ls.Nt + 1;  // [NR + 1]
    ls.stage_prefix(tp_start, rp_start);
    __syncthreads();
    int64_t n = classes ? ls.ntp_cls * (2 * ls.Dm + 1) : ls.ntp * ls.nrp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int a, b, ra, rb;
        if (classes) {
            int nd = 2 * ls.Dm + 1;
            int64_t tpi = k / nd;
            int dl = (int)(k % nd) - ls.Dm;
            ls.tp_decode(tp_start, tpi, &a, &b);
            ra = dl < 0 ? -dl : 0;
            rb = ra + dl;
        } else {
            int64_t tpi = k / ls.nrp;
            int64_t rpi = k % ls.nrp;
            ls.tp_decode(tp_start, tpi, &a, &b);
            ls.rp_decode(rp_start, rpi, &ra, &rb);
        }
        lors[2 * k] = ra * ls.Nt + a;
        lors[2 * k + 1] = rb * ls.Nt + b;
    }
}

// ------------------------------------------------------------ MLEM steps
__global__ void em_ratio_kernel(const float *__restrict__ y, const float *__restrict__ yh,
                                float *__restrict__ r, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float d = yh[i];
        r[i] = d > 0.0f ? y[i] / d : 0.0f;
    }
}

__global__ void em_update_kernel(float *__restrict__ x, const float *__restrict__ bp,
                                 const float *__restrict__ sens, float floor_, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = sens[i];
        x[i] = s >= floor_ && s > 0.0f ? x[i] * bp[i] / s : 0.0f;
    }
}

int grid_for(int64_t n, int block) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)sms * 8;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// ---------------------------------------------------------- kernel timing
namespace {
struct TimerPending {
    const char *name;
    cudaEvent_t a, b;
};
struct TimerAcc {
    std::string name;
    int64_t launches;
    double ms;
};
std::mutex g_tmu;
std::atomic<bool> g_ton{false};
std::vector<TimerPending> g_tpending;
std::vector<TimerAcc> g_tacc;
std::vector<cudaEvent_t> g_tpool;

cudaEvent_t pool_event() {
    if (!g_tpool.empty()) {
        cudaEvent_t e = g_tpool.back();
        g_tpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Fold the recorded pairs into the accumulators (caller holds the lock).
int drain_pending() {
    int rc = PSF_OK;
    for (const TimerPending &p : g_tpending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
            rc = PSF_ECUDA;
        } else {
            size_t k = 0;
            while (k < g_tacc.size() && g_tacc[k].name != p.name) ++k;
            if (k == g_tacc.size()) g_tacc.push_back({p.name, 0, 0.0});
            g_tacc[k].launches += 1;
            g_tacc[k].ms += ms;
        }
        g_tpool.push_back(p.a);
        g_tpool.push_back(p.b);
    }
    g_tpending.clear();
    return rc;
}
}  // namespace

bool timing_on() { return g_ton.load(std::memory_order_relaxed); }

cudaEvent_t timing_start(cudaStream_t st) {
    std::lock_guard<std::mutex> lock(g_tmu);
    cudaEvent_t e = pool_event();
    if (e && cudaEventRecord(e, st) != cudaSuccess) {
        g_tpool.push_back(e);
        return nullptr;
    }
    return e;
}

void timing_stop(const char *name, cudaStream_t st, cudaEvent_t start) {
    std::lock_guard<std::mutex> lock(g_tmu);
    cudaEvent_t e = pool_event();
    if (!e || cudaEventRecord(e, st) != cudaSuccess) {
        g_tpool.push_back(start);
        if (e) g_tpool.push_back(e);
        return;
    }
    g_tpending.push_back({name, start, e});
}

static std::atomic<int64_t> g_wait_limit{int64_t(1) << 31};  // about a second at 2 GHz

int64_t wait_limit() { return g_wait_limit.load(); }

}  // namespace psf

using namespace psf;

extern "C" int psf_set_wait_limit(int64_t cycles) {
    g_wait_limit.store(cycles);
    return PSF_OK;
}

extern "C" int psf_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lock(g_tmu);
    const int rc = drain_pending();
    g_tacc.clear();
    g_ton.store(on != 0);
    return rc;
}

extern "C" int psf_timing_read(int32_t index, const char **name, int64_t *launches, double *ms) {
    if (!name || !launches || !ms) return PSF_EINVAL;
    std::lock_guard<std::mutex> lock(g_tmu);
    const int rc = drain_pending();
    if (rc) return rc;
    if (index < 0 || (size_t)index >= g_tacc.size()) return PSF_EINVAL;
    *name = g_tacc[index].name.c_str();
    *launches = g_tacc[index].launches;
    *ms = g_tacc[index].ms;
    return PSF_OK;
}

extern "C" const char *psf_strerror(int code) {
    switch (code) {
        case PSF_OK: return "ok";
        case PSF_EINVAL: return "invalid argument";
        case PSF_ECAPACITY: return "output capacity too small";
        case PSF_ECUDA: return cudaGetErrorString(g_last_cuda);
        case PSF_ETIMEOUT: return "bounded device wait gave up";
        case PSF_EDEBUG: return "device bounds check failed";
        case PSF_ENOSCRATCH:
            return "LOR set too large for the fixed scratch of the no-allocation entry point";
        default: return "unknown error";
    }
}

extern "C" int psf_table_size(const psf_table_desc *d, int64_t *n_table, int64_t *n_eta) {
    if (!d || !n_table || !n_eta) return PSF_EINVAL;
    if (d->n_ang_t < 1 || d->n_ang_a < 1 || d->n_sub_t < 1 || d->n_sub_a < 1 ||
        d->max_off_t < 1 || d->max_off_a < 1)
        return PSF_EINVAL;
    int64_t e = (int64_t)d->n_ang_t * d->n_ang_a * d->n_sub_t * d->n_sub_a;
    *n_table = e * d->max_off_t * d->max_off_a;
    *n_eta = e * (d->max_off_t + 1);
    return PSF_OK;
}

extern "C" int psf_lor_set_size(const psf_scanner *s, const psf_lor_set *set, int64_t *n_lors,
                                int64_t *n_classes) {
    LorSet ls;
    int rc = make_lorset(s, set, &ls);
    if (rc) return rc;
    if (n_lors) *n_lors = ls.ntp * ls.nrp;
    if (n_classes) *n_classes = ls.ntp_cls * (2 * ls.Dm + 1);
    return PSF_OK;
}

static int lorset_list(const psf_scanner *s, const psf_lor_set *set, int32_t *lors, void *stream,
                       bool classes) {
    LorSet ls;
    int rc = make_lorset(s, set, &ls);
    if (rc) return rc;
    if (!lors) return PSF_EINVAL;
    int64_t n = classes ? ls.ntp_cls * (2 * ls.Dm + 1) : ls.ntp * ls.nrp;
    if (n == 0) return PSF_OK;
    size_t sh = sizeof(int32_t) * (ls.Nt + ls.NR + 2);
    {
        PSF_TIMED("lorset_list_kernel", as_stream(stream));
        lorset_list_kernel<<<grid_for(n, 256), 256, sh, as_stream(stream)>>>(ls, lors, classes);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

extern "C" int psf_lor_set_list(const psf_scanner *s, const psf_lor_set *set, int32_t *lors,
                                void *stream) {
    PSF_RANGE("psf_lor_set_list");
    return lorset_list(s, set, lors, stream, false);
}

extern "C" int psf_lor_set_classes(const psf_scanner *s, const psf_lor_set *set, int32_t *lors,
                                   void *stream) {
    PSF_RANGE("psf_lor_set_classes");
    return lorset_list(s, set, lors, stream, true);
}

extern "C" int psf_em_ratio(const float *y, const float *yhat, float *ratio, int64_t n,
                            void *stream) {
    PSF_RANGE("psf_em_ratio");
    if (n < 0 || (n > 0 && (!y || !yhat || !ratio))) return PSF_EINVAL;
    if (n == 0) return PSF_OK;
    {
        PSF_TIMED("em_ratio_kernel", as_stream(stream));
        em_ratio_kernel<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(y, yhat, ratio, n);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}

extern "C" int psf_em_update(float *x, const float *bp, const float *sens, float floor_,
                             int64_t n, void *stream) {
    PSF_RANGE("psf_em_update");
    if (n < 0 || (n > 0 && (!x || !bp || !sens))) return PSF_EINVAL;
    if (n == 0) return PSF_OK;
    {
        PSF_TIMED("em_update_kernel", as_stream(stream));
        em_update_kernel<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(x, bp, sens, floor_, n);
    }
    PSF_LAUNCHED();
    return PSF_OK;
}
