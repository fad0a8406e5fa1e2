// Structured LOR set of a ring scanner (see psf_lor_set in psf.h): index
// arithmetic shared by the set enumeration, the factored PSF projector and the
// spread-class lookup.
#pragma once

#include <cstdint>

#include "psf_common.cuh"

namespace psf {

struct LorSet {
    int Nt, NR, Nb, F, Dm;
    int64_t ntp, nrp, ntp_cls;

    __host__ __device__ int tp_lo(int a) const {
        int lo = a + Nt / 2 - F;
        return lo > a + 1 ? lo : a + 1;
    }
    __host__ __device__ int tp_hi(int a) const {
        int hi = a + Nt / 2 + F;
        return hi < Nt - 1 ? hi : Nt - 1;
    }
    __host__ __device__ int tp_count(int a) const {
        int c = tp_hi(a) - tp_lo(a) + 1;
        return c > 0 ? c : 0;
    }
    __host__ __device__ int rp_lo(int r) const { return r - Dm > 0 ? r - Dm : 0; }
    __host__ __device__ int rp_hi(int r) const { return r + Dm < NR - 1 ? r + Dm : NR - 1; }
    __host__ __device__ int rp_count(int r) const { return rp_hi(r) - rp_lo(r) + 1; }

    // Block-cooperative prefix tables: tp_start[a] = rows of transaxial pairs
    // with first crystal < a, rp_start[r] likewise for ring pairs.
    __device__ void stage_prefix(int32_t *tp_start, int32_t *rp_start) const {
        if (threadIdx.x < 32) {
            unsigned lane = threadIdx.x;
            int32_t carry = 0;
            for (int base = 0; base < Nt; base += 32) {
                int a = base + lane;
                int32_t v = a < Nt ? tp_count(a) : 0;
                int32_t inc = v;
                for (int o = 1; o < 32; o <<= 1) {
                    int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= (unsigned)o) inc += t;
                }
                if (a < Nt) tp_start[a] = carry + inc - v;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
            if (lane == 0) tp_start[Nt] = carry;
            carry = 0;
            for (int base = 0; base < NR; base += 32) {
                int r = base + lane;
                int32_t v = r < NR ? rp_count(r) : 0;
                int32_t inc = v;
                for (int o = 1; o < 32; o <<= 1) {
                    int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= (unsigned)o) inc += t;
                }
                if (r < NR) rp_start[r] = carry + inc - v;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
            if (lane == 0) rp_start[NR] = carry;
        }
    }

    __device__ void tp_decode(const int32_t *tp_start, int64_t idx, int *a, int *b) const {
        int lo = 0, hi = Nt - 1;  // largest a with tp_start[a] <= idx
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (tp_start[mid] <= idx) lo = mid; else hi = mid - 1;
        }
        *a = lo;
        *b = tp_lo(lo) + (int)(idx - tp_start[lo]);
    }

    // Transaxial pairs in order of their crystal difference d = b - a, then
    // of a: the idx-th pair of that order.  Pairs of one difference cycle
    // through the spread classes of that difference (and their rotations), so
    // kernels that walk the pairs in this order touch few classes at a time.
    __device__ void tp_decode_diff(int64_t idx, int *a, int *b) const {
        const int dlo = Nt / 2 - F > 1 ? Nt / 2 - F : 1, dhi = Nt / 2 + F < Nt - 1 ? Nt / 2 + F : Nt - 1;
        // pairs with difference below d: sum over e in [dlo, d) of (Nt - e)
        auto before = [&](int d) -> int64_t {
            const int64_t k = d - dlo;
            return k * Nt - k * (dlo + d - 1) / 2;
        };
        int lo = dlo, hi = dhi;  // largest d with before(d) <= idx
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (before(mid) <= idx) lo = mid; else hi = mid - 1;
        }
        *a = (int)(idx - before(lo));
        *b = *a + lo;
    }

    __device__ void rp_decode(const int32_t *rp_start, int64_t idx, int *ra, int *rb) const {
        int lo = 0, hi = NR - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (rp_start[mid] <= idx) lo = mid; else hi = mid - 1;
        }
        *ra = lo;
        *rb = rp_lo(lo) + (int)(idx - rp_start[lo]);
    }

    // Membership of the ordered LOR (a, ra) -> (b, rb) with a < b required.
    __device__ bool member(int a, int b, int ra, int rb) const {
        if (a < 0 || b >= Nt || a >= b) return false;
        int d = b - a;
        if (d < Nt / 2 - F || d > Nt / 2 + F) return false;
        if (ra < 0 || rb < 0 || ra >= NR || rb >= NR) return false;
        int dr = rb - ra;
        return dr <= Dm && dr >= -Dm;
    }

    __device__ int64_t row_of(const int32_t *tp_start, const int32_t *rp_start, int a, int b,
                              int ra, int rb) const {
        int64_t tp = tp_start[a] + (b - tp_lo(a));
        int64_t rp = rp_start[ra] + (rb - rp_lo(ra));
        return tp * nrp + rp;
    }

    // Spread class: rotate the first crystal into block 0 (roles kept) and
    // keep only the ring difference.
    __device__ int64_t class_of(const int32_t *tp_start, int a, int b, int ra, int rb) const {
        int a0 = a % Nb;
        int b0 = b - (a - a0);
        int64_t tp = tp_start[a0] + (b0 - tp_lo(a0));
        return tp * (2 * Dm + 1) + (rb - ra + Dm);
    }
};

int make_lorset(const psf_scanner *s, const psf_lor_set *set, LorSet *out);

}  // namespace psf
