// Exact-parameter chord tracer shared by the row generators.
//
// A LOR's segment S -> E (grid-local voxel units) is parametrised by
// alpha in [0, 1], stored as a 64-bit fixed-point integer with 2^40 units per
// segment (2^-40 of a ~260 mm segment is ~2.4e-10 mm).  Plane k of an axis
// is crossed at A(k) = A0 + k * DA with A0 and DA rounded once per ray from
// FP64, so consecutive slabs tile the segment exactly and every membership
// decision (which voxels a segment meets, in which order) is an integer
// comparison.  FP32 is used only to guess a voxel index, which an exact
// comparison then corrects.  Voxels are visited in ascending voxel index
// (z slab, then y row, then x), which is the CSR column order.
#pragma once

#include <cstring>

#include "psf_common.cuh"

namespace psf {

constexpr double FX = 1099511627776.0;  // 2^40 units per segment
constexpr long long FX_BIG = (long long)1 << 62;

__host__ __device__ __forceinline__ float u32_to_f(unsigned v) {
#ifdef __CUDA_ARCH__
    return __uint2float_rn(v);
#else
    return (float)v;
#endif
}

// Non-negative parameter difference (< 2^48) to float, rounded once: both
// 24-bit halves convert exactly and the FMA rounds hi * 2^24 + lo once.
__host__ __device__ __forceinline__ float units_to_f(long long v) {
    const unsigned hi = (unsigned)(v >> 24), lo = (unsigned)(v & ((1 << 24) - 1));
    return fmaf(u32_to_f(hi), 16777216.0f, u32_to_f(lo));
}

// Bit copies between float and int (host and device).
__host__ __device__ __forceinline__ float bits_float(int v) {
#ifdef __CUDA_ARCH__
    return __int_as_float(v);
#else
    float f;
    memcpy(&f, &v, sizeof f);
    return f;
#endif
}
__host__ __device__ __forceinline__ int float_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_int(f);
#else
    int v;
    memcpy(&v, &f, sizeof v);
    return v;
#endif
}

struct Axis {
    int kind;   // 0: parallel to the planes (index fixed), 1: linear, 2: nearly parallel
    int fixed;  // voxel index when kind == 0
    int n;      // voxels along the axis
    int inc;    // 1 if the coordinate grows along the segment
    long long A0, DA;
    double S, D;  // grid-local start / extent
    float sf, df;
};

// Chords shorter than this are rounding artefacts of a segment passing
// through a voxel edge or corner (exact chord 0) and are not stored.
constexpr double MIN_CHORD_MM = 1e-7;

struct Ray {
    Axis ax[3];
    long long amin, amax;
    long long min_units;  // MIN_CHORD_MM in fixed-point units of this segment
    float len_mm;
    bool empty;
};

__host__ __device__ __forceinline__ long long plane_alpha(const Axis &a, int k) {
    if (a.kind == 1) return a.A0 + (long long)k * a.DA;
    double t = ((double)k - a.S) / a.D;
    t = fmin(fmax(t, -4.0), 4.0);
    return d2ll_rn(t * FX);
}

// alpha-interval of slab k of an axis
__host__ __device__ __forceinline__ void slab(const Axis &a, int k, long long &lo, long long &hi) {
    if (a.kind == 0) {
        lo = a.fixed == k ? -FX_BIG : FX_BIG;
        hi = a.fixed == k ? FX_BIG : -FX_BIG;
        return;
    }
    long long p = plane_alpha(a, k), q = plane_alpha(a, k + 1);
    lo = p < q ? p : q;
    hi = p < q ? q : p;
}

// Index of the slab containing parameter al (slab k holds [lo, hi)).
// Returns false if the correction did not settle (cannot happen for a
// consistent ray; kept as a bounded loop).
__host__ __device__ __forceinline__ bool voxel_at(const Axis &a, long long al, int &k) {
    if (a.kind == 0) {
        k = a.fixed;
        return true;
    }
    // guess in FP32 from the top 32 of the parameter's 40 fraction bits (no
    // FP64 on this path); al is inside [amin, amax] within [0, 2^40]
    const float af = u32_to_f((unsigned)(al >> 8)) * 2.3283064365386963e-10f;  // 2^-32
    float g = fmaf(af, a.df, a.sf);
    g = fminf(fmaxf(g, -2.0f), (float)a.n + 1.0f);
    int k0 = f2i_rd(g);
    const bool inc = a.inc;
    for (int it = 0; it < 64; ++it) {
        long long lo, hi;
        slab(a, k0, lo, hi);
        if (al < lo) {
            k0 += inc ? -1 : 1;
        } else if (al >= hi) {
            k0 += inc ? 1 : -1;
        } else {
            k = k0;
            return true;
        }
    }
    k = k0;
    return false;
}

__host__ __device__ __forceinline__ void make_axis(Axis &a, double s, double e, int n, bool &empty) {
    a.n = n;
    a.S = s;
    a.D = e - s;
    a.A0 = 0;
    a.DA = 0;
    a.fixed = 0;
    a.sf = (float)s;
    a.df = (float)a.D;
    a.inc = a.D > 0.0;
    if (fabs(a.D) < 1e-9) {
        // parallel: a coordinate within 1e-9 voxel of a plane lies on it and
        // belongs to the voxel above
        double r = rint(s);
        double c = fabs(s - r) < 1e-9 ? r : s;
        a.kind = 0;
        a.fixed = (int)floor(c);
        a.D = 0.0;
        a.df = 0.0f;
        if (a.fixed < 0 || a.fixed >= n) empty = true;
    } else if (fabs(a.D) < 1.0 / 1024.0) {
        a.kind = 2;
    } else {
        a.kind = 1;
        double inv = 1.0 / a.D;
        a.A0 = d2ll_rn(-s * inv * FX);
        a.DA = d2ll_rn(inv * FX);
    }
}

// Segment P -> Q (mm) through image im.
__host__ __device__ __forceinline__ void make_ray(Ray &r, const Img &im, double px, double py, double pz,
                                         double qx, double qy, double qz) {
    r.empty = false;
    const double sx = (px - im.ox) * im.idx, ex = (qx - im.ox) * im.idx;
    const double sy = (py - im.oy) * im.idy, ey = (qy - im.oy) * im.idy;
    const double sz = (pz - im.oz) * im.idz, ez = (qz - im.oz) * im.idz;
    make_axis(r.ax[0], sx, ex, im.nx, r.empty);
    make_axis(r.ax[1], sy, ey, im.ny, r.empty);
    make_axis(r.ax[2], sz, ez, im.nz, r.empty);
    // the length only scales the chords (FP32 precision is enough)
    const float lx = (float)(qx - px), ly = (float)(qy - py), lz = (float)(qz - pz);
    r.len_mm = sqrtf(lx * lx + ly * ly + lz * lz);
    r.min_units = (long long)ceilf((float)MIN_CHORD_MM / r.len_mm * (float)FX);
    long long amin = 0, amax = (long long)FX;
    for (int c = 0; c < 3; ++c) {
        const Axis &a = r.ax[c];
        if (a.kind == 0) continue;
        long long p = plane_alpha(a, 0), q = plane_alpha(a, a.n);
        long long lo = p < q ? p : q, hi = p < q ? q : p;
        amin = lo > amin ? lo : amin;
        amax = hi < amax ? hi : amax;
    }
    r.amin = amin;
    r.amax = amax;
    if (amax <= amin) r.empty = true;
}

// Chord (fixed-point units) of voxel ix inside a row interval [lo, hi).
__host__ __device__ __forceinline__ long long chord_in_row(const Axis &X, int ix, long long lo,
                                                            long long hi) {
    long long a, b;
    slab(X, ix, a, b);
    a = a > lo ? a : lo;
    b = b < hi ? b : hi;
    return b - a;
}

// Visit the rows (z slab, y row) of a ray in ascending order; for each, call
// row(iz, iy, ix_first, ix_last, lo, hi) with the row's parameter interval.
// Only the first and last voxel of a row can hold a chord shorter than a
// full slab, so those two are trimmed when below min_units; every voxel
// passed to row() then has a chord of at least MIN_CHORD_MM.
// Returns false if a voxel lookup failed to settle.
template <class RowFn>
__host__ __device__ __forceinline__ bool trace_rows(const Ray &r, RowFn &&row) {
    if (r.empty) return true;
    bool ok = true;
    const Axis &X = r.ax[0], &Y = r.ax[1], &Z = r.ax[2];
    int za, zb;
    ok &= voxel_at(Z, r.amin, za);
    ok &= voxel_at(Z, r.amax - 1, zb);
    int z0 = za < zb ? za : zb, z1 = za < zb ? zb : za;
    z0 = z0 < 0 ? 0 : z0;
    z1 = z1 > Z.n - 1 ? Z.n - 1 : z1;
    for (int iz = z0; iz <= z1; ++iz) {
        long long zl, zh;
        slab(Z, iz, zl, zh);
        zl = zl > r.amin ? zl : r.amin;
        zh = zh < r.amax ? zh : r.amax;
        if (zh <= zl) continue;
        int ya, yb;
        ok &= voxel_at(Y, zl, ya);
        ok &= voxel_at(Y, zh - 1, yb);
        int y0 = ya < yb ? ya : yb, y1 = ya < yb ? yb : ya;
        y0 = y0 < 0 ? 0 : y0;
        y1 = y1 > Y.n - 1 ? Y.n - 1 : y1;
        for (int iy = y0; iy <= y1; ++iy) {
            long long yl, yh;
            slab(Y, iy, yl, yh);
            yl = yl > zl ? yl : zl;
            yh = yh < zh ? yh : zh;
            if (yh <= yl) continue;
            int xa, xb;
            ok &= voxel_at(X, yl, xa);
            ok &= voxel_at(X, yh - 1, xb);
            int x0 = xa < xb ? xa : xb, x1 = xa < xb ? xb : xa;
            x0 = x0 < 0 ? 0 : x0;
            x1 = x1 > X.n - 1 ? X.n - 1 : x1;
            if (x1 >= x0 && chord_in_row(X, x0, yl, yh) < r.min_units) ++x0;
            if (x1 >= x0 && chord_in_row(X, x1, yl, yh) < r.min_units) --x1;
            if (x1 >= x0) row(iz, iy, x0, x1, yl, yh);
        }
    }
    return ok;
}

// Resumable form of trace_rows: yields one voxel per call, in the same
// ascending order and with the same trimming, so a kernel can interleave the
// voxels of several rays (row-by-row state: slab, row, voxel).
struct VoxelCursor {
    int iz, z1, iy, y1, ix, x1;
    long long zl, zh, yl, yh;
    bool done, ok;
};

// Move to the first voxel of the next non-empty row (or set done).
__host__ __device__ __forceinline__ void cursor_next_row(const Ray &r, VoxelCursor &c) {
    const Axis &X = r.ax[0], &Y = r.ax[1], &Z = r.ax[2];
    for (;;) {
        ++c.iy;
        if (c.iy > c.y1) {
            ++c.iz;
            if (c.iz > c.z1) {
                c.done = true;
                return;
            }
            slab(Z, c.iz, c.zl, c.zh);
            c.zl = c.zl > r.amin ? c.zl : r.amin;
            c.zh = c.zh < r.amax ? c.zh : r.amax;
            if (c.zh <= c.zl) {
                c.y1 = c.iy - 1;  // empty slab: no rows
                --c.iy;
                continue;
            }
            int ya, yb;
            c.ok &= voxel_at(Y, c.zl, ya);
            c.ok &= voxel_at(Y, c.zh - 1, yb);
            int y0 = ya < yb ? ya : yb, y1 = ya < yb ? yb : ya;
            y0 = y0 < 0 ? 0 : y0;
            c.y1 = y1 > Y.n - 1 ? Y.n - 1 : y1;
            c.iy = y0;
            if (c.iy > c.y1) {
                --c.iy;
                continue;
            }
        }
        slab(Y, c.iy, c.yl, c.yh);
        c.yl = c.yl > c.zl ? c.yl : c.zl;
        c.yh = c.yh < c.zh ? c.yh : c.zh;
        if (c.yh <= c.yl) continue;
        int xa, xb;
        c.ok &= voxel_at(X, c.yl, xa);
        c.ok &= voxel_at(X, c.yh - 1, xb);
        int x0 = xa < xb ? xa : xb, x1 = xa < xb ? xb : xa;
        x0 = x0 < 0 ? 0 : x0;
        x1 = x1 > X.n - 1 ? X.n - 1 : x1;
        if (x1 >= x0 && chord_in_row(X, x0, c.yl, c.yh) < r.min_units) ++x0;
        if (x1 >= x0 && chord_in_row(X, x1, c.yl, c.yh) < r.min_units) --x1;
        if (x1 >= x0) {
            c.ix = x0;
            c.x1 = x1;
            return;
        }
    }
}

__host__ __device__ __forceinline__ void cursor_start(const Ray &r, VoxelCursor &c) {
    c.done = r.empty;
    c.ok = true;
    if (c.done) return;
    const Axis &Z = r.ax[2];
    int za, zb;
    c.ok &= voxel_at(Z, r.amin, za);
    c.ok &= voxel_at(Z, r.amax - 1, zb);
    int z0 = za < zb ? za : zb, z1 = za < zb ? zb : za;
    z0 = z0 < 0 ? 0 : z0;
    c.z1 = z1 > Z.n - 1 ? Z.n - 1 : z1;
    c.iz = z0 - 1;
    c.iy = 0;
    c.y1 = -1;
    c.zl = c.zh = 0;
    cursor_next_row(r, c);
}

// Current voxel (slab, row, x) and chord; then advance.  Requires !c.done.
__host__ __device__ __forceinline__ void cursor_take(const Ray &r, VoxelCursor &c, int &iz, int &iy,
                                                     int &ix, long long &chord) {
    iz = c.iz;
    iy = c.iy;
    ix = c.ix;
    chord = chord_in_row(r.ax[0], c.ix, c.yl, c.yh);
    if (++c.ix > c.x1) cursor_next_row(r, c);
}

}  // namespace psf
