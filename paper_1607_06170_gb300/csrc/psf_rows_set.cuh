// Warp-cooperative emission for the structured-set row generator.
//
// The 2D cells of a transaxial pair are kept in ray order (their parameter
// boundaries are monotone there) and are also addressable in voxel order
// (ascending iy, then ix): runs of equal iy are contiguous in ray order, iy is
// monotone along the ray and so is ix inside a run.  The cells a z slab cuts
// out, a ray-order range [ca, cb], are at most three ranges of the voxel-order
// list (the part of the first run, the whole runs in between, the part of the
// last run), so a warp can copy them with consecutive lanes on consecutive
// output slots.  Included by psf_rows.cu (needs Cells2D, ZRay, piece).
#pragma once

namespace psf {

// Voxel-order position of ray-order cell cc.
__host__ __device__ __forceinline__ int sorted_pos(const Cells2D &c, int cc, bool xinc,
                                                   bool yinc) {
    const int r = c.run[cc], n = c.hdr[0];
    const int rs = c.rstart[r], re = c.rstart[r + 1];
    const int spos = yinc ? rs : n - re;
    return spos + (xinc ? cc - rs : re - 1 - cc);
}

// The cells [ca, cb] as up to three disjoint voxel-order ranges [lo, hi],
// returned in ascending order.  Returns the number of ranges.
__host__ __device__ __forceinline__ int slab_segments(const Cells2D &c, int ca, int cb,
                                                      bool xinc, bool yinc, int lo[3],
                                                      int hi[3]) {
    const int n = c.hdr[0];
    const int ra = c.run[ca], rb = c.run[cb];
    int k = 0;
    int p0, p1;
    if (ra == rb) {
        p0 = sorted_pos(c, ca, xinc, yinc);
        p1 = sorted_pos(c, cb, xinc, yinc);
        lo[k] = p0 < p1 ? p0 : p1;
        hi[k] = p0 < p1 ? p1 : p0;
        return 1;
    }
    p0 = sorted_pos(c, ca, xinc, yinc);  // first run: ca .. end of its run
    p1 = sorted_pos(c, c.rstart[ra + 1] - 1, xinc, yinc);
    lo[k] = p0 < p1 ? p0 : p1;
    hi[k] = p0 < p1 ? p1 : p0;
    ++k;
    if (rb > ra + 1) {  // whole runs in between: one block in voxel order
        lo[k] = yinc ? c.rstart[ra + 1] : n - c.rstart[rb];
        hi[k] = yinc ? c.rstart[rb] - 1 : n - c.rstart[ra + 1] - 1;
        ++k;
    }
    p0 = sorted_pos(c, c.rstart[rb], xinc, yinc);  // last run: its start .. cb
    p1 = sorted_pos(c, cb, xinc, yinc);
    lo[k] = p0 < p1 ? p0 : p1;
    hi[k] = p0 < p1 ? p1 : p0;
    ++k;
    // the three ranges are disjoint; order them by start
    for (int i = 1; i < k; ++i)
        for (int j = i; j > 0 && lo[j] < lo[j - 1]; --j) {
            int t = lo[j]; lo[j] = lo[j - 1]; lo[j - 1] = t;
            t = hi[j]; hi[j] = hi[j - 1]; hi[j - 1] = t;
        }
    return k;
}

// Slab iz of a ring pair: parameter interval, overlapping ray-order cells and
// the number of stored voxels (pieces of at least min_units).
struct SlabCut {
    long long zl, zh;
    int ca, cb, count;
};

__host__ __device__ __forceinline__ void cut_slab(const Cells2D &c, const ZRay &zr, int iz,
                                                  SlabCut &s) {
    const int n = c.hdr[0], nflag = c.hdr[2];
    slab(zr.Z, iz, s.zl, s.zh);
    s.zl = s.zl > zr.amin ? s.zl : zr.amin;
    s.zh = s.zh < zr.amax ? s.zh : zr.amax;
    s.count = 0;
    s.ca = 0;
    s.cb = -1;
    if (s.zh <= s.zl) return;
    s.ca = first_cell_after(c.bnd, n, s.zl);
    s.cb = last_cell_before(c.bnd, n, s.zh);
    if (s.cb < s.ca) return;
    int cnt = s.cb - s.ca + 1;
    if (piece(c.bnd, s.ca, s.zl, s.zh) < zr.min_units) --cnt;
    if (s.cb != s.ca && piece(c.bnd, s.cb, s.zl, s.zh) < zr.min_units) --cnt;
    if (nflag <= SET_MAXF) {
        for (int f = 0; f < nflag; ++f) {
            const int cc = c.flag[f];
            if (cc > s.ca && cc < s.cb && c.bnd[cc + 1] - c.bnd[cc] < zr.min_units) --cnt;
        }
    } else {
        for (int cc = s.ca + 1; cc < s.cb; ++cc)
            if (c.bnd[cc + 1] - c.bnd[cc] < zr.min_units) --cnt;
    }
    s.count = cnt;
}

// z-slab range of a ring pair's segment
__host__ __device__ __forceinline__ void zray_slabs(const ZRay &zr, int nz, int &z0, int &z1) {
    int za = 0, zb = -1;
    if (!zr.empty) {
        voxel_at(zr.Z, zr.amin, za);
        voxel_at(zr.Z, zr.amax - 1, zb);
        if (za > zb) { int t = za; za = zb; zb = t; }
        za = za < 0 ? 0 : za;
        zb = zb > nz - 1 ? nz - 1 : zb;
    }
    z0 = za;
    z1 = zb;
}

// Broadcast the ring pair owned by lane `src` to the whole warp.
__device__ __forceinline__ void shfl_zray(ZRay &d, const ZRay &s, int src) {
    const unsigned F = 0xffffffffu;
    d.Z.kind = __shfl_sync(F, s.Z.kind, src);
    d.Z.fixed = __shfl_sync(F, s.Z.fixed, src);
    d.Z.n = __shfl_sync(F, s.Z.n, src);
    d.Z.inc = __shfl_sync(F, s.Z.inc, src);
    d.Z.A0 = __shfl_sync(F, s.Z.A0, src);
    d.Z.DA = __shfl_sync(F, s.Z.DA, src);
    d.Z.S = __shfl_sync(F, s.Z.S, src);
    d.Z.D = __shfl_sync(F, s.Z.D, src);
    d.Z.sf = __shfl_sync(F, s.Z.sf, src);
    d.Z.df = __shfl_sync(F, s.Z.df, src);
    d.amin = __shfl_sync(F, s.amin, src);
    d.amax = __shfl_sync(F, s.amax, src);
    d.min_units = __shfl_sync(F, s.min_units, src);
    d.to_mm = __shfl_sync(F, s.to_mm, src);
    d.empty = __shfl_sync(F, (int)s.empty, src);
}

}  // namespace psf
