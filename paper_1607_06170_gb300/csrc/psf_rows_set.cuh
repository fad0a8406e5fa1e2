// Slab walk of the structured-set row generator.
//
// The 2D cells of a transaxial pair are kept in ray order (their parameter
// boundaries are monotone there) and are also addressable in voxel order
// (ascending iy, then ix): runs of equal iy are contiguous in ray order, iy is
// monotone along the ray and so is ix inside a run.  The cells a z slab cuts
// out, a ray-order range [ca, cb], are at most three ranges of the voxel-order
// list (the part of the first run, the whole runs in between, the part of the
// last run), so a warp can copy them with consecutive lanes on consecutive
// output slots.
//
// A ring pair's z-plane crossings depend only on its two rings (z changes
// linearly from ring a's plane to ring b's along every segment of the pair),
// so each ring pair's z axis is computed once per call (ZAx) and combined with
// the transaxial pair's cells per row.  Included by psf_rows.cu (needs
// Cells2D, piece, first_cell_after, last_cell_before).
#pragma once

namespace psf {

// The pair-constant header words the slab walk uses (cell count, short-cell
// count, cells per parameter unit), read once per pair into registers.
struct CellsHead {
    int n, nflag;
    float per_unit;
};

__host__ __device__ __forceinline__ CellsHead cells_head(const Cells2D &c) {
    CellsHead h;
    h.n = c.hdr[0];
    h.nflag = c.hdr[2];
    h.per_unit = bits_float(c.hdr[13]);
    return h;
}

// Voxel-order position of ray-order cell cc (n: the pair's cell count).
__host__ __device__ __forceinline__ int sorted_pos(const Cells2D &c, int cc, bool xinc,
                                                   bool yinc, int n) {
    const int r = c.run[cc];
    const int rs = c.rstart[r], re = c.rstart[r + 1];
    const int spos = yinc ? rs : n - re;
    return spos + (xinc ? cc - rs : re - 1 - cc);
}

// The cells [ca, cb] as up to three disjoint voxel-order ranges [lo, hi],
// returned in ascending order.  Returns the number of ranges.  (Every index
// is static so the arrays stay in registers.)
__host__ __device__ __forceinline__ void cswap_range(int lo[3], int hi[3], int i, int j) {
    if (lo[j] < lo[i]) {
        int t = lo[i]; lo[i] = lo[j]; lo[j] = t;
        t = hi[i]; hi[i] = hi[j]; hi[j] = t;
    }
}

__host__ __device__ __forceinline__ int slab_segments(const Cells2D &c, int ca, int cb,
                                                      bool xinc, bool yinc, int lo[3],
                                                      int hi[3], int n) {
    const int ra = c.run[ca], rb = c.run[cb];
    int p0 = sorted_pos(c, ca, xinc, yinc, n), p1;
    if (ra == rb) {
        p1 = sorted_pos(c, cb, xinc, yinc, n);
        lo[0] = p0 < p1 ? p0 : p1;
        hi[0] = p0 < p1 ? p1 : p0;
        return 1;
    }
    p1 = sorted_pos(c, c.rstart[ra + 1] - 1, xinc, yinc, n);  // first run: ca .. end of its run
    lo[0] = p0 < p1 ? p0 : p1;
    hi[0] = p0 < p1 ? p1 : p0;
    p0 = sorted_pos(c, c.rstart[rb], xinc, yinc, n);  // last run: its start .. cb
    p1 = sorted_pos(c, cb, xinc, yinc, n);
    lo[1] = p0 < p1 ? p0 : p1;
    hi[1] = p0 < p1 ? p1 : p0;
    if (rb > ra + 1) {  // whole runs in between: one block in voxel order
        lo[2] = yinc ? c.rstart[ra + 1] : n - c.rstart[rb];
        hi[2] = yinc ? c.rstart[rb] - 1 : n - c.rstart[ra + 1] - 1;
        cswap_range(lo, hi, 0, 1);
        cswap_range(lo, hi, 1, 2);
        cswap_range(lo, hi, 0, 1);
        return 3;
    }
    cswap_range(lo, hi, 0, 1);
    return 2;
}

// The cell holding parameter al (bnd[c] <= al < bnd[c+1], al in [bnd[0],
// bnd[n])).  The boundaries are the union of two arithmetic progressions
// (the x and the y plane crossings), so the index is within two of
// proportional to al: a guess from the proportion, a few steps along the
// list, and the binary search if the steps do not settle.
__host__ __device__ __forceinline__ int cell_at(const long long *bnd, int n, long long al,
                                                float per_unit) {
    int g = (int)((float)(al - bnd[0]) * per_unit);
    g = g < 0 ? 0 : (g > n - 1 ? n - 1 : g);
    for (int it = 0; it < 6; ++it) {
        if (bnd[g + 1] <= al) {
            ++g;
        } else if (bnd[g] > al) {
            --g;
        } else {
            return g;
        }
    }
    return first_cell_after(bnd, n, al);
}

// Cells [ca, cb] overlapping the (clipped) slab interval [zl, zh), the
// number of them that keep a chord of at least minu units, and how many of
// the dropped ones are interior cells (not ca or cb).
struct SlabCells {
    int ca, cb, count, inner;
};

__host__ __device__ __forceinline__ SlabCells cut_cells(const Cells2D &c, const CellsHead &h,
                                                        long long zl, long long zh,
                                                        long long minu) {
    SlabCells s;
    s.ca = 0;
    s.cb = -1;
    s.count = 0;
    s.inner = 0;
    const int n = h.n, nflag = h.nflag;
    if (zh <= zl || n == 0) return s;
    // parameters are integers: the last cell starting before zh holds zh - 1
    const float per_unit = h.per_unit;
    s.ca = cell_at(c.bnd, n, zl, per_unit);
    s.cb = cell_at(c.bnd, n, zh - 1, per_unit);
    if (s.cb < s.ca) return s;
    int cnt = s.cb - s.ca + 1;
    if (piece(c.bnd, s.ca, zl, zh) < minu) --cnt;
    if (s.cb != s.ca && piece(c.bnd, s.cb, zl, zh) < minu) --cnt;
    int inner = 0;
    if (nflag <= SET_MAXF) {
        for (int f = 0; f < nflag; ++f) {
            const int cc = c.flag[f];
            if (cc > s.ca && cc < s.cb && c.bnd[cc + 1] - c.bnd[cc] < minu) ++inner;
        }
    } else {
        for (int cc = s.ca + 1; cc < s.cb; ++cc)
            if (c.bnd[cc + 1] - c.bnd[cc] < minu) ++inner;
    }
    s.count = cnt - inner;
    s.inner = inner;
    return s;
}

// z axis of the segments of ring pair (ra, rb) (same numbers as the per-LOR
// tracer's make_ray for any transaxial pair).
struct ZAx {
    Axis Z;
    long long lo, hi;  // parameter interval of the grid's z range (kind != 0)
    float lz;          // axial extent of the segment (mm)
    int empty;         // parallel to the z planes and outside the grid
};

__host__ __device__ __forceinline__ void zaxis_of(const Scan &sc, const Img &im, int ra, int rb,
                                                  ZAx &z) {
    const double za = sc.z064 + ra * sc.pa64, zb = sc.z064 + rb * sc.pa64;
    bool empty = false;
    make_axis(z.Z, (za - im.oz) * im.idz, (zb - im.oz) * im.idz, im.nz, empty);
    z.lo = 0;
    z.hi = 0;
    if (z.Z.kind != 0) {
        const long long p = plane_alpha(z.Z, 0), q = plane_alpha(z.Z, im.nz);
        z.lo = p < q ? p : q;
        z.hi = p < q ? q : p;
    }
    z.lz = (float)(zb - za);
    z.empty = empty;
}

// One row (transaxial pair x ring pair): z axis, clipped parameter interval,
// chord scale and its z-slab range [z0, z0 + nsl).
struct RingPair {
    Axis Z;
    long long amin, amax, minu;
    float to_mm;
    int z0, nsl;
};

__device__ __forceinline__ void rp_setup(const Cells2D &c, const ZAx *__restrict__ zt, int j,
                                         int nrp, int nz, float lx, float ly, RingPair &r) {
    r.nsl = 0;
    r.z0 = 0;
    r.amin = r.amax = r.minu = 0;
    r.to_mm = 0.0f;
    r.Z.kind = 0;
    r.Z.fixed = 0;
    r.Z.A0 = r.Z.DA = 0;
    r.Z.S = r.Z.D = 0.0;
    if (j >= nrp) return;
    const ZAx &zx = zt[j];
    r.Z = zx.Z;
    bool empty = c.hdr[0] == 0 || zx.empty;
    long long amin = c.clip[0], amax = c.clip[1];
    if (zx.Z.kind != 0) {
        amin = zx.lo > amin ? zx.lo : amin;
        amax = zx.hi < amax ? zx.hi : amax;
    }
    if (amax <= amin) empty = true;
    const float lz = zx.lz;
    const float len = sqrtf(lx * lx + ly * ly + lz * lz);
    r.amin = amin;
    r.amax = amax;
    r.minu = (long long)ceilf((float)MIN_CHORD_MM / len * (float)FX);
    r.to_mm = len * (float)(1.0 / FX);
    if (empty) return;
    int za = 0, zb = -1;
    voxel_at(r.Z, amin, za);
    voxel_at(r.Z, amax - 1, zb);
    if (za > zb) { const int t = za; za = zb; zb = t; }
    za = za < 0 ? 0 : za;
    zb = zb > nz - 1 ? nz - 1 : zb;
    r.z0 = za;
    r.nsl = zb >= za ? zb - za + 1 : 0;
}

// A row's slab-walk parameters, staged once per group in the warp's shared
// work area so that a slab lane reads its row's numbers instead of carrying
// all 32 rows' z axes in registers.
struct SlabRow {
    long long A0, DA;             // z axis, linear kind
    long long amin, amax, minu;   // clipped parameter interval, shortest stored chord
    double S, D;                  // z axis, nearly parallel kind
    float to_mm;                  // mm per parameter unit
    int z0, start;                // first slab, its flattened index in the group
    int kf;                       // axis kind | fixed voxel << 2
};

__device__ __forceinline__ void slab_row_put(const RingPair &r, int start, SlabRow &o) {
    o.A0 = r.Z.A0;
    o.DA = r.Z.DA;
    o.amin = r.amin;
    o.amax = r.amax;
    o.minu = r.minu;
    o.S = r.Z.S;
    o.D = r.Z.D;
    o.to_mm = r.to_mm;
    o.z0 = r.z0;
    o.start = start;
    o.kf = r.Z.kind | (r.Z.fixed << 2);
}

// The slab with flattened index f of a warp's 32 rows (incl: inclusive
// prefix of the rows' slab counts, held one per lane; rows: the rows'
// parameters): its row q (-1 when f >= total), slab iz and clipped parameter
// interval.  Every lane must call.
struct SlabOf {
    int q, iz;
    long long zl, zh, minu;
    float to_mm;
};

__device__ __forceinline__ void slab_of(const SlabRow *rows, int incl, int f, int total,
                                        SlabOf &s) {
    const unsigned F = 0xffffffffu;
    int q = 0;  // rows whose slabs end at or before f
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(F, incl, q + step - 1);
        if (v <= f) q += step;
    }
    q = q > 31 ? 31 : q;
    s.q = f < total ? q : -1;
    s.zl = 0;
    s.zh = 0;
    s.minu = 0;
    s.to_mm = 0.0f;
    s.iz = 0;
    if (s.q < 0) return;
    const SlabRow &R = rows[q];
    const int kf = R.kf;
    s.minu = R.minu;
    s.to_mm = R.to_mm;
    s.iz = R.z0 + (f - R.start);
    long long zl, zh;
    if ((kf & 3) == 1) {  // linear axis (nearly every row): slab() without the FP64 fields
        const long long DA = R.DA, p = R.A0 + (long long)s.iz * DA, p1 = p + DA;
        zl = p < p1 ? p : p1;
        zh = p < p1 ? p1 : p;
    } else {
        Axis Z;
        Z.kind = kf & 3;
        Z.fixed = kf >> 2;
        Z.A0 = R.A0;
        Z.DA = R.DA;
        Z.S = R.S;
        Z.D = R.D;
        slab(Z, s.iz, zl, zh);
    }
    s.zl = zl > R.amin ? zl : R.amin;
    s.zh = zh < R.amax ? zh : R.amax;
}

// Per-warp work area of the set kernels.  A fill round uses one of two
// layouts: the copy form (every cell of the round's ranges is stored, the
// ranges trimmed of dropped end cells) or the general form (a keep decision
// per cell, for rounds where a short interior cell is dropped).
constexpr int SEG_MAX = 3 * 32;
struct SetWarp {
    union {
        struct {
            int start[SEG_MAX + 32];  // range: flattened start; INT_MAX past the last
            int4 rec[SEG_MAX];        // range: voxel-order position - start, column
                                      // base of its slab, mm per unit (bits), -
        } cp;
        struct {
            int2 rs[SEG_MAX];  // range: flattened start, first voxel-order position |
                               // slab lane << 16
            int4 sa[32];       // slab: z offset, voxel-order positions of its first /
                               // last ray-order cells, keep bits of those two
            float4 sf[32];     // slab: chords of those two (mm), mm per unit, -
            long long sm[32];  // slab: shortest stored chord (units)
        } gen;
    };
    int cnt[32];       // count kernel: voxels of each row of the group
    SlabRow row[32];   // the group's rows
};

}  // namespace psf

namespace psf {
static_assert(sizeof(ZAx) == 80, "the no-allocation entry point documents 80 bytes per ring pair");
}
