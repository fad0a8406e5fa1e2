/*
 * psf.h -- C ABI of the GB300 P-SPIR PSF system-matrix library (libpsf.so).
 *
 * Method: Sun et al., "Fast and accurate generation method of PSF-based
 * system matrix for PET reconstruction", Chinese Physics C (2016).  The
 * library builds the positional single-photon incidence response (P-SPIR)
 * tables (Sec. 2.1.1-2.1.3), the homogenization spread of every LOR over its
 * neighbouring crystal pairs (Sec. 2.2-2.3), the PSF-weighted geometric rows,
 * and the forward / back projectors used inside MLEM (Sec. 3).
 *
 * Conventions shared by every entry point
 *  - Pointers marked (device) are device pointers owned by the caller; the
 *    library never frees caller memory and never retains a caller pointer
 *    past the call, except where psf_matrix_create says so.  Pointers marked
 *    (host) are host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously on it unless the entry point
 *    says it synchronises.
 *  - Return value: PSF_OK (0) or a negative PSF_E* code; psf_strerror()
 *    describes it.  On an error nothing has been enqueued unless stated.
 *  - Crystal id = ring * Nt + block * Nb + i, Nt = n_blocks * nt_block; block
 *    b is centred at angle 2*pi*b/n_blocks, crystal i of a block at
 *    tangential offset (i - (Nb-1)/2) * (xtal_w_t + gap_t), the index growing
 *    counter-clockwise; crystal rings are centred on z = 0.
 *  - Image voxel index = (iz * ny + iy) * nx + ix; voxels are half-open boxes
 *    [o + i*d, o + (i+1)*d) on every axis.
 *  - Floating-point work is FP32 except the FP64 normalisation sums named
 *    below.
 */
#ifndef PSF_H
#define PSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSF_OK 0
#define PSF_EINVAL (-1)    /* bad argument or unsupported combination        */
#define PSF_ECAPACITY (-2) /* output buffer too small; *nnz_out = required   */
#define PSF_ECUDA (-3)     /* a CUDA runtime call failed                     */
#define PSF_ETIMEOUT (-4)  /* a bounded device-side wait gave up             */
#define PSF_EDEBUG (-5)    /* a device-side bounds check recorded a fault    */
#define PSF_ENOSCRATCH (-6) /* problem too large for the fixed scratch of
                               psf_sysmat_rows_set_noalloc                    */

/* Ring scanner of flat blocks (Sec. 3; Fig. 6 for the block corner layout). */
typedef struct {
    int32_t n_blocks;       /* R: blocks per ring (Eq. 2)                     */
    int32_t nt_block;       /* Nb: transaxial crystals per block              */
    int32_t na_block;       /* axial crystals per block                       */
    int32_t n_block_rings;  /* block rings (1 with na_block 1 = planar ring)  */
    double xtal_w_t;        /* lambda of Eq. 5: transaxial crystal width (mm) */
    double xtal_w_a;        /* axial crystal width (mm)                       */
    double depth;           /* crystal depth (mm)                             */
    double gap_t, gap_a;    /* air gap between crystals inside a block (mm)   */
    double radius;          /* axis to block front-face centre (mm)           */
    double block_gap_a;     /* axial gap between block rings (mm); must equal
                               gap_a when n_block_rings > 1                   */
    double mu;              /* linear attenuation coefficient (1/mm)          */
} psf_scanner;

/* P-SPIR table description (Sec. 2.1.1).  Incidence-angle nodes sit at
 * k * ang_max/n_ang, k = 0..n_ang-1 (transaxial angle to the face normal;
 * polar angle to the transaxial plane) and are looked up nearest-node; each
 * crystal face is cut into n_sub_t x n_sub_a entry sub-positions evaluated at
 * their centres; max_off_t x max_off_a crystal offsets along the travel
 * direction are stored per entry. */
typedef struct {
    int32_t n_ang_t, n_ang_a;
    int32_t n_sub_t, n_sub_a;
    int32_t max_off_t, max_off_a;
    double ang_max_t_deg, ang_max_a_deg;
} psf_table_desc;

/* Voxel grid; (ox, oy, oz) is the outer corner of voxel (0,0,0). */
typedef struct {
    int32_t nx, ny, nz, reserved;
    double dx, dy, dz;
    double ox, oy, oz;
} psf_image;

/* Structured LOR set of a ring scanner: transaxial pairs (a, b), a < b, with
 * Nt/2 - fan_half <= b - a <= Nt/2 + fan_half, times ordered crystal-ring
 * pairs (ra, rb) with |ra - rb| <= max_ring_diff.  Row order: transaxial pair
 * major (lexicographic), ring pair minor (lexicographic); LOR = (ra*Nt + a,
 * rb*Nt + b).  fan_half = Nt/2 - 1 on a planar ring lists all crystal pairs. */
typedef struct {
    int32_t fan_half;
    int32_t max_ring_diff;
} psf_lor_set;

typedef enum { PSF_F32 = 0, PSF_BF16 = 1, PSF_F16 = 2 } psf_dtype;
typedef enum { PSF_NORM_NONE = 0, PSF_NORM_EFF = 1, PSF_NORM_UNIT = 2 } psf_norm;

const char *psf_strerror(int code);

/* Sizes of the outputs of psf_response_build for a table description. */
int psf_table_size(const psf_table_desc *desc, int64_t *n_table, int64_t *n_eta);

/*
 * P-SPIR response table (Sec. 2.1.1, Eq. 1; normalisation Sec. 2.1.3, Eq. 6-7).
 * The GATE count ratio M_i/M of Eq. 1 is replaced by the analytic
 * first-interaction probability exp(-mu L_before)(1 - exp(-mu L_i)) of a ray
 * entering a flat crystal array (gaps are air).
 *   table (device, float) [n_ang_t][n_ang_a][n_sub_t][n_sub_a][max_off_t][max_off_a]
 *         entry (dx, dz) = crystal dx laterally / dz axially along the travel
 *         direction from the entry crystal; sub-positions counted from the
 *         edge the ray moves away from.
 *   eta   (device, double) [n_ang_t][n_ang_a][n_sub_t][n_sub_a][max_off_t + 1]
 *         FP64 prefix sums over dx of the table summed over dz:
 *         eta[..][k] = sum_{dx < k} sum_dz table[..][dx][dz], so eta[..][max_off_t]
 *         is the counting rate eta of Eq. 6 (rho0 = table / eta sums to 1).
 * PSF_EINVAL if max_off_t/max_off_a cannot hold the lateral/axial reach of the
 * largest node angle (every crystal a ray can reach must be stored).
 */
int psf_response_build(const psf_scanner *scanner, const psf_table_desc *desc, float *table,
                       double *eta, void *stream);

/*
 * Homogenization spread (Sec. 2.2 Eq. 10, Sec. 2.3 Eq. 11-12, Sec. 2.1.2
 * Eq. 2, 4, 5 for the neighbouring-block path).  For each LOR (lors[2k],
 * lors[2k+1], device int32 crystal ids) the sub-LORs joining the
 * n_sub_t*n_sub_a sub-position centres of the two crystal faces are averaged;
 * each contributes the product of the two single-photon responses.  Pairs in
 * the same transaxial block get zero.
 *   spread (device, float) [n_lors][E][E], E = (2*half_t+1)*(2*half_a+1),
 *          e = (dt + half_t)*(2*half_a+1) + (da + half_a); end 1 = lors[2k].
 *   norm   PSF_NORM_EFF: window total = untruncated mean of eta1*eta2 (FP64);
 *          PSF_NORM_UNIT: total 1; PSF_NORM_NONE: as summed.
 * table/eta are the outputs of psf_response_build for the same scanner/desc.
 */
int psf_bin_spread(const psf_scanner *scanner, const psf_table_desc *desc, const float *table,
                   const double *eta, const int32_t *lors, int64_t n_lors, int32_t half_t,
                   int32_t half_a, int32_t norm, float *spread, void *stream);

/*
 * Top-N truncation of spreads (Sec. 4.3, Table 3: the extended bins kept in
 * descending order of proportion, up to N).  For each of n_lors spreads
 * (device float [n_lors][E][E], E = (2 half_t + 1)(2 half_a + 1), e.g. the
 * output of psf_bin_spread) the window entries are ranked by weight -- a
 * negative weight ranks as 0; equal weights rank the smaller offset
 * |dt1|+|da1|+|dt2|+|da2| first, then the lower window index e1*E + e2 (the
 * paper gives no tie rule) -- and the first n_keep are written in rank order:
 * idx (device int32 [n_lors][n_keep], window index e1*E + e2) and w (device
 * float [n_lors][n_keep]), the kept weights scaled so that they sum to the
 * untruncated window's total (unscaled when the kept weights sum to 0).
 * 1 <= n_keep <= min(64, E*E) and E*E <= 2432, else PSF_EINVAL.
 */
int psf_spread_topn(const float *spread, int64_t n_lors, int32_t half_t, int32_t half_a,
                    int32_t n_keep, int32_t *idx, float *w, void *stream);

/*
 * Top-N weights in BF16 with FP32 accumulation (the list-mode step after
 * Sec. 5, no counterpart in the paper's text): for each of n_spreads rows of
 * n_keep weights (device float, e.g. psf_spread_topn's w), scale[i] = the
 * largest |w| of row i (1 when all are 0) and w16[i][k] = w[i][k] / scale[i]
 * rounded to the nearest BF16 (ties to even): device bf16 [n_spreads][n_keep],
 * device float [n_spreads], caller-owned.  1 <= n_keep <= 64, else PSF_EINVAL.
 */
int psf_spread_topn_bf16(const float *w, int64_t n_spreads, int32_t n_keep, void *w16,
                         float *scale, void *stream);

/*
 * List-mode data (the next step the paper names in Sec. 5; events stand for
 * the histogram organisation of Sec. 4, Table 1).  psf_event_rows writes the
 * row of each event's crystal pair (device int32 [n_events][2] crystal ids, in
 * either order) in the structured set, or -1 when the pair is not in it
 * (device int64 [n_events]).  psf_histogram overwrites counts (device float
 * [n_rows]) with weight times the number of events per row (rows < 0 or
 * >= n_rows are skipped).  With weight = the number of subsets, one OSEM
 * sub-iteration over a subset of events is the MLEM update of the set's
 * projector on those counts: x <- x * A^T(c / A x) / A^T 1.
 */
int psf_event_rows(const psf_scanner *scanner, const psf_lor_set *set, const int32_t *events,
                   int64_t n_events, int64_t *rows, void *stream);
int psf_histogram(const int64_t *rows, int64_t n_events, float weight, float *counts,
                  int64_t n_rows, void *stream);

/* Sinogram view and bin (device int32 [ntp] each) of every transaxial pair of
 * the set, in set order -- the histogram organisation of Sec. 4, Table 1 (192
 * angles x 199 bins for 384 crystals per ring and fan 99).  Ideal-ring reading:
 * u = a + b, view = (u mod Nt) / 2, bin = sg (b - a - Nt/2) + fan_half with
 * sg = +1 for u < Nt, else -1; one to one onto Nt/2 views x (2 fan_half + 1)
 * bins.  Row of LOR (transaxial pair T, ring pair j) = T * n_ring_pairs + j.
 * PSF_EINVAL for an odd Nt or fan_half >= Nt/2. */
int psf_sino_bins(const psf_scanner *scanner, const psf_lor_set *set, int32_t *view,
                  int32_t *bin, void *stream);

/*
 * Voxel-driven homogenization (Sec. 2.3, Eq. 11-12, Figs. 7-8): the paper's own
 * generator of the PSF matrix, for a planar scanner (one crystal ring, an image
 * of one slice).  A point source at each pixel centre emits k lines at
 * theta_i = pi i / k with proportion 1/k each; each line enters a crystal face
 * at both ends (the crystal and sub-position cell under the hit point; a hit in
 * a gap or off the faces gives nothing; a hit on a cell boundary is shared half
 * and half by the two cells -- a reading, the paper is silent), and the
 * detected pair (c1 + d1, c2 + d2), |d| <= half_t, receives rho1[d1] rho2[d2] / k
 * from the two single-photon responses (table, eta: psf_response_build; the
 * gap path of Eq. 2, 4, 5 included).  A: device float [n_lors][nx*ny], dense,
 * rows in set order (pairs outside the set are dropped), overwritten.
 * PSF_EINVAL unless the set has one crystal ring, image nz = 1, k >= 1,
 * n_lors <= 16384 and n_lors * nx * ny <= 2^31.
 */
int psf_voxel_homog(const psf_scanner *scanner, const psf_table_desc *desc, const float *table,
                    const double *eta, const psf_image *image, const psf_lor_set *set, int32_t k,
                    int32_t half_t, float *A, void *stream);

/* Number of LORs of a structured set, and of its spread classes (one per
 * transaxial pair with a < nt_block times ring difference; every LOR of the
 * set has the spread of its class by the ring's rotation and axial
 * translation symmetry). */
int psf_lor_set_size(const psf_scanner *scanner, const psf_lor_set *set, int64_t *n_lors,
                     int64_t *n_classes);

/* Writes the LORs of the set (device int32 [n_lors][2]) in row order. */
int psf_lor_set_list(const psf_scanner *scanner, const psf_lor_set *set, int32_t *lors,
                     void *stream);

/* Writes one representative LOR per spread class (device int32 [n_classes][2]),
 * in class order; feed them to psf_bin_spread to get the class spreads. */
int psf_lor_set_classes(const psf_scanner *scanner, const psf_lor_set *set, int32_t *lors,
                        void *stream);

/*
 * Spreads of all classes of a structured set (Sec. 2.2 Eq. 10, Sec. 2.3
 * Eq. 11-12), class_lors being the output of psf_lor_set_classes, spread as
 * in psf_bin_spread ([n_classes][E][E]).  Two reflections map the set's
 * classes onto each other: A, through the scanner's axial centre plane (ring
 * r -> NR-1-r for both crystals; the ring lattice has one pitch): ring
 * difference d -> -d and every axial offset negated; T, through block 0's
 * centre plane (crystal x -> (Nb-1-x) mod Nt): every transaxial offset
 * negated, and when the reflected first crystal comes after the second the
 * ends swap (the spread is transposed, d -> -d).  The smallest class index of
 * each orbit {c, Ac, Tc, ATc} goes through the spread kernel, the others are
 * its images.  Equal to psf_bin_spread on the class list up to FP32 rounding
 * (the decisions of a sub-LOR and of its image can round apart only on a
 * node or cell boundary).  Allocates 4 bytes per class of stream-ordered
 * scratch; PSF_EINVAL beyond 2^28 classes or 256 window entries per end.
 */
int psf_bin_spread_classes(const psf_scanner *scanner, const psf_table_desc *desc,
                           const float *table, const double *eta, const psf_lor_set *set,
                           const int32_t *class_lors, int32_t half_t, int32_t half_a,
                           int32_t norm, float *spread, void *stream);

/*
 * System-matrix rows (Sec. 2.3, Eq. 12: each LOR's matrix row is the sum of
 * its neighbouring geometric rows weighted by the homogenization spread; the
 * geometric rows are the ray-driven chord lengths through the image that the
 * paper's Sec. 3 reconstruction uses) in CSR (row_ptr int64 [n_lors+1], col
 * int32 sorted ascending, duplicates merged).
 *  spread == NULL: geometric rows G -- chord lengths (mm) of the segment
 *    joining the two crystals' front-face centres through the voxel grid; a
 *    voxel belongs to a row iff its chord is positive.
 *  spread != NULL: PSF rows A = S G over the listed LORs: row m is the sum of
 *    w_g[e1][e2] * G_g over every listed LOR g and window entry landing on
 *    LOR m's crystal pair (pairs outside the list are dropped).  Supported
 *    when the image has at most 49152 voxels (dense merge in shared memory);
 *    use the factored projector otherwise.
 *  val: float (PSF_F32) or bf16/fp16 (PSF_BF16/PSF_F16) with row_scale
 *    (device float [n_lors]) holding each row's FP32 scale (stored value =
 *    value / scale, scale = row max); row_scale must be NULL for PSF_F32.
 *  col == NULL: size query, only row_ptr and *nnz_out are written.
 *  capacity < nnz: PSF_ECAPACITY with *nnz_out = required nnz.
 * Synchronises `stream` once (to read nnz).  *nnz_out (host).
 */
int psf_sysmat_rows(const psf_scanner *scanner, const psf_image *image, const int32_t *lors,
                    int64_t n_lors, const float *spread, int32_t half_t, int32_t half_a,
                    int32_t dtype, int64_t *row_ptr, int32_t *col, void *val, float *row_scale,
                    int64_t capacity, int64_t *nnz_out, void *stream);

/*
 * Geometric rows G of a structured LOR set (rows in set order), the same
 * matrix psf_sysmat_rows returns for the list psf_lor_set_list writes, with
 * the same conventions, size query, capacity rule and synchronisation.  All
 * ring pairs of a transaxial pair share the transaxial projection of their
 * segment, so its crossings with the x and y planes are traced once per pair
 * and only split at each ring pair's z-plane crossings.  F32 values only.
 * PSF_EINVAL if nx + ny + 1 > 1024.  Allocates stream-ordered scratch for
 * the call: 8 bytes per 2048 rows, 80 bytes per ring pair and, when the
 * device has room, a cache of each transaxial pair's cells (about
 * 16 (nx + ny) bytes per transaxial pair) that saves the fill a second
 * tracing of the pair; freed before the call returns.
 */
int psf_sysmat_rows_set(const psf_scanner *scanner, const psf_image *image,
                        const psf_lor_set *set, int64_t *row_ptr, int32_t *col, float *val,
                        int64_t capacity, int64_t *nnz_out, void *stream);

/*
 * psf_sysmat_rows_set with a choice of value format (the mixed-precision rows
 * of the projectors used in Sec. 3's iterations): dtype PSF_F32 is exactly
 * psf_sysmat_rows_set (row_scale must be NULL); PSF_BF16 / PSF_F16 store each
 * chord divided by its row's scale, rounded to nearest, in val (device
 * uint16 [capacity]), with row_scale (device float [n_rows], written with the
 * fill) = (longest cell chord of the row's transaxial pair in the transaxial
 * plane) x (the row's length per unit of that chord) -- an upper bound of
 * the row's chords (mm), so every stored value lies in (0, 1] and the value
 * is stored x row_scale.  Columns, row pointers, size query (col == NULL:
 * row_scale may be NULL), capacity rule and synchronisation are those of
 * psf_sysmat_rows_set.  PSF_EINVAL for another dtype or a missing/extra
 * row_scale.
 */
int psf_sysmat_rows_set_typed(const psf_scanner *scanner, const psf_image *image,
                              const psf_lor_set *set, int32_t dtype, int64_t *row_ptr,
                              int32_t *col, void *val, float *row_scale, int64_t capacity,
                              int64_t *nnz_out, void *stream);

/*
 * psf_sysmat_rows_set_noalloc -- psf_sysmat_rows_set for callers that may not
 * allocate device memory.  The paper has no counterpart; this is a service
 * of the library.  Some callers cannot let a library call cudaMalloc or
 * cudaMallocAsync: an application that reserves its whole device budget at
 * start-up and forbids later allocations, a pipeline whose latency cannot
 * absorb the implicit device synchronisation of cudaMalloc, or code whose
 * memory is owned by an allocator it does not control.  This entry point
 * performs no allocation of any kind (no cudaMalloc/cudaFree, no allocating
 * library routine): its only scratch -- the scan's per-tile sums (8 bytes
 * per 2048 rows), a status word and the ring-pair z-axis table (80 bytes per
 * ring pair) -- lives in one file-scope device array of
 * PSF_NOALLOC_SCRATCH_BYTES (1 MiB) that every GPU loading the library keeps
 * until the process exits.  The caller still provides row_ptr, col and val.
 *  - Limit: a set of at most PSF_NOALLOC_MAX_ROWS rows whose tile sums and
 *    ring-pair table fit in the array together; other sets return
 *    PSF_ENOSCRATCH before any device work.
 *  - Set-up: the first call on a device (the current device) looks up the
 *    array's device address once and keeps it for later calls on that
 *    device.  The address is not looked up again, so after cudaDeviceReset (by the caller, torch
 *    or any other code in the process) this entry point must not be called
 *    again on that device in the same process.
 *  - All calls share the array and leave their contents in it: calls whose
 *    work overlaps on the GPU (different streams, or host threads) race and
 *    must be serialised by the caller.
 *  - Like psf_sysmat_rows_set it synchronises `stream` (it reads the
 *    nonzero count and the status word back to the host).
 * Arguments, results, size query and capacity rule are those of
 * psf_sysmat_rows_set.
 */
#define PSF_NOALLOC_SCRATCH_BYTES (1 << 20)
#define PSF_NOALLOC_MAX_ROWS ((int64_t)((PSF_NOALLOC_SCRATCH_BYTES - 64) / 8 - 1) * 2048)
int psf_sysmat_rows_set_noalloc(const psf_scanner *scanner, const psf_image *image,
                                const psf_lor_set *set, int64_t *row_ptr, int32_t *col,
                                float *val, int64_t capacity, int64_t *nnz_out, void *stream);

/*
 * Projector plan over caller CSR (pointers retained until destroy; the caller
 * keeps them alive).  The plan owns its scratch (allocated here).
 */
typedef struct psf_matrix psf_matrix;

int psf_matrix_create(psf_matrix **out, int64_t n_rows, int64_t n_cols, const int64_t *row_ptr,
                      const int32_t *col, const void *val, int32_t dtype, const float *row_scale,
                      void *stream);

/* A projector plan without stored rows, for list-mode reconstruction with
 * rows generated on the fly (the next step the paper names in Sec. 5): its
 * rows are the geometric rows of the structured set on the image -- the
 * rows psf_sysmat_rows_set would store, from the same exact per-LOR tracer,
 * so equal to them bit for bit -- and every projection traces the rows it
 * needs, one thread per row: psf_forward_masked only the listed sources of
 * the masked rows, psf_back after psf_matrix_build_sparse_adjoint only the
 * rows with S^T y != 0, the full projections every row.  Combine with
 * psf_matrix_set_spread / _topn for the factored form.  Not tunable
 * (psf_matrix_autotune, psf_matrix_set_launch: PSF_EINVAL); psf_back_sens
 * traces twice.  Rows < 2^31, voxels < 2^31; a tracer lookup that does not
 * settle records PSF_EDEBUG (psf_matrix_check). */
int psf_matrix_create_otf(psf_matrix **out, const psf_scanner *scanner, const psf_image *image,
                          const psf_lor_set *set, void *stream);

/* Factored PSF form A = S G (Sec. 2.3) for a structured LOR set: the rows of
 * the plan are G in set order, and S applies the class spreads
 * (device float [n_classes][E][E], kept by pointer) in LOR space. */
int psf_matrix_set_spread(psf_matrix *m, const psf_scanner *scanner, const psf_lor_set *set,
                          int32_t half_t, int32_t half_a, const float *class_spread);

/* The same factored form with top-N class spreads (the output of
 * psf_spread_topn on the class spreads: idx int32 and w float, device
 * [n_classes][n_keep], kept by pointer): S applies only each class's kept
 * entries.  S^T gathers in rank order; S scatters with FP32 atomics (the
 * last bits of a sum may vary between runs).  Replaces a previous
 * psf_matrix_set_spread, and vice versa. */
int psf_matrix_set_spread_topn(psf_matrix *m, const psf_scanner *scanner,
                               const psf_lor_set *set, int32_t half_t, int32_t half_a,
                               int32_t n_keep, const int32_t *idx, const float *w);

/* The same with the kept weights as BF16 codes and one FP32 scale per class
 * (the output of psf_spread_topn_bf16 on the class weights: w16 device bf16
 * [n_classes][n_keep], scale device float [n_classes], kept by pointer): each
 * tap's weight is code x scale, products and sums in FP32. */
int psf_matrix_set_spread_topn_bf16(psf_matrix *m, const psf_scanner *scanner,
                                    const psf_lor_set *set, int32_t half_t, int32_t half_a,
                                    int32_t n_keep, const int32_t *idx, const void *w16,
                                    const float *scale);

/* For a plan with top-N spreads (list-mode reconstruction, the next step of
 * Sec. 5): build the transpose of S -- for every measured LOR the source LORs
 * whose kept entries land on it, with their weights (plan-owned: 8 bytes per
 * kept tap, 12 bytes per LOR) -- with two passes over the taps (count, scan,
 * fill).  Afterwards S^T of an input with at most 1/16 nonzero entries (one
 * subset's counts or ratios) lists those entries and scatters from them with
 * FP32 atomics (the summation order varies between runs); denser inputs keep
 * the gather; psf_back then also lists the rows with S^T y != 0 and, when at
 * most a quarter of the rows are listed, back-projects only those (one warp
 * per listed row).  The decisions are taken on the device, so the calls stay
 * capturable.  A later psf_matrix_set_spread(_topn) drops the transpose.
 * Synchronises `stream`; PSF_EINVAL for other plans or more than 2^31 - 1
 * rows. */
int psf_matrix_build_sparse_adjoint(psf_matrix *m, void *stream);

int psf_matrix_destroy(psf_matrix *m);

/*
 * Launch tuning of the stored-row projectors (batching of rows of uneven
 * length, no counterpart in the paper).  For each direction it times, with
 * CUDA events on `stream`, the grid-stride kernels, the persistent work-queue
 * kernels (each warp takes the next chunk of rows from a counter) at chunk in
 * {1,2,4,...,128} rows and {128,256,512} threads per CTA and, for the forward
 * projection of FP32 rows, streaming tiles (64 rows per CTA, entries loaded
 * 16 bytes at a time independently of row boundaries) and the bulk-staged
 * kernels (FP32 rows with 16-byte aligned column and value arrays: chunks of
 * 4096 entries brought into shared memory by cp.async.bulk copies completing
 * on an mbarrier, one chunk ahead; each chunk owns the rows that start in it),
 * on all-ones vectors, and keeps the fastest for psf_forward / psf_back of
 * this plan; the pair back-projection of psf_back_sens takes the faster of
 * the back launch and the bulk-staged kernel (psf_back keeps launches that
 * skip rows with y = 0, which a bulk-staged pass cannot); for a
 * factored plan with full-window spreads it also times the staged forms of the
 * LOR-space spread stencil in each direction and keeps the fastest (call it after
 * psf_matrix_set_spread; the candidates are forms 3, 4 and, when it fits, 5).
 * chunk_out / threads_out: host arrays of 2
 * (forward, back), may be NULL; chunk -2 = bulk-staged, -1 = streaming tiles,
 * 0 = grid-stride, > 0 = work queue.  Synchronises; allocates a temporary
 * image-sized buffer and, for the bulk-staged forms, a plan-owned table of 8
 * bytes per 4096 entries;
 * call it outside stream capture, after which the projections of the plan can
 * be captured in a CUDA graph.
 */
int psf_matrix_autotune(psf_matrix *m, int32_t *chunk_out, int32_t *threads_out, void *stream);

/* Set that launch explicitly for both directions: chunk 0 selects the
 * grid-stride kernels; chunk in [1, 2^20] rows per take with threads a
 * multiple of 32 in [32, 1024] the work-queue kernels; chunk -1 (FP32 rows
 * only) the streaming forward (back: grid-stride); chunk -2 (FP32 rows,
 * 16-byte aligned arrays, at least one entry; synchronises the default
 * stream once to build its table) the bulk-staged kernels in every
 * direction.  PSF_EINVAL otherwise. */
int psf_matrix_set_launch(psf_matrix *m, int32_t chunk, int32_t threads);

/* Cycle limit of the library's bounded device waits (the bulk-staged
 * projectors' waits for their copies; no counterpart in the paper): a wait
 * that has not seen its event after `cycles` SM clock cycles gives up and
 * records PSF_ETIMEOUT in the plan's status word (read by psf_matrix_check);
 * the copies already in flight are still waited for, with the default limit,
 * before a CTA exits.  Default 2^31 (about a second); a negative value makes
 * the waits give up at once (a test of the timeout path).  Process-wide,
 * read at launch. */
int psf_set_wait_limit(int64_t cycles);

/* Device status of the plan's bounded waits: synchronises `stream`, returns
 * PSF_OK, or PSF_ETIMEOUT when a bulk-staged kernel gave up waiting for a
 * copy since the last call (its outputs are then incomplete), and clears it. */
int psf_matrix_check(const psf_matrix *m, void *stream);

/* Stencil form of a factored plan, both directions (no counterpart in the
 * paper): 0 the default (the fastest form that fits, or the autotuner's
 * choice), 1 the plain one-output-per-thread stencil, 2 the register-blocked
 * form, 3 and 4 the cp.async-staged forms, 5 the bulk-copy pipeline (a
 * producer warp stages each partner's ring-pair plane and weight slice with
 * cp.async.bulk into a ring of shared-memory stages; it packs the LOR-space
 * input into padded planes first and, after each psf_matrix_set_spread,
 * re-lays the class spreads out into plan-owned slices -- so with form 5 the
 * spreads are read at the first projection after psf_matrix_set_spread, and
 * changing them in place needs another psf_matrix_set_spread).  Forms that
 * do not fit the set fall back to the default.  PSF_EINVAL outside 0..5. */
int psf_matrix_set_stencil_form(psf_matrix *m, int32_t form);

/* Declare the voxel grid of the plan's columns (n_cols = nx * ny * nz, else
 * PSF_EINVAL; nx <= 65535).  No counterpart in the paper: it lets the pair
 * back-projection of psf_back_sens on a factored plan over a structured set
 * (rows in set order) accumulate each transaxial pair's rows in shared memory
 * and add each touched voxel to the image once (about 12 entries per voxel
 * on the 3D ring), instead of one global FP32-pair atomic per entry.  The
 * pair's cells are read from its direct-plane row of the middle ring; an
 * entry whose voxel is not among them, or past the shared-memory capacity,
 * takes the global atomic, so any rows give the same result up to FP32
 * summation order.  Used by default once declared (psf_matrix_autotune times
 * it against the other pair forms).  Host only; checks the division
 * constants it derives over the grid's range (grids up to 2^26 voxels;
 * PSF_EDEBUG if one fails). */
int psf_matrix_set_image(psf_matrix *m, const psf_image *image);

/*
 * x = A^T 1, the sensitivity image of MLEM (Sec. 3), x (device float
 * [n_cols], overwritten).  For a factored plan S^T 1 is formed from the class
 * spreads' window sums over in-set measured LORs (the all-ones input needs no
 * stencil), then G^T is applied; for stored rows it is psf_back of ones.
 * Equal to psf_back(m, ones) up to FP32 summation order.
 */
int psf_sensitivity(const psf_matrix *m, float *x, void *stream);

/*
 * x = A^T y and sens = A^T 1 (both device float [n_cols], overwritten) with one
 * pass over the stored rows: each entry adds its two products to an
 * interleaved image pair with one 8-byte atomic.  MLEM's first iteration
 * needs both (an initial image of ones gives the same forward projection as
 * ones on the voxels the scanner sees, because the other voxels' columns are
 * zero).  Results equal psf_back and psf_sensitivity up to FP32 summation
 * order.
 */
int psf_back_sens(const psf_matrix *m, const float *y, float *x, float *sens, void *stream);

/* Forward projection of the MLEM / OSEM iterations (Sec. 3; with a factored
 * plan A = S G of Sec. 2.3, Eq. 12, applied as G then S): y = A x
 * (overwrite), x (device float [n_cols]), y (device float [n_rows]).
 * A plan with no rows returns PSF_OK at once (y may then be NULL). */
int psf_forward(const psf_matrix *m, const float *x, float *y, void *stream);

/* Back-projection of the MLEM / OSEM iterations (Sec. 3; factored plan:
 * S^T then G^T), the exact adjoint of psf_forward: x = A^T y (overwrite);
 * with no rows x is zeroed (y may then be NULL).  The same holds for the
 * LOR-space arguments of psf_back_sens and psf_forward_masked. */
int psf_back(const psf_matrix *m, const float *y, float *x, void *stream);

/* y = A x on the rows with mask != 0 (mask: device float [n_rows],
 * non-negative, e.g. a subset's counts); every other entry of y is 0.  Only
 * the stored rows that reach a masked row are evaluated (for a factored plan:
 * the sources with S^T mask != 0), so a subset of list-mode events costs in
 * proportion to the LORs it touches.  Uses the plan's scratch; rows of the
 * plan < 2^31. */
int psf_forward_masked(const psf_matrix *m, const float *x, const float *mask, float *y,
                       void *stream);

/* MLEM steps (Sec. 3): ratio[i] = y[i] / yhat[i] (0 where yhat[i] <= 0). */
int psf_em_ratio(const float *y, const float *yhat, float *ratio, int64_t n, void *stream);

/* x[v] = x[v] * bp[v] / sens[v] where sens[v] >= floor, else 0. */
int psf_em_update(float *x, const float *bp, const float *sens, float floor, int64_t n,
                  void *stream);

/*
 * Kernel timing -- instrumentation of the library, no counterpart in the
 * paper.  While enabled, every kernel the library launches is bracketed by a
 * pair of CUDA events recorded on the launching stream, and the device time
 * between them is accumulated per kernel name.
 * psf_timing_enable(on): waits for the pending event pairs, clears the
 *   accumulators and switches recording on (on != 0) or off.
 * psf_timing_read(i, name, launches, ms): waits for the pending event pairs
 *   (synchronising with the GPU work they bracket) and returns kernel i of the
 *   accumulators: its name (valid until the next psf_timing_enable), number of
 *   launches and total milliseconds.  PSF_EINVAL past the last kernel.
 * Timing adds two event records per launch; results are unaffected.
 */
int psf_timing_enable(int32_t on);
int psf_timing_read(int32_t index, const char **name, int64_t *launches, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* PSF_H */
