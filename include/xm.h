/*
 * xm.h -- C ABI of the GB300-native sky cross-match library (libxm.so).
 *
 * The library implements the "Sky" functional case of the paper (§2.1): for
 * every source of catalogue A (the paper's first catalogue) a region -- circle,
 * ellipse or rectangle -- is centred on its position, sized by fixed values or
 * by per-source columns and oriented by a position angle with a zero-point and
 * a direction of rotation; the sources of catalogue B (the second catalogue)
 * inside that region are its members. Catalogue B is held in a sky-partitioned
 * index (§2.3), the members of each A source are then selected ("all" or
 * "best", §2.2) and joined (the five join types of §2.2).
 *
 * Conventions shared by every entry point
 *  - Every call returns an xm_status. No exception, abort or exit crosses the
 *    ABI. xm_last_error() gives a one-line reason for the last failure on the
 *    calling thread.
 *  - Arrays are passed as plain pointers plus sizes. A pointer argument is
 *    host memory or device memory as the accompanying `on_device` flag says;
 *    inputs are borrowed for the duration of the call (the library copies what
 *    it keeps) and never modified.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). All device
 *    work of a call is ordered on it. Calls that must learn a data-dependent
 *    size (xm_build_index, xm_match, xm_join) synchronise `stream` once to read
 *    it; their outputs are written by work queued on `stream`, so use them on
 *    that stream or after synchronising it.
 *  - Outputs are opaque handles owned by the library and released with the
 *    matching xm_*_free. Their device arrays stay valid until then.
 *  - Device memory comes from the allocator installed with xm_set_allocator,
 *    else from the library's block cache in front of cudaMallocAsync on the
 *    call's stream (xm_set_cache_limit).
 *  - Angles: longitudes/latitudes and position angles in degrees; region sizes
 *    in `size_unit_arcsec` arcseconds times `size_scale`; separations are
 *    returned in arcseconds (float64).
 *  - Rows are 0-based indices into the caller's catalogue arrays; -1 marks a
 *    missing side in join output. Catalogues hold at most 2^31 - 1 rows.
 */
#ifndef XM_H
#define XM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define XM_API __attribute__((visibility("default")))
#else
#define XM_API
#endif

typedef enum {
    XM_OK = 0,
    XM_EINVAL = 1,      /* invalid argument or invalid catalogue value */
    XM_ENOMEM = 2,      /* a device or host allocation failed */
    XM_ECUDA = 3,       /* a CUDA runtime call failed */
    XM_ETIMEOUT = 4,    /* a bounded wait in a kernel or on the host ran out */
    XM_EOVERFLOW = 5,   /* a result does not fit the caller's buffer or limit */
    XM_EBUSY = 6,       /* admission refused: not enough free device memory */
    XM_EUNSUPPORTED = 7 /* valid request the library does not implement */
} xm_status;

/* Coordinate systems of paper §2 (equatorial ICRS/J2000; IAU galactic). */
typedef enum { XM_FRAME_EQ = 0, XM_FRAME_GAL = 1 } xm_frame;

/* Region shapes of paper §2.1. CIRCLE uses `a` as its radius; ELLIPSE uses
 * semi-axes a (along the position angle) and b; RECT uses half-sides a (along
 * the position angle) and b. The region is the set of points whose
 * azimuthal-equidistant coordinates about the A source satisfy the shape's
 * inequality (closed boundary). */
typedef enum { XM_CIRCLE = 0, XM_ELLIPSE = 1, XM_RECT = 2 } xm_shape;

/* Match selection of paper §2.2 (a bit mask: both may be requested). */
typedef enum { XM_SEL_ALL = 1, XM_SEL_BEST = 2 } xm_selection;

/* Arithmetic of the membership test. FP64 evaluates every candidate in
 * float64. FP32_RECHECK evaluates candidates in float32 on tangent-plane
 * offsets from float64 cell centres and re-evaluates in float64 every
 * candidate whose float32 value lies inside a proven guard band around the
 * region boundary; both give the same member sets. */
typedef enum { XM_PREC_FP64 = 0, XM_PREC_FP32_RECHECK = 1 } xm_precision;

/* Join types of paper §2.2: i) 1 and 2, ii) 1 or 2, iii) all from 1 / all
 * from 2, iv) 1 not 2 / 2 not 1, v) 1 xor 2. */
typedef enum {
    XM_JOIN_AND = 0,
    XM_JOIN_OR = 1,
    XM_JOIN_ALL1 = 2,
    XM_JOIN_ALL2 = 3,
    XM_JOIN_NOT1_2 = 4,
    XM_JOIN_NOT2_1 = 5,
    XM_JOIN_XOR = 6
} xm_join_type;

/* A catalogue as columns: n positions (lon_deg[i], lat_deg[i]) in `frame`.
 * Longitudes are taken modulo 360; |lat| > 90, NaN or infinite values make the
 * call fail with XM_EINVAL. `id` (nullable) is an int64 id column kept with
 * the index. on_device: 1 if the pointers are device memory, 0 if host. */
typedef struct {
    const double* lon_deg;
    const double* lat_deg;
    const int64_t* id;
    int64_t n;
    int32_t frame;
    int32_t on_device;
} xm_columns;

/* Region of each A source (paper §2.1). A size or angle comes from its column
 * when the column pointer is non-NULL (one value per A source, same placement
 * as the A columns), else from the fixed value. Effective sizes are
 * value * size_scale * size_unit_arcsec arcsec (e.g. size_scale 0.5 turns an
 * FWHM column into a radius). The effective position angle is
 * pa_zero_deg + pa_dir * PA, counted east of north of the A catalogue's own
 * frame; pa_dir is +1 or -1. A size of zero gives an empty region (that A
 * source matches nothing); a negative or non-finite value is XM_EINVAL. */
typedef struct {
    int32_t shape;
    int32_t pa_dir;
    double a, b, pa_deg;
    const double* a_col;
    const double* b_col;
    const double* pa_col;
    double size_scale;
    double size_unit_arcsec;
    double pa_zero_deg;
} xm_region;

/* Options of the B index (the sky partition of paper §2.3). The index cuts
 * the sphere into declination zones of height zone_height_arcsec, each zone
 * into RA cells about as wide as they are high; B sources are sorted by
 * (zone, RA). 0 selects 20 arcsec. build_fp64 also stores float64 unit
 * vectors, which the FP64 path reads (it falls back to computing them). */
typedef struct {
    double zone_height_arcsec;
    int32_t build_fp64;
    int32_t deferred_check; /* 1: return without synchronising; invalid B positions (or a
                               failed sort) are then reported by every xm_match or
                               xm_match_batch on the index, which synchronise anyway. The
                               columns must stay valid until `stream` has run the build. */
} xm_index_opts;

/* Order in which the scan visits the A sources (results do not depend on it):
 * by (zone, RA) after a radix sort, which keeps the B records a warp reads
 * close together, or in input order, which skips the sort and writes the
 * per-source results and the pair list contiguously. The default is input
 * order (faster on every workload measured: dense ellipses and all-sky
 * circles). */
typedef enum { XM_A_ORDER_DEFAULT = 0, XM_A_ORDER_SORTED = 1, XM_A_ORDER_INPUT = 2 } xm_a_order;

typedef struct {
    int32_t selection; /* XM_SEL_ALL and/or XM_SEL_BEST */
    int32_t precision; /* xm_precision */
    int32_t block;     /* threads per block of the scan kernel, 0 = default */
    int32_t a_order;   /* xm_a_order */
} xm_match_opts;

typedef struct xm_index xm_index;
typedef struct xm_result xm_result;
typedef struct xm_rows xm_rows;
typedef struct xm_pending xm_pending;

/* Per-call counters (cumulative over calls on the handle's device). */
typedef struct {
    uint64_t candidates;   /* B sources tested against a region */
    uint64_t rechecked;    /* FP32 tests that fell in the guard band */
    uint64_t flipped;      /* rechecks whose FP64 decision differed from q<=1 in FP32 */
    uint64_t members;      /* (A, B) memberships found */
    uint64_t tie_resolved; /* A sources whose best pair was decided in FP64 */
    uint64_t kernel_launches;
    uint64_t sort_key_passes; /* keys moved by radix-sort passes (keys x passes) */
    uint64_t sort_pay_passes; /* of those, keys that carried a 64-bit payload */
} xm_stats;

/* ---- status and configuration ------------------------------------------ */

XM_API const char* xm_status_str(xm_status s);
/* One-line description of the last failure on this host thread ("" if none). */
XM_API const char* xm_last_error(void);
/* Library version string. */
XM_API const char* xm_version(void);

/* Installs the device allocator used by every later call (NULL restores
 * cudaMallocAsync/cudaFreeAsync). alloc returns NULL on failure; both get the
 * call's stream and ctx. */
XM_API xm_status xm_set_allocator(void* (*alloc)(size_t bytes, void* stream, void* ctx),
                                  void (*release)(void* ptr, void* stream, void* ctx), void* ctx);

/* Without an installed allocator, device blocks the library frees are kept
 * per device for reuse by later calls instead of going back to the CUDA
 * stream-ordered pool (taking a large block from the pool can hold the
 * calling thread for tens of milliseconds while copies run). A kept block
 * carries an event recorded on the freeing stream; a later allocation reuses
 * it once that event has completed, or at once on the same stream. When the
 * pool runs out, kept blocks go back to it and the allocation is retried.
 *
 * xm_set_cache_limit: at most `bytes` are kept per device (blocks past it go
 * back to the pool, oldest first, at the next free); 0 keeps nothing; a
 * negative value restores the default, half the device's memory.
 * xm_free_cached: every block kept for the current device goes back to the
 * pool, ordered on `stream` after its free point (no host wait).
 * xm_mem_info: bytes of the current device the library holds in live
 * objects and temporaries, and bytes kept for reuse (either may be NULL). */
XM_API xm_status xm_set_cache_limit(int64_t bytes);
XM_API xm_status xm_free_cached(void* stream);
XM_API xm_status xm_mem_info(int64_t* live_bytes, int64_t* kept_bytes);

/* Counters accumulated since the last reset. */
XM_API xm_status xm_get_stats(xm_stats* out);
XM_API xm_status xm_reset_stats(void);

/* Kernel timing: while enabled, the library brackets every kernel launch
 * with CUDA events on the launching stream. xm_prof_read synchronises those
 * events and returns, for the kernel whose name is given, the summed device
 * time and launch count since the last enable. */
XM_API xm_status xm_prof_enable(int32_t on);
XM_API xm_status xm_prof_read(const char* kernel, double* total_ms, int64_t* launches);
/* Name and totals of the i-th timed kernel (XM_EOVERFLOW past the end). */
XM_API xm_status xm_prof_entry(int32_t i, const char** kernel, double* total_ms,
                               int64_t* launches);

/* ---- the B index (paper §2.3, sky partitioning) ------------------------ */

/* Builds the resident, immutable index of catalogue B: ingest (longitude
 * normalisation, validity), zone and RA key per source, a stable radix sort
 * on (zone, RA key), per-zone offsets, and per-source float32 tangent-plane
 * offsets from float64 cell centres. The index keeps B's frame; an A
 * catalogue in another frame is rotated into it at match time. Synchronises
 * `stream` once. Errors: XM_EINVAL (bad opts or coordinates), XM_ENOMEM,
 * XM_ECUDA. */
XM_API xm_status xm_build_index(const xm_columns* B, const xm_index_opts* opts, void* stream,
                                xm_index** out);
/* Frees an index. Its device memory returns to the pool in the order of the
 * stream it was built on, which must still exist: work queued on other
 * streams that reads the index (matches, batches, a server's slots) must be
 * ordered before that point, e.g. by making the build stream wait on an
 * event recorded after it. NULL is a no-op. */
XM_API xm_status xm_index_free(xm_index* index);
/* n sources, zones, zone height (arcsec) and device bytes held. */
XM_API xm_status xm_index_info(const xm_index* index, int64_t* n, int64_t* zones,
                               double* zone_height_arcsec, int64_t* device_bytes);

/* ---- matching (paper §2.1 Sky case, §2.2 selection) -------------------- */

/* Finds the members of every A source among the indexed B sources and keeps
 * the selections asked for in opts->selection:
 *   ALL:  every member pair, ordered by A row then B row;
 *   BEST: per A row, the member of smallest angular separation, ties to the
 *         lowest B row (-1 / NaN when the A source has no member).
 * Synchronises `stream` once, for the pair count (the pair list of a result
 * whose member records fit 2^23 is placed and sorted on the GPU meanwhile).
 * Errors: XM_EINVAL (bad region/opts/coordinates), XM_ENOMEM, XM_ECUDA. */
XM_API xm_status xm_match(const xm_index* index, const xm_columns* A, const xm_region* region,
                          const xm_match_opts* opts, void* stream, xm_result** out);
/* xm_match in two calls, for a caller with more work to queue before the
 * match's synchronisation. xm_match_async checks the arguments and queues
 * everything of the match up to its pair count on `stream` (for host A, the
 * copy of A's columns comes first), then returns without waiting;
 * xm_match_wait takes the one synchronisation and queues the rest, giving
 * the result of xm_match. Copies of host memory queued on any stream run in
 * the order they were queued, so an input copy queued after xm_match_async
 * (an index build's, say) does not hold up this match's. Every pending match
 * must be waited for exactly once, by any host thread; until then the A and
 * region columns it was given must stay valid and unchanged, and `index`
 * alive. An error from either call leaves nothing behind (after a failed
 * xm_match_wait the pending match is gone). Errors: those of xm_match. */
XM_API xm_status xm_match_async(const xm_index* index, const xm_columns* A,
                                const xm_region* region, const xm_match_opts* opts, void* stream,
                                xm_pending** out);
XM_API xm_status xm_match_wait(xm_pending* pending, xm_result** out);
/* Frees the result's device arrays in the order of the stream it was computed
 * on (work queued there that reads them runs first); that stream must still
 * exist. */
XM_API xm_status xm_result_free(xm_result* result);

/* Device arrays of a result (valid until xm_result_free):
 *  n_pairs, a_row[n_pairs], b_row[n_pairs], sep_arcsec[n_pairs]   (ALL)
 *  n_a, count[n_a] (int32 members per A row),
 *  best_b_row[n_a] (int64, -1 = none), best_sep_arcsec[n_a] (NaN = none) (BEST)
 * Arrays of a selection that was not requested come back NULL. */
typedef struct {
    int64_t n_pairs, n_a, n_b;
    const int64_t* a_row;
    const int64_t* b_row;
    const double* sep_arcsec;
    const int32_t* count;
    const int64_t* best_b_row;
    const double* best_sep_arcsec;
} xm_result_view;
XM_API xm_status xm_result_get(const xm_result* result, xm_result_view* view);

/* ---- joins (paper §2.2) ------------------------------------------------ */

/* Builds the rows of one join type over one selection of a result. A row is
 * (a_row, b_row, sep_arcsec); a missing side is -1 / NaN. A source counts as
 * matched when it appears in the selected pairs. Row order: every row that
 * carries an A source in ascending (a_row, b_row), then the rows of unmatched
 * B sources in ascending b_row. Does not synchronise: the rows are written on
 * `stream` into room for the most rows the join can have, and the first
 * xm_rows_get reads the row count (one synchronisation of that stream).
 * Errors: XM_EINVAL (selection not in the result, bad join type), XM_ENOMEM,
 * XM_ECUDA; XM_ETIMEOUT from xm_rows_get. */
XM_API xm_status xm_join(const xm_result* result, int32_t selection, int32_t join_type,
                         void* stream, xm_rows** out);
/* Frees the rows' device arrays in the order of the stream they were written
 * on (work queued there that reads them runs first; to read them on another
 * stream, make the rows' stream wait for that work before freeing); that
 * stream must still exist. */
XM_API xm_status xm_rows_free(xm_rows* rows);

typedef struct {
    int64_t n;
    const int64_t* a_row;
    const int64_t* b_row;
    const double* sep_arcsec;
    int64_t n_unmatched_a, n_unmatched_b;
} xm_rows_view;
XM_API xm_status xm_rows_get(const xm_rows* rows, xm_rows_view* view);

/* The join of xm_join for callers that cannot allocate device memory when
 * they need it: a process or framework whose own allocator has reserved the
 * whole GPU (an allocation by this library would fail or fragment its pool),
 * or a latency-critical loop that must not enter the driver's allocator. The
 * paper has no counterpart: it is an interface addition of this library.
 * It allocates nothing. The caller passes device arrays a_row, b_row, sep of
 * `capacity` rows; the rows (same content and order as xm_join's) are
 * written there by work queued on `stream`, and *n_rows receives their
 * number. Scratch is one device array built into the library, sized for
 * results of at most 2^20 A rows and 2^23 B rows (about 16 MB, held on every
 * GPU that loads the library until the process exits); larger results are
 * XM_EOVERFLOW, as is a row count above `capacity` (*n_rows still reports
 * it, nothing is written). The current device must be the one the result
 * was computed on (else XM_EINVAL). All calls share the array: calls whose
 * work overlaps on the GPU (on different streams without ordering) race and
 * must not be made. Synchronises `stream` once, to read the row count, so it
 * must not be called while `stream` is being captured into a graph; its
 * first call on a device also looks up the array's device address, a query
 * that fails while any stream is being captured in global mode. */
XM_API xm_status xm_join_noalloc(const xm_result* result, int32_t selection, int32_t join_type,
                                 int64_t* a_row, int64_t* b_row, double* sep, int64_t capacity,
                                 int64_t* n_rows, void* stream);

/* ---- catalogue 1 split across processes (paper §2.3) --------------------- */

/* The paper's tool splits the first catalogue across processes, each
 * matching its part against the whole second catalogue. Here each process
 * (one per GPU) matches a contiguous slice of A rows against its own copy of
 * the index (xm_match); the only exchange is the set of matched B rows,
 * which the B-side joins need over all slices (a B source is unmatched only
 * if no slice matched it).
 *
 * xm_result_mark_b ORs into `bits` (device memory, (n_b + 31) / 32 words,
 * bit j of word j / 32 = B row j) the B rows of the result's selected pairs
 * (selection ALL or BEST). It does not clear `bits`. Does not synchronise.
 * Errors: XM_EINVAL (NULL argument, selection not in the result), XM_ECUDA.
 *
 * xm_join_shard builds the join rows of one slice as xm_join would for the
 * whole catalogue: `b_matched` (device, the OR over every slice's
 * xm_result_mark_b) decides which B rows are unmatched; every A row written
 * is shifted by a_row_offset (the slice's first row in the whole
 * catalogue); B-only rows are written only when with_b_rows is non-zero
 * (give it to the last slice, so that the rows of the slices, concatenated in
 * slice order, are exactly xm_join's rows of the whole catalogue), and their
 * number is in n_unmatched_b either way. Does not synchronise; xm_rows_get
 * reads the count. Errors: as xm_join; XM_EINVAL for a NULL b_matched or a
 * negative offset. */
XM_API xm_status xm_result_mark_b(const xm_result* result, int32_t selection, uint32_t* bits,
                                  void* stream);
XM_API xm_status xm_join_shard(const xm_result* result, int32_t selection, int32_t join_type,
                               const uint32_t* b_matched, int64_t a_row_offset,
                               int32_t with_b_rows, void* stream, xm_rows** out);

/* ---- the Exact Value functional case (paper §2.1) ------------------------ */

typedef enum { XM_KEY_INT64 = 0, XM_KEY_FLOAT64 = 1 } xm_key_type;

/* Matches A_i with B_j when their key columns (one per catalogue, n_a and
 * n_b values of key_type, host or device by on_device) hold the same value:
 * integers compare as integers, float64 as numbers (-0 equals +0, NaN
 * equals nothing). The result has the layout of xm_match: pairs in ascending
 * A row then B row with sep_arcsec 0, member counts, and for XM_SEL_BEST the
 * lowest matching B row (sep 0; -1 / NaN when none), so xm_join applies; it
 * holds no positions (xm_pick_pairs refuses it). B keys are sorted once
 * (stable radix sort over the key bits that differ) and bucketed; each A key
 * is searched inside one bucket. Synchronises `stream` twice. Errors: XM_EINVAL, XM_ENOMEM, XM_ECUDA,
 * XM_ETIMEOUT. */
XM_API xm_status xm_match_values(const void* a_keys, int64_t n_a, const void* b_keys, int64_t n_b,
                                 int32_t key_type, int32_t on_device, int32_t selection,
                                 void* stream, xm_result** out);

/* ---- further readings of "best pairs" (paper §2.2) ----------------------- */

/* The paper keeps "all" matches or only the "best pairs" without saying
 * whose best; XM_SEL_BEST reads it per A source. These are the other two
 * readings, over the pair list of an "all" result:
 *   XM_PICK_BEST_B  for every B source held by some pair, the pair of
 *                   smallest angular separation (ties to the lowest A row);
 *   XM_PICK_MUTUAL  the pairs that are the best pair of both their A source
 *                   (as XM_SEL_BEST) and their B source. */
typedef enum { XM_PICK_BEST_B = 1, XM_PICK_MUTUAL = 2 } xm_pick;

/* Rows (a_row, b_row, sep_arcsec; n_unmatched_* = 0) of the pairs kept by
 * `pick`, in ascending A row then B row. Separations closer than the float32
 * error bound are decided in float64 from the exact positions, so the choice
 * is the float64 one. `result` must come from xm_match on `index` with the
 * ALL selection (and BEST for XM_PICK_MUTUAL). Synchronises `stream` once.
 * Errors: XM_EINVAL (selection missing, another index), XM_EUNSUPPORTED
 * (results without positions: views of batch results, xm_match_values),
 * XM_ENOMEM, XM_ECUDA, XM_ETIMEOUT. */
XM_API xm_status xm_pick_pairs(const xm_index* index, const xm_result* result, int32_t pick,
                               void* stream, xm_rows** out);

/* ---- normalised distance and concentric regions (paper §2.2, §3) ----- */

/* The normalised distance of a pair is the factor by which A's region must be
 * scaled about A's position (same orientation) to reach B: rho / r for a
 * circle, sqrt((X/a)^2 + (Y/b)^2) for an ellipse, max(|X|/a, |Y|/b) for a
 * rectangle, with (X, Y) B's coordinates in A's region frame; members have it
 * at most 1. Over it:
 *   - the best pair of every A source by normalised distance (the member
 *     lying deepest inside the region; ties to the lowest B row), a third
 *     reading of the paper's "best pairs" (§2.2);
 *   - concentric regions (§3, ClumpPopulator): copies of each region scaled
 *     by n_scales factors s_0 < s_1 < ... in (0, 1], the matched region being
 *     the outermost. A pair's level is the first copy that holds it
 *     (dist <= s_k), n_scales when only the matched region does. */
typedef struct xm_levels xm_levels;

/* Computes, in float64 from the exact positions, the normalised distance of
 * every pair of `result` (which must come from xm_match on `index` with the
 * ALL selection), the best pair by it, and, when n_scales > 0, the level of
 * every pair and per A source the number of members inside each copy.
 * `scales` is a host array of n_scales (0..64) strictly increasing values in
 * (0, 1]. Does not synchronise: the arrays are written on `stream`.
 * Errors: XM_EINVAL (selection missing, another index, bad scales),
 * XM_EUNSUPPORTED (results without positions: views of batch results,
 * xm_match_values), XM_ENOMEM, XM_ECUDA. */
XM_API xm_status xm_levels_compute(const xm_index* index, const xm_result* result,
                                   const double* scales, int32_t n_scales, void* stream,
                                   xm_levels** out);
XM_API xm_status xm_levels_free(xm_levels* levels);

/* Device arrays of a levels result (valid until xm_levels_free):
 *  dist[n_pairs]                 normalised distance of each pair of the result
 *  best_b_row[n_a] (-1 = none), best_dist[n_a] (NaN = none)
 *  level[n_pairs] (int32, 0..n_scales), n_within[n_a * n_scales] (int32,
 *  row-major by A: members with dist <= s_k); NULL when n_scales == 0. */
typedef struct {
    int64_t n_pairs, n_a;
    int32_t n_scales;
    const double* dist;
    const int64_t* best_b_row;
    const double* best_dist;
    const int32_t* level;
    const int32_t* n_within;
} xm_levels_view;
XM_API xm_status xm_levels_get(const xm_levels* levels, xm_levels_view* view);

/* ---- batches of requests (one launch of the persistent scan) --------- */

/* One cross-match request of a batch: an A catalogue, its region (§2.1), the
 * selections to keep (§2.2) and optionally one join type applied to one of
 * them. join_type < 0 asks for no join. */
typedef struct {
    xm_columns A;
    xm_region region;
    int32_t selection;       /* XM_SEL_ALL and/or XM_SEL_BEST */
    int32_t join_type;       /* xm_join_type, or -1 */
    int32_t join_selection;  /* XM_SEL_ALL or XM_SEL_BEST: the pairs the join uses */
    int32_t reserved;
} xm_request;

typedef struct {
    int32_t precision;          /* xm_precision, for every request */
    int32_t use_graph;          /* capture the device pipeline in a CUDA graph */
    int32_t persistent_blocks;  /* blocks per SM of the persistent scan, 0 = 4 */
    int32_t a_order;            /* xm_a_order of the scan over all requests' sources */
    int64_t pair_capacity;      /* pair arena; 0 = estimate (grown and rerun if short) */
    int64_t row_capacity;       /* join-row arena; 0 = estimate (likewise) */
} xm_batch_opts;

typedef struct xm_batch xm_batch;

/* Matches every request of a batch against one resident index in one pass:
 * all A sources of all requests are ingested, sorted on (zone, RA) together
 * and scanned by one persistent kernel whose warps take 32-source chunks
 * from a device work queue, so uneven requests share the GPU evenly. The
 * device work of the pass has no host synchronisation inside, so with
 * use_graph it is captured as one CUDA graph and launched once. Per request
 * the results are those of xm_match (pairs in ascending A row then B row,
 * best pairs, member counts), plus, when a join is asked for, its A-side rows
 * (pairs and unmatched A rows as the join type takes them, in the order of
 * xm_join) and its numbers of unmatched A and B rows. Synchronises `stream`
 * once (twice if an arena was too small). Errors: as xm_match; XM_EINVAL
 * names the request. */
XM_API xm_status xm_match_batch(const xm_index* index, const xm_request* requests, int64_t n,
                                const xm_batch_opts* opts, void* stream, xm_batch** out);
/* Frees a batch. Its device memory is released in the order of the stream it
 * was computed on, which must still exist: work queued on other streams that
 * reads the batch's arrays must be ordered before that point. */
XM_API xm_status xm_batch_free(xm_batch* batch);

/* Device arrays of one request of a batch (valid until xm_batch_free). A rows
 * are the request's own rows. B-only rows of a join are not materialised
 * here (their number is n_unmatched_b); xm_batch_join builds them. */
typedef struct {
    int64_t n_a, n_pairs;
    const int64_t* a_row;
    const int64_t* b_row;
    const double* sep_arcsec;
    const int32_t* count;
    const int64_t* best_b_row;
    const double* best_sep_arcsec;
    int64_t n_rows;            /* A-side join rows */
    const int64_t* row_a;
    const int64_t* row_b;
    const double* row_sep;
    int64_t n_unmatched_a, n_unmatched_b;
} xm_batch_view;
XM_API xm_status xm_batch_get(const xm_batch* batch, int64_t request, xm_batch_view* view);

/* All rows of the request's join, B-only rows included, as xm_join builds
 * them. */
XM_API xm_status xm_batch_join(const xm_batch* batch, int64_t request, void* stream,
                               xm_rows** out);

/* Totals of a batch: A sources, pairs, and the device time of its pass (ms,
 * from events around the device work). */
XM_API xm_status xm_batch_info(const xm_batch* batch, int64_t* total_a, int64_t* total_pairs,
                               double* device_ms);

/* ---- tuning (the paper's tunables: partition resolution and parallelism,
 *      §2.3 and §4, chosen here by timed trials) ---------------------------- */

typedef struct {
    double zone_heights_arcsec[8]; /* candidate zone heights; n = 0 -> 6, 12, 24, 48 */
    int32_t n_zone_heights;
    int32_t blocks_per_sm[4];      /* candidate persistent grids; n = 0 -> 2, 4, 8 */
    int32_t n_blocks;
    int32_t repeats;               /* timed repeats per trial, 0 -> 2 (minimum kept) */
    int32_t reserved;
} xm_tune_space;

typedef struct {
    double zone_height_arcsec;  /* best zone height for the index */
    int32_t persistent_blocks;  /* best blocks per SM for batches */
    int32_t trials;             /* trials run (0 when the answer came from the cache) */
    double best_ms;             /* device time of the best trial */
} xm_tuned;

/* Picks the index zone height and the batch kernel's grid for a catalogue B
 * and a sample batch of requests by timing every combination of the
 * candidates (one index build per zone height, `repeats` batch passes per
 * grid). Answers are cached per (size of B, frame, sample) for the life of
 * the process. Errors: as xm_build_index and xm_match_batch. */
XM_API xm_status xm_autotune(const xm_columns* B, const xm_request* sample, int64_t n_sample,
                             const xm_tune_space* space, int32_t precision, void* stream,
                             xm_tuned* out);

/* ---- serving: continuous batching of requests against a resident index -- */

typedef struct {
    int32_t slots;               /* batches in flight at once (0 -> 2) */
    int32_t max_batch_requests;  /* requests per batch (0 -> 256) */
    int64_t max_batch_a;         /* A sources per batch (0 -> 2^26) */
    int64_t mem_budget_bytes;    /* device memory for requests in flight (0 -> 60 % of free,
                                    counting blocks the library keeps for reuse as free) */
    int32_t precision;           /* xm_precision */
    int32_t use_graph;           /* run each batch as a CUDA graph */
    int32_t persistent_blocks;   /* 0 -> 4 */
    int32_t reserved;
} xm_serve_opts;

typedef struct {
    int64_t submitted, completed, failed, refused;
    int64_t a_sources;            /* A sources of completed requests */
    int64_t batches;
    double p50_ms, p99_ms, max_ms;  /* latency: entry into xm_serve_submit (the copy of the
                                       request's columns included) -> results complete on
                                       the device */
    double busy_s;                /* wall time with at least one batch on the device */
    int64_t mem_in_use, mem_budget;
} xm_serve_stats;

typedef struct xm_server xm_server;

/* Opens a server on a built index (which must outlive it). Each slot is a
 * host thread with its own stream: it takes the requests waiting at the head
 * of the queue (first come, first served) while they fit the batch limits
 * and the free part of the memory budget, runs them as one xm_match_batch,
 * and marks them done; slots work concurrently, so requests that arrive
 * while others are on the GPU are admitted as soon as a slot and memory
 * free up and their work overlaps on the device. */
XM_API xm_status xm_serve_open(const xm_index* index, const xm_serve_opts* opts, xm_server** out);

/* Queues a request; its columns are copied (host or device, by on_device)
 * before it returns, so the caller may free them on return; its latency is
 * counted from the call. *ticket identifies it. XM_EBUSY when the request alone exceeds the
 * memory budget (it could never be admitted); XM_EINVAL as xm_match. */
XM_API xm_status xm_serve_submit(xm_server* server, const xm_request* request, int64_t* ticket);

/* State of a ticket: 0 queued, 1 running, 2 done, 3 failed (the batch's
 * status is returned by xm_serve_wait). */
XM_API xm_status xm_serve_poll(xm_server* server, int64_t ticket, int32_t* state);

/* Waits until the ticket is done or failed, at most timeout_ms (< 0: no
 * limit); XM_ETIMEOUT if it is still pending; the failure status otherwise. */
XM_API xm_status xm_serve_wait(xm_server* server, int64_t ticket, int32_t timeout_ms);

/* Results of a done ticket (as xm_batch_get), valid until xm_serve_release. */
XM_API xm_status xm_serve_result(xm_server* server, int64_t ticket, xm_batch_view* view);

/* Frees the ticket's results; a batch's memory returns to the budget when
 * all its tickets are released. */
XM_API xm_status xm_serve_release(xm_server* server, int64_t ticket);

XM_API xm_status xm_serve_get_stats(xm_server* server, xm_serve_stats* out);

/* Starts a new statistics window: counters and busy time restart from zero
 * and latencies are kept only for requests submitted from now on (requests
 * still in flight complete normally). mem_in_use and mem_budget are not
 * windowed. */
XM_API xm_status xm_serve_reset_stats(xm_server* server);

/* Stops the slots after the batches in flight, fails queued tickets, frees
 * everything. */
XM_API xm_status xm_serve_close(xm_server* server);

/* Copies a device array of `bytes` bytes to host memory on `stream` and
 * waits for it (convenience for callers without their own CUDA runtime). */
XM_API xm_status xm_copy_to_host(void* dst, const void* src, size_t bytes, void* stream);

/* ---- measured ceilings of this device (no counterpart in the paper) ----- */

/* The denominators of the library's rooflines, measured on the current
 * device with kernels built into the library (each the best of five
 * event-timed launches on `stream` after one untimed launch):
 *   XM_PEAK_FP32_FMA  float32 fused multiply-add rate, TFLOP/s (2 per FMA);
 *   XM_PEAK_FP64_FMA  float64 fused multiply-add rate, TFLOP/s;
 *   XM_PEAK_HBM_READ  read-only streaming bandwidth over a 4 GiB buffer
 *                     (far beyond L2), GB/s.
 * Allocates (and frees) a 4 GiB buffer for XM_PEAK_HBM_READ. Synchronises
 * `stream`. Errors: XM_EINVAL, XM_ENOMEM, XM_ECUDA. */
typedef enum { XM_PEAK_FP32_FMA = 0, XM_PEAK_FP64_FMA = 1, XM_PEAK_HBM_READ = 2 } xm_peak;
XM_API xm_status xm_measure_peak(int32_t what, double* value, void* stream);

/* ---- test hook (no counterpart in the paper) ----------------------------- */

/* Sets the look-back of the radix sort's counting passes for tests of its
 * bounded waits: spin_limit is the number of polls after which a look-back
 * gives up (0 restores the default, one to two seconds of polling), and
 * silent_tile (-1 = none) is a tile that publishes none of its status words,
 * so the look-backs after it wait on words nobody writes. A look-back that
 * gives up lets its kernel finish (that pass's output is then not sorted)
 * and the call that ran the sort returns XM_ETIMEOUT; the device stays
 * usable. The setting holds for every later sort in the process until it is
 * reset; it is for tests, not for production use. Errors: XM_EINVAL. */
XM_API xm_status xm_debug_lookback(int32_t spin_limit, int32_t silent_tile);

/* Host only, no device work: the library's galactic -> equatorial rotation
 * (row major, v_eq = m v_gal) built from the IAU frame angles of paper §2's
 * galactic coordinate system (north galactic pole at RA 192.85948 deg,
 * Dec 27.12825 deg; galactic longitude of the north celestial pole
 * 122.93192 deg). */
XM_API xm_status xm_frame_matrix(double m[9]);

#ifdef __cplusplus
}
#endif
#endif /* XM_H */
