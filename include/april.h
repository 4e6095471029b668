/*
 * april.h -- C ABI of the GB300 APRIL intermediate filter.
 *
 * APRIL (Georgiadis, Tzirita Zacharatou, Mamoulis, "Raster Interval Object
 * Approximations for Spatial Intersection Joins", arXiv 2307.01716)
 * approximates every polygon by two sorted lists of disjoint Hilbert-order
 * cell intervals on a 2^N x 2^N grid (Sec. 4.1): the A-list (every cell the
 * polygon meets) and the F-list (the cells it fully covers).  For a candidate
 * pair (r, s) from an MBR join, three merge joins decide the pair
 * (Sec. 4.2, Algorithm 2):
 *     A(r) x A(s) has no overlapping intervals        -> true negative
 *     A(r) x F(s) or F(r) x A(s) has an overlap       -> true hit
 *     otherwise                                       -> inconclusive
 *
 * Conventions
 *   - Every function returns an april_status: APRIL_OK (0), APRIL_PENDING (1)
 *     or a negative error code.  No C++ exception crosses this boundary.
 *     april_last_error() returns the text of the most recent error of the
 *     calling thread.
 *   - Coordinates are integer lattice points: the data space [0,1]^2 is the
 *     lattice {0..2^24}^2.  Cell corners and centres of any grid with a cell
 *     side of at least 2 lattice units are lattice points, so all geometric
 *     predicates are exact.
 *   - Intervals are half-open [st, end) of uint32 Hilbert ids (Sec. 3.2,
 *     Sec. 4.1).  On a 2^16 grid the end of an interval that contains the
 *     last cell (id 2^32 - 1) is stored as 0 (2^32 mod 2^32); consumers
 *     compare "last = end - 1" in uint32 arithmetic.
 *   - Device memory and streams belong to the caller.  "stream" arguments are
 *     cudaStream_t values passed as void*.  The library never frees caller
 *     memory.  Objects the library allocates (april_sets, april_ctx) are
 *     released by their *_destroy function.
 */
#ifndef APRIL_H
#define APRIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t april_status;

#define APRIL_OK 0
#define APRIL_PENDING 1
#define APRIL_ERR_INVALID_ARG (-1)      /* bad pointer, size, mode or grid */
#define APRIL_ERR_OUT_OF_RANGE_ID (-2)  /* a pair names an object id >= n_objects */
#define APRIL_ERR_OVER_BUDGET (-3)      /* a request exceeds the memory budget */
#define APRIL_ERR_CUDA (-4)             /* a CUDA runtime call failed */
#define APRIL_ERR_DEVICE_TIMEOUT (-5)   /* a bounded device wait ran out */
#define APRIL_ERR_CANCELLED (-6)        /* the request was cancelled */
#define APRIL_ERR_NO_MEMORY (-7)        /* host allocation failed */
#define APRIL_ERR_GEOMETRY (-8)         /* degenerate polygon (< 3 vertices, outside the grid) */

/* Verdict byte per pair (Algorithm 2; "refinement" is returned as
 * APRIL_INCONCLUSIVE instead of being run). */
#define APRIL_TRUE_NEGATIVE 0
#define APRIL_TRUE_HIT 1
#define APRIL_INCONCLUSIVE 2
#define APRIL_VERDICT_ERROR 0xFF        /* the pair named an out-of-range object */

/* Filter kernels (see april_filter_pairs). */
#define APRIL_MODE_PLAIN 0    /* one pair per thread, Algorithm 2 as written */
#define APRIL_MODE_WARP 1     /* one pair per warp, windowed parallel merge */
#define APRIL_MODE_BATCHED 2  /* length-binned persistent kernel, long pairs split over a CTA */
#define APRIL_MODE_BATCHED_PACKED 3 /* as BATCHED, decoding the compressed lists (Sec. 5.1) while joining */

/* A 2^order x 2^order grid of square cells of side 2^log2_cell lattice units
 * with lower-left corner (ox, oy) (Sec. 3.1: one global grid per data space;
 * Sec. 5.2: one per partition).  1 <= order <= 16, log2_cell >= 1.  The
 * global grid of order N over [0,1]^2 is {0, 0, 24 - N, N}. */
typedef struct april_grid {
    int64_t ox;
    int64_t oy;
    uint32_t log2_cell;
    uint32_t order;
} april_grid;

/* The Hilbert id (Sec. 3.2) of the cell of the grid that holds lattice point
 * (x[k], y[k]), for k < n: the cell (floor((x - ox) / 2^log2_cell),
 * floor((y - oy) / 2^log2_cell)) taken half-open; UINT64_MAX for a point
 * outside the grid.  The batched filter's triage maps MBR points to cells the
 * same way.  x, y and ids are host arrays.  Errors: APRIL_ERR_INVALID_ARG (a
 * NULL array with n > 0, a bad grid). */
april_status april_cell_ids(const april_grid *grid, const int64_t *x, const int64_t *y, uint64_t n, uint64_t *ids);

/* ---------------------------------------------------------------- errors */

/* Copies the calling thread's most recent error message (NUL-terminated,
 * truncated to buf_size) into buf.  Returns APRIL_OK. */
april_status april_last_error(char *buf, size_t buf_size);

/* --------------------------------------------------------- construction */

/* Host-side A/F interval lists of a polygon set (library-owned). */
typedef struct april_sets april_sets;

/* Builds the APRIL approximation of n_polys simple polygons (Sec. 4.1 lists;
 * construction in the spirit of Sec. 6: the cells an edge touches are found by
 * exact grid traversal, the cells between them in Hilbert order are
 * classified one gap at a time by a point-in-polygon test, Sec. 6.2).
 *
 *   xy        int32 lattice coordinates, interleaved x,y; polygon p owns
 *             vertices vert_off[p] .. vert_off[p+1]-1 (the ring is implicitly
 *             closed; either orientation).  Host memory, read only.
 *   vert_off  n_polys+1 uint64 offsets (in vertices).
 *   grid      the grid (see april_grid).  Every polygon must meet the grid.
 *   n_threads host threads to use (0 = all hardware threads).
 *   out       receives the new sets; free with april_sets_destroy.
 *
 * Cell semantics: a closed cell is in A when it meets the closed polygon and
 * in F when it lies inside it.  Lists are maximal (consecutive ids merged).
 * Errors: APRIL_ERR_INVALID_ARG (null pointers, bad grid),
 * APRIL_ERR_GEOMETRY (a polygon with < 3 vertices or outside the grid),
 * APRIL_ERR_NO_MEMORY. */
april_status april_build_sets(const int32_t *xy, const uint64_t *vert_off, uint32_t n_polys,
                              const april_grid *grid, uint32_t n_threads, april_sets **out);

/* Quantizes polygons given in data-space coordinates (doubles over the unit
 * square [0,1]^2, the paper's map extent) to the integer lattice of 2^24
 * units per side that april_build_sets takes: each coordinate becomes
 * nearest-integer(x * 2^24) with ties to even (the product is exact), clamped
 * to [0, 2^24]; consecutive equal vertices, and a closing vertex equal to the
 * first, are dropped.  out_xy (int32 pairs) needs room for every input
 * vertex, out_off for n_polys + 1 offsets.  A non-finite coordinate:
 * APRIL_ERR_INVALID_ARG.  A polygon may come out with fewer than 3
 * vertices, which april_build_sets then rejects. */
april_status april_quantize_polygons(const double *xy, const uint64_t *vert_off, uint32_t n_polys, int32_t *out_xy,
                                     uint64_t *out_off);

void april_sets_destroy(april_sets *sets);

/* Sets from interval lists computed elsewhere (another construction, another
 * space-filling curve, or lists kept on disk), for n objects on a global grid
 * of order `order` (1..16).  Object o's A-list is a_iv[2k], a_iv[2k+1] for k
 * in [a_off[o], a_off[o+1]) as [st, end) pairs, likewise its F-list from
 * f_off / f_iv; at order 16 an end of 2^32 is written as 0.  The filter only
 * needs each list sorted and disjoint (Sec. 4.2's merge), so any cell order
 * works as long as both join inputs use the same one; as for every APRIL
 * approximation, the F cells must be among the A cells (Sec. 4.1: each F
 * interval inside one A interval), which the GPU kernels rely on when they
 * order the joins.  mbr (4 int32 per object, as april_sets_mbrs) may be NULL.
 * Lists that are empty-interval, unsorted, overlapping, past the grid, or
 * with F not inside A: APRIL_ERR_INVALID_ARG. */
april_status april_sets_from_lists(uint32_t n, uint32_t order, const uint64_t *a_off, const uint32_t *a_iv,
                                   const uint64_t *f_off, const uint32_t *f_iv, const int32_t *mbr,
                                   april_sets **out);

typedef struct april_sets_info {
    uint32_t n_objects;
    uint32_t order;
    uint64_t a_intervals;        /* total A intervals */
    uint64_t f_intervals;        /* total F intervals */
    uint64_t iv_slots;           /* interval slots in the device image (with alignment padding) */
    uint64_t device_bytes;       /* bytes april_upload needs */
    uint32_t parts;              /* partitions per dimension (0: one global grid) */
    uint32_t n_entries;          /* approximations: one per object, or one per (object, partition) */
    uint32_t packed;             /* 1 after april_sets_compress */
    uint32_t reserved;
    uint64_t raw_list_bytes;     /* descriptors + intervals */
    uint64_t packed_list_bytes;  /* compressed descriptors + anchors + gaps (0 if not packed) */
} april_sets_info;

april_status april_sets_get_info(const april_sets *sets, april_sets_info *info);

/* Host view of one list of entry `entry` (the object id for sets on one
 * grid): *iv points to 2*(*n) uint32 values st0,end0,st1,... owned by the
 * sets.  which: 0 = A-list, 1 = F-list. */
april_status april_sets_list(const april_sets *sets, uint32_t entry, int which, const uint32_t **iv,
                             uint32_t *n);

/* Closed MBR of every object in lattice units: mbr[4o .. 4o+3] = x0, y0, x1,
 * y1 (caller-owned host array of 4 * n_objects int32). */
april_status april_sets_mbrs(const april_sets *sets, int32_t *mbr);

/* Lengths of every entry's lists: a_len[e] and f_len[e] receive |A| and |F|
 * of entry e, for e < info.n_entries (caller-owned host arrays). */
april_status april_sets_lengths(const april_sets *sets, uint32_t *a_len, uint32_t *f_len);

/* Entries of object `obj`: *first .. *first + *count - 1 (one entry, the
 * object itself, for sets on one grid). */
april_status april_sets_object_entries(const april_sets *sets, uint32_t obj, uint32_t *first, uint32_t *count);

/* Partition id and grid of an entry of partitioned sets. */
april_status april_sets_entry_grid(const april_sets *sets, uint32_t entry, uint32_t *pid, april_grid *grid);

/* The entries each candidate pair is evaluated on (host call; Sec. 5.2): for
 * sets on one global grid the objects themselves; for partitioned sets the
 * two objects' entries for the partition that holds the lower-left corner of
 * MBR(r) n MBR(s), the partition april_filter_pairs routes the pair to.
 * er[k], es[k] receive the entries of pair k (caller-owned host arrays of n),
 * or UINT32_MAX for an out-of-range id.  R and S must be on the same grid. */
april_status april_route_pairs(const april_sets *R, const april_sets *S, const uint32_t *pr, const uint32_t *ps,
                               uint64_t n, uint32_t *er, uint32_t *es);

/* Builds partitioned sets for both join inputs (Sec. 5.2, "Partitioning").
 * The data space [0, 2^24]^2 is split into parts x parts equal partitions
 * (parts a power of two, 1..4096).  Each polygon gets one approximation (an
 * "entry") for every partition its closed MBR meets, on that partition's own
 * grid of the given order.  A partition's raster area is the smallest square
 * of power-of-two side, with its corner on a multiple of its cell side, that
 * covers the MBRs of all polygons of R and S that meet the partition.  A
 * candidate pair is evaluated in the partition holding the lower-left corner
 * of MBR(r) n MBR(s) (reference-point duplicate avoidance), which
 * april_filter_pairs and april_host_filter apply by themselves.  Polygon
 * arguments as for april_build_sets; both sets are returned. */
april_status april_build_partitioned_sets(const int32_t *r_xy, const uint64_t *r_vert_off, uint32_t r_n,
                                          const int32_t *s_xy, const uint64_t *s_vert_off, uint32_t s_n,
                                          uint32_t parts, uint32_t order, uint32_t n_threads, april_sets **out_r,
                                          april_sets **out_s);

/* Adds compressed copies of every list (Sec. 5.1, "Compression": delta
 * encoding, decoded while joining): the endpoint sequence
 * st_0 < end_0 < st_1 < ... of a list is cut into blocks of 32 endpoints.  A
 * block is its first endpoint (uint32 anchor) and the 31 gaps to the next
 * endpoints, stored as uint16 when all 31 fit, else as uint32.  The kernels
 * of APRIL_MODE_BATCHED_PACKED decode the blocks in registers while joining.
 * The raw lists stay available. */
april_status april_sets_compress(april_sets *sets);

/* Host view of a compressed list of n intervals: blocks[2b] is block b's
 * anchor and blocks[2b+1] = off | wide << 31 locates its 32 gap slots at
 * gaps + 64 * off (uint32 slots when wide, else uint16; slot 0 unused). */
april_status april_sets_packed_list(const april_sets *sets, uint32_t entry, int which, const uint32_t **blocks,
                                    const uint8_t **gaps, uint32_t *n);

/* ------------------------------------------------------------ device sets */

/* Device image of a set, as written by april_upload.
 *   desc: n_entries records of 4 uint32 {a_off, a_len, f_off, f_len};
 *         offsets count intervals from iv and are even (16-byte aligned).
 *   iv:   iv_slots intervals of 2 uint32 {st, end}.
 *   The partition and compressed arrays are set when the sets have them,
 *   else NULL.  All pointers are device addresses inside the caller's buffer. */
typedef struct april_dev_sets {
    const uint32_t *desc;       /* per entry {a_off, a_len, f_off, f_len} */
    const uint32_t *iv;         /* intervals {st, end} */
    uint32_t n_objects;
    uint32_t order;
    uint64_t iv_slots;
    uint32_t n_entries;         /* entries (== n_objects on one grid) */
    uint32_t parts;             /* partitions per dimension, 0 = one grid */
    const int32_t *obj_ll;      /* parts > 0: per object (x0, y0), lower-left MBR corner */
    const uint32_t *obj_entry;  /* parts > 0: n_objects + 1 entry offsets */
    const uint32_t *entry_pid;  /* parts > 0: partition id of every entry */
    const uint32_t *pdesc;      /* compressed: per entry {a_block, a_len, f_block, f_len} */
    const uint32_t *anchors;    /* compressed: block table, per block {anchor, gap_off64 | wide << 31} */
    const uint8_t *gaps;        /* compressed: gap blocks (64 or 128 bytes each) */
    const int32_t *mbr;         /* per object {x0, y0, x1, y1}: closed MBR in lattice units */
    const uint32_t *posts;      /* skip index: the last cell of interval slot 16 q + 15, per q */
    int64_t grid_ox;            /* grid_known: the grid the lists were built on (lattice origin, */
    int64_t grid_oy;            /*   log2 of the cell side); the batched filter's triage maps */
    uint32_t grid_log2_cell;    /*   MBR points to cells with it */
    uint32_t grid_known;        /* 1: built from polygons (april_build_sets, april_build_sets_device,
                                   april_build_partitioned_sets) */
    const int64_t *part_grid;   /* parts > 0 and grid_known: per partition {ox, oy, log2_cell, used} */
    uint64_t grid_id;           /* grid_known: fingerprint of the grid(s); the triage needs R's == S's */
} april_dev_sets;

/* Copies the sets into a caller-allocated device buffer of at least
 * info.device_bytes bytes (256-byte aligned), asynchronously on stream, and
 * fills *out; a small kernel on the same stream then derives the interval
 * slots' skip index (posts) that the filter's start searches read.  The host
 * sets must stay alive until the copy completed.  The filter entry points
 * need the sets as these calls (or april_build_sets_device) lay them out:
 * interval slots starting 256-byte aligned, with their skip index. */
april_status april_upload(const april_sets *sets, void *dev_buf, size_t dev_bytes, void *stream,
                          april_dev_sets *out);

/* ---------------------------------------------------------------- context */

typedef struct april_ctx april_ctx;

/* Creates a filter context on CUDA device `device`.  The context owns a
 * 256-byte device status block (allocated here with cudaMalloc) that kernels
 * use to report out-of-range ids and exhausted waits.  A context is used by
 * one host thread at a time: the filter calls update its captured graph and
 * april_set_tune / april_autotune its tuning, without locks.  Threads that
 * filter concurrently each create their own context. */
april_status april_ctx_create(int device, april_ctx **out);
void april_ctx_destroy(april_ctx *ctx);

/* ------------------------------------------------------------------ tuning */

/* Knobs of APRIL_MODE_BATCHED (a build-side addition; the paper's CPU
 * filter has none).  Defaults: {0xFFFFFFFF, 4, 32, 128, 0, -, 2, 0, 0}: the
 * triage first (where it applies), then every pair it left joined by a group
 * of 4 lanes with windows of 32 intervals per list, galloping (a window that
 * advances one list only is followed by a search of that list), AA first
 * after the triage; the long-pair scope (cta_threshold, cta_window) is off. */
typedef struct april_tune {
    uint32_t cta_threshold;  /* pairs with |A(r)| + |A(s)| above this ("long pairs") are joined
                                first, each by one warp or by a whole CTA (see cta_window) */
    uint32_t group_lanes;    /* lanes that share one pair below the threshold: 4, 8, 16 or 32 */
    uint32_t group_window;   /* first window of such a join, intervals per list: a power of two
                                in [group_lanes, 8 * group_lanes]; later windows double */
    uint32_t cta_window;     /* first window of a long pair's join, a power of 2: 32..128 = the
                                pair is joined by one warp (eight long pairs per CTA at once),
                                256..2048 = by the whole CTA */
    uint32_t blocks_per_sm;  /* persistent grid: CTAs per SM (0 = as many as fit) */
    float ms;                /* output of april_autotune: best time of the sample (ms) */
    uint32_t join_order;     /* order of a pair's joins in the batched kernels (the verdicts are
                                the same, Sec. 4.2): 0 = AF, AA, FA (a true hit from AF takes
                                one join); 1 = AA, AF, FA, Algorithm 2's (a true negative takes
                                one join); 2 (default) = 1 for the pairs the triage left, else 0 */
    uint32_t escalate_windows; /* 0, or 1..64: a join of the lane groups that still runs after
                                this many windows is handed, at the position it reached, to a
                                second kernel that joins it by a whole warp (first window
                                2 * cta_window when that is below 256, else 128) */
    uint32_t triage_off;     /* 0 (default): with no long-pair threshold, lane groups of 4..16 and
                                sets built from polygons on the same grid(s) (grid_known, equal
                                grid_id; raw or compressed, one grid or partitioned), a
                                triage pass first settles the pairs whose MBR-intersection centre
                                cell lies in A(r) and F(s) or in F(r) and A(s) (true hits); 1: off */
} april_tune;

april_status april_set_tune(april_ctx *ctx, const april_tune *tune);
april_status april_get_tune(const april_ctx *ctx, april_tune *tune);

/* Counts of the batched pipeline's CUDA graph on this context since its
 * creation: captures (one for every new argument set or tuning) and launches
 * (one per APRIL_MODE_BATCHED / BATCHED_PACKED call).  Either pointer may be
 * NULL.  Host-only; no device work. */
april_status april_ctx_graph_stats(const april_ctx *ctx, uint64_t *captures, uint64_t *launches);

/* Times APRIL_MODE_BATCHED on the given pairs (typically a sample of the
 * workload) for a grid of candidate tunings, keeps the
 * fastest in the context, and returns it in *out (candidates: cta_threshold in
 * {2048, 4096, 8192, 16384, none} x (group_lanes, group_window) in
 * {(4,8), (4,16), (8,16), (8,32), (16,32), (16,64), (32,64)} x long pairs by a
 * warp (cta_window 64 or 128) or by the CTA (the context's cta_window if >= 256,
 * else 256) x join_order in {0, 1}).  The context's current tuning is timed
 * first and is kept unless a candidate is more than 2% faster, so that
 * repeated runs settle on the same tuning.  Arguments as for
 * april_filter_pairs; synchronizes `stream`. */
april_status april_autotune(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                            const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *d_verdict,
                            void *d_scratch, size_t scratch_bytes, void *stream, april_tune *out);

/* ------------------------------------------------------------------ filter */

/* Device scratch (bytes) april_filter_pairs needs for `mode` and n pairs.
 * PLAIN and WARP need none; BATCHED and BATCHED_PACKED need 256 bytes of
 * work counters plus 16 bytes per pair (the list of long pairs or of the
 * pairs the triage left, for partitioned sets each pair's two routed
 * entries, and a queue of joins
 * handed from the lane groups to whole warps with room for a quarter of the
 * pairs), each part rounded up to 256 bytes. */
april_status april_filter_scratch_bytes(int mode, uint64_t n, size_t *bytes);

/* Runs the APRIL intermediate filter (Algorithm 2) on n candidate pairs.
 *
 *   R, S       device sets from april_upload (same grid).
 *   d_r, d_s   device arrays of n uint32 object ids (pair k = (d_r[k], d_s[k])).
 *   d_verdict  device array of n bytes; receives APRIL_TRUE_NEGATIVE,
 *              APRIL_TRUE_HIT, APRIL_INCONCLUSIVE, or APRIL_VERDICT_ERROR for
 *              a pair with an out-of-range id.
 *   mode       APRIL_MODE_PLAIN / _WARP / _BATCHED / _BATCHED_PACKED.  Partitioned
 *              sets (april_build_partitioned_sets) need one of the BATCHED
 *              modes: each pair is first routed to the partition of the
 *              lower-left corner of MBR(r) n MBR(s) (Sec. 5.2).  BATCHED_PACKED
 *              needs compressed sets (april_sets_compress) and decodes their
 *              blocks while the same kernels join them.
 *   d_scratch  device scratch of april_filter_scratch_bytes() bytes
 *              (256-byte aligned), or NULL when that is 0.
 *   stream     cudaStream_t (void*); all work is enqueued on it.
 *
 * APRIL_MODE_BATCHED enqueues a CUDA graph (counter reset, partition
 * routing for partitioned sets, the triage or the length binning as the
 * tuning says, the persistent lane-group filter) that is captured on first
 * use of an argument set and
 * replayed afterwards; the context's tuning (april_set_tune /
 * april_autotune) applies.  Calls on one context must not overlap in time
 * from several host threads.
 *
 * Asynchronous: launch errors are returned at once; device-side errors (an
 * out-of-range id, an exhausted bounded wait) are recorded in the context and
 * returned by april_sync_status.  n == 0 is a no-op. */
april_status april_filter_pairs(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *d_verdict,
                                int mode, void *d_scratch, size_t scratch_bytes, void *stream);

/* End-to-end variant for host data: copies the n pairs from host memory to the
 * device, runs april_filter_pairs, copies the n verdicts back to host memory,
 * and waits for the stream.  h_r, h_s and h_verdict are host arrays (pinned
 * memory makes the copies asynchronous DMA); d_work is a caller-allocated
 * device buffer of april_filter_host_work_bytes() bytes (256-byte aligned)
 * that holds the staged pairs, the verdicts and the mode's scratch.  In the
 * batched modes the pairs are pipelined in up to 8 chunks, on streams of the
 * context (created on first use) that follow the work queued on `stream`
 * before the call and that `stream` waits for.  Where the triage runs (see
 * april_tune.triage_off), the chunks double from 2^18 to 2^21
 * pairs (the last takes what is left), each is triaged as soon as it has
 * been copied in while the next one is, and one lane-group launch over the
 * pairs left follows before the verdicts are copied out.  Otherwise the
 * chunks hold at least 2^22 pairs, and a chunk's pairs are copied in while
 * the previous chunk is filtered and its verdicts copied out while the next
 * is.  The verdicts are those of one
 * april_filter_pairs call over all n pairs.  Returns the same codes as
 * april_filter_pairs followed by april_sync_status. */
april_status april_filter_host_work_bytes(int mode, uint64_t n, size_t *bytes);
april_status april_filter_pairs_host(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                     const uint32_t *h_r, const uint32_t *h_s, uint64_t n, uint8_t *h_verdict,
                                     int mode, void *d_work, size_t work_bytes, void *stream);

/* Filter variants (paper Sec. 4.3.2 and Sec. 5.3) on sets built on global
 * grids, by the batched kernels (long pairs by CTAs, the rest by warps).
 *   predicate APRIL_PREDICATE_INTERSECTS: Algorithm 2 when R and S use the
 *     same order; when they differ (Sec. 5.3, "Different Granularity") the
 *     finer side's intervals are coarsened while they are read,
 *     [st, end) -> [st >> n, ((end - 1) >> n) + 1) with n = 2 |order_r - order_s|,
 *     and the filter is AA then the one join with the coarse side's F-list
 *     (A(r') x F(s) when r is finer, F(r) x A(s') when s is finer).
 *   predicate APRIL_PREDICATE_WITHIN (Sec. 4.3.2, "Spatial Within Joins";
 *     equal orders): AA (no overlap: APRIL_TRUE_NEGATIVE, r is not within s),
 *     then whether every A(r) interval lies inside one F(s) interval
 *     (APRIL_TRUE_HIT: r is within s) or not (APRIL_INCONCLUSIVE).
 * Other arguments and the scratch size are those of april_filter_pairs with
 * APRIL_MODE_BATCHED; the context's cta_threshold applies.  For
 * APRIL_PREDICATE_INTERSECTS on different orders with no long-pair threshold
 * (the default tuning), triage_off 0, and sets built from polygons on one
 * grid each with the same origin and extent (grid_ox, grid_oy and
 * grid_log2_cell + order equal), a first pass settles as APRIL_TRUE_HIT the
 * pairs whose MBR-intersection centre lies in a coarse cell c of the coarse
 * side's F-list while the finer side's A-list meets the fine cells of c; the
 * verdicts are the same. */
#define APRIL_PREDICATE_INTERSECTS 0
#define APRIL_PREDICATE_WITHIN 1
april_status april_filter_pairs_ex(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                   const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *d_verdict,
                                   int predicate, void *d_scratch, size_t scratch_bytes, void *stream);

/* Waits for `stream`, then returns and clears the context's device status:
 * APRIL_OK, APRIL_ERR_OUT_OF_RANGE_ID or APRIL_ERR_DEVICE_TIMEOUT (or
 * APRIL_ERR_CUDA if the stream itself failed). */
april_status april_sync_status(april_ctx *ctx, void *stream);

/* ----------------------------------------------------------------- serving */

/* A serving loop over resident sets (a build-side addition; the paper runs
 * one join at a time).  Requests (lists of candidate pairs in host memory)
 * are queued by april_submit and admitted in arrival order by a runtime
 * thread whenever one of max_inflight stream slots is free and the request's
 * device buffers fit in the caller's arena (the memory budget).  Each
 * admitted request is copied in, filtered by the batched kernels (at most one
 * CTA per 256 pairs, so small requests share the GPU with the others) and
 * copied out on its own stream; requests on different slots run
 * concurrently.  max_inflight = 1 serves one request per launch.  Nothing on
 * the device waits on the host: completion is detected with CUDA events. */
typedef struct april_server april_server;

typedef struct april_req_stats {
    uint64_t n_pairs;
    int64_t submit_ns;  /* host steady clock, nanoseconds */
    int64_t admit_ns;   /* when its copy-in and kernels were enqueued */
    int64_t done_ns;    /* when the runtime saw its verdicts land in host memory */
    uint32_t slot;
    int32_t status;
} april_req_stats;

typedef struct april_server_info {
    uint64_t admitted;
    uint64_t completed;
    uint64_t pending;
    uint64_t in_flight;
    uint64_t max_concurrent;    /* most requests on the device at once so far */
    uint64_t arena_bytes;
    uint64_t arena_peak_bytes;  /* most arena bytes in use at once so far */
} april_server_info;

/* Creates a server for sets R and S (already uploaded; they stay resident).
 * d_arena/arena_bytes: caller-allocated device memory (256-byte aligned) that
 * bounds all request buffers: a request of n pairs needs about 25 n bytes.
 * max_inflight: 1..64 stream slots.  The context must outlive the server,
 * and while the server runs its worker thread reads the context's tuning:
 * leave that context to the server (no april_set_tune, april_autotune or
 * filter calls on it) and filter elsewhere through another context. */
april_status april_server_create(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S, void *d_arena,
                                 size_t arena_bytes, uint32_t max_inflight, april_server **out);

/* Queues a request of n pairs (h_r[k], h_s[k]); its verdicts will be written
 * to h_verdict (n bytes).  The three host buffers must stay valid until the
 * request is done (pinned memory makes the copies asynchronous).  Never
 * blocks on the GPU.  Returns APRIL_ERR_OVER_BUDGET if the request alone
 * needs more than the whole arena. */
april_status april_submit(april_server *server, const uint32_t *h_r, const uint32_t *h_s, uint64_t n,
                          uint8_t *h_verdict, uint64_t *ticket);

/* APRIL_PENDING while the request is queued or running; otherwise fills
 * *stats (optional), forgets the ticket and returns APRIL_OK or the
 * request's error (APRIL_ERR_OUT_OF_RANGE_ID, APRIL_ERR_CANCELLED,
 * APRIL_ERR_CUDA). */
april_status april_poll(april_server *server, uint64_t ticket, april_req_stats *stats);

/* As april_poll, but first waits up to timeout_ms for the request to finish
 * (returns APRIL_PENDING if it has not). */
april_status april_wait(april_server *server, uint64_t ticket, uint32_t timeout_ms, april_req_stats *stats);

/* Cancels a request that is still queued (APRIL_OK; its poll then returns
 * APRIL_ERR_CANCELLED).  A request already on the device runs to completion
 * (returns APRIL_PENDING). */
april_status april_cancel(april_server *server, uint64_t ticket);

april_status april_server_get_info(april_server *server, april_server_info *info);

/* Cancels queued requests, waits for the ones on the device, and frees the
 * server (not the arena, which belongs to the caller). */
void april_server_destroy(april_server *server);

/* ------------------------------------------------- allocation-free filter */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they filter -- code that runs where
 * cudaMalloc is not allowed or would stall the device (a latency-bound
 * serving loop, a plugin whose host owns all allocations).  It runs the same
 * computation as april_filter_pairs(..., APRIL_MODE_BATCHED, ...) with the
 * default tuning, but without a context and without caller scratch: its
 * scratch is a static device array inside libapril (16 MiB + 512 bytes),
 * which every GPU that loads the library holds until the process exits.
 *
 *   R, S, d_r, d_s, n, d_verdict, stream: as for april_filter_pairs.
 *
 * It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * call.  The first call on a device (with that device current) loads the
 * library's kernel module if nothing else has, which commits the array's
 * device memory, and queries the launch shape: make that first call as a
 * warm-up, outside the latency-bound path and before any stream capture.
 * The array's device address is looked up on every call (cudaGetSymbolAddress,
 * which does not allocate).  All calls share the one array and each call
 * clears its counters first: calls whose work overlaps on the GPU (several
 * streams or host threads) race and must be serialized by the caller.
 * Out-of-range ids give APRIL_VERDICT_ERROR verdicts.  Device errors (bad
 * ids, a bounded wait that ran out) are recorded in the array's status word,
 * which keeps them across calls until april_noalloc_sync_status reads it.
 * After a timeout the verdicts of the pairs the stopped warps held read
 * APRIL_VERDICT_ERROR and pairs no warp reached keep their old contents:
 * treat every verdict of the calls since the last status query as invalid.
 * n larger than APRIL_NOALLOC_MAX_PAIRS is rejected with APRIL_ERR_INVALID_ARG.
 * Asynchronous on `stream`. */
#define APRIL_NOALLOC_MAX_PAIRS 4194304u
april_status april_filter_pairs_noalloc(const april_dev_sets *R, const april_dev_sets *S, const uint32_t *d_r,
                                        const uint32_t *d_s, uint64_t n, uint8_t *d_verdict, void *stream);

/* The paper has no counterpart; the status query of april_filter_pairs_noalloc
 * on the current device, for the same callers (it allocates nothing either).
 * Synchronizes `stream`, reads the status word of the static array and
 * clears it.  Returns APRIL_OK, APRIL_ERR_DEVICE_TIMEOUT (a bounded device
 * wait ran out in one of the calls since the last query) or
 * APRIL_ERR_OUT_OF_RANGE_ID (a pair named an out-of-range id), or
 * APRIL_ERR_CUDA. */
april_status april_noalloc_sync_status(void *stream);

/* ------------------------------------------------- diagnostics */

/* The paper has no counterpart; a diagnostic for the error path of the
 * filter kernels.  Every wait of a filter kernel for its window copies gives
 * up after `spins` polls of its mbarrier (default APRIL_WAIT_LIMIT_DEFAULT);
 * the kernel then waits (with the default limit) for the copies in flight,
 * marks the pairs it held as APRIL_VERDICT_ERROR, records
 * APRIL_ERR_DEVICE_TIMEOUT in the status word and stops.  spins = 0 makes
 * every such wait give up at once, so the timeout path can be run without
 * any fault.  Applies to the current device, to every context and to the
 * allocation-free entry point, until set again; set it only while no filter
 * kernel runs.  Synchronous.  Returns APRIL_OK or APRIL_ERR_CUDA. */
#define APRIL_WAIT_LIMIT_DEFAULT 16777216u
april_status april_debug_set_wait_limit(uint32_t spins);

/* ------------------------------------------------- construction on the GPU */

/* Builds the APRIL approximation of polygons that are in device memory and
 * writes the device image the filter reads, on the GPU (Sec. 4.1 lists,
 * constructed as in Sec. 6: touched cells per edge, sorted by Hilbert id,
 * one point-in-polygon test per gap).  The lists equal april_build_sets'
 * list for list (same exact arithmetic; the lists are canonical).
 *   d_xy, d_vert_off  device arrays as for april_build_sets: int32 lattice
 *                     (x, y) pairs and n_polys + 1 uint64 vertex offsets
 *                     (8-byte aligned).
 *   grid              as for april_build_sets.
 *   d_work            device work buffer (256-byte aligned) of at least
 *                     info->work_bytes; a call with a smaller one (or NULL)
 *                     returns APRIL_ERR_OVER_BUDGET with info->work_bytes set
 *                     to what counting needs, and the next call with that
 *                     much reports the full sizes.
 *   d_image           device image buffer (256-byte aligned) of at least
 *                     info->image_bytes: descriptors, MBRs, interval
 *                     slots (each polygon's lists in a slot range sized from
 *                     its cell count; unused slots are never read) and the
 *                     slots' skip index.
 *   out               receives the device sets (no partitions, no packed
 *                     lists); pointers into d_image.
 * The call counts cells on the device and synchronizes the stream once to
 * read the sizes (filled into *info even when a buffer is too small, in
 * which case it returns APRIL_ERR_OVER_BUDGET and builds nothing); the
 * construction itself is then enqueued asynchronously on `stream`.
 * A polygon with fewer than 3 vertices, outside the grid or meeting no cell:
 * APRIL_ERR_GEOMETRY naming the first such polygon. */
typedef struct april_device_build_info {
    uint64_t touched_cells;  /* cell incidences of all edges (before merging) */
    uint64_t work_bytes;     /* work buffer bytes the build needs */
    uint64_t image_bytes;    /* image buffer bytes the build needs */
    uint64_t iv_slots;       /* interval slots reserved in the image */
} april_device_build_info;

april_status april_build_sets_device(april_ctx *ctx, const int32_t *d_xy, const uint64_t *d_vert_off,
                                     uint32_t n_polys, const april_grid *grid, void *d_work, size_t work_bytes,
                                     void *d_image, size_t image_bytes, april_dev_sets *out,
                                     april_device_build_info *info, void *stream);

/* ------------------------------------------------------ selection queries */

/* Selection queries (Sec. 4.3.1): the data polygons R are pre-processed
 * (APRIL lists on the device plus a bucket index over their MBRs); a batch of
 * query polygons Q, with its own APRIL lists on the same grid, is answered by
 * one april_select call: every pair (r, q) whose closed MBRs meet is found on
 * the GPU and filtered (true negative / true hit / inconclusive), the pairs
 * grouped by query.
 *
 * The index is a uniform grid of 2^bucket_bits x 2^bucket_bits buckets over
 * the lattice square; an object is listed in every bucket its MBR meets.
 * bucket_bits 0 picks about one object per bucket; at most 12.  R must be
 * built on one global grid (not partitioned).  Errors: APRIL_ERR_INVALID_ARG,
 * APRIL_ERR_NO_MEMORY. */
typedef struct april_index april_index;

typedef struct april_index_info {
    uint32_t bucket_bits;
    uint32_t n_objects;
    uint64_t n_entries;     /* object copies over all buckets */
    uint64_t device_bytes;  /* bytes april_index_upload needs */
} april_index_info;

april_status april_index_build(const april_sets *R, uint32_t bucket_bits, april_index **out);
void april_index_destroy(april_index *index);
april_status april_index_get_info(const april_index *index, april_index_info *info);

/* Device image of an index, as written by april_index_upload (pointers into
 * the caller's buffer):
 *   off: (2^b)^2 + 1 bucket offsets into ent (buckets in row-major order);
 *   ent: object ids, bucket by bucket, ascending within a bucket;
 *   ebx: the bucket column of every entry. */
typedef struct april_dev_index {
    const uint32_t *off;
    const uint32_t *ent;
    const uint16_t *ebx;
    uint32_t bucket_bits;
    uint32_t n_objects;
    uint64_t n_entries;
} april_dev_index;

/* Copies the index into a caller-allocated device buffer of at least
 * info.device_bytes bytes (256-byte aligned), asynchronously on stream; the
 * host index must stay alive until the copy completed. */
april_status april_index_upload(const april_index *index, void *dev_buf, size_t dev_bytes, void *stream,
                                april_dev_index *out);

/* Device scratch april_select needs for up to `capacity` candidate pairs. */
april_status april_select_scratch_bytes(uint64_t capacity, size_t *bytes);

/* Answers the selection queries Q over R.
 *   I            index built over R (april_index_build) and uploaded.
 *   R, Q         device sets on the same global grid, with MBRs (april_upload).
 *   capacity     room in d_r, d_q and d_verdict, in pairs.
 *   d_r, d_q     receive the candidate pairs (data object, query), grouped by
 *                query; within a query in a fixed order (bucket row, bucket,
 *                object id), the same on every call.
 *   d_verdict    receives each pair's verdict (as april_filter_pairs).
 *   d_query_off  n_queries + 1 uint32: query q's pairs are
 *                [d_query_off[q], d_query_off[q + 1]).
 *   n_pairs      receives the number of candidate pairs.
 * The call counts the candidates first and synchronizes the stream once to
 * read the count; the pairs and the filter are then enqueued asynchronously
 * (device errors as for april_filter_pairs, via april_sync_status).  With
 * d_r, d_q and d_verdict all NULL it only counts (and fills d_query_off).
 * More pairs than capacity: APRIL_ERR_OVER_BUDGET with *n_pairs set and
 * d_query_off filled, nothing else written. */
april_status april_select(april_ctx *ctx, const april_dev_index *I, const april_dev_sets *R,
                          const april_dev_sets *Q, uint64_t capacity, uint32_t *d_r, uint32_t *d_q,
                          uint8_t *d_verdict, uint32_t *d_query_off, uint64_t *n_pairs, void *d_scratch,
                          size_t scratch_bytes, void *stream);

/* ----------------------------------------------------- host Algorithm 2 */

/* Algorithm 2 exactly as printed (sequential merge joins AA, AF, FA with early
 * exit), run on the host over built sets; a CPU reference execution of the
 * paper's method used for measurement, never by april_filter_pairs.
 * consumed[k] (optional) receives the number of intervals the three joins read
 * for pair k: for every join that ran, (position where the merge stopped + 1)
 * on each side, capped at the list lengths.  Out-of-range ids give
 * APRIL_VERDICT_ERROR and consumed 0. */
april_status april_host_filter(const april_sets *R, const april_sets *S, const uint32_t *pr,
                               const uint32_t *ps, uint64_t n, uint32_t n_threads, uint8_t *verdict,
                               uint64_t *consumed);

/* Algorithm 2 run the way the batched GPU kernels run it with the default
 * tuning.  On sets built on one shared grid the triage comes first: a pair
 * whose MBR-intersection centre cell lies in A(r) and F(s), or in F(r) and
 * A(s), is a true hit; the other pairs are joined in the order AA, AF, FA.
 * Without the triage the order is AF, AA, FA (an AF or FA overlap implies an
 * AA overlap, so the verdicts are Algorithm 2's whatever the order, Sec.
 * 4.2).  Every merge join starts at each list's first interval whose last
 * cell reaches the
 * other list's first start (found by binary search; the sequential merge from
 * the front passes over the intervals before it without a verdict).  The
 * merge gallops: after 16 consecutive advances of one list it jumps, by
 * binary search, to that list's first interval whose last cell reaches the
 * other list's current start (the intervals passed over meet nothing).  The
 * verdicts equal april_host_filter's.  consumed[k] counts, for every join
 * that ran, the intervals the merge reads plus the probes of every search
 * (the bit width of the searched length), and for the triage 4 (the two
 * MBRs' bytes) plus bit_width(n / 16) + 5 for each list looked up: the bytes
 * model of the kernels' reading, used for their roofline.  (The kernels start up to 16 intervals
 * before the exact start and gallop after a whole window that advanced one
 * list only, so they read at least this much; the verdicts are the same.) */
april_status april_host_filter_searched(const april_sets *R, const april_sets *S, const uint32_t *pr,
                                        const uint32_t *ps, uint64_t n, uint32_t n_threads, uint8_t *verdict,
                                        uint64_t *consumed);

/* The filter variants of april_filter_pairs_ex, run sequentially on the host
 * over built sets on global grids (a CPU reference execution used for
 * measurement, never by april_filter_pairs_ex).  Same verdicts and
 * consumed-interval counts as april_host_filter for
 * APRIL_PREDICATE_INTERSECTS on equal orders.  Out-of-range ids give
 * APRIL_VERDICT_ERROR and consumed 0; partitioned sets, an unknown predicate
 * or APRIL_PREDICATE_WITHIN on different orders return
 * APRIL_ERR_INVALID_ARG.  consumed may be NULL. */
april_status april_host_filter_ex(const april_sets *R, const april_sets *S, const uint32_t *pr, const uint32_t *ps,
                                  uint64_t n, int predicate, uint32_t n_threads, uint8_t *verdict, uint64_t *consumed);

#ifdef __cplusplus
}
#endif

#endif /* APRIL_H */
