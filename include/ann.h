/*
 * ann.h -- C ABI of libann: the online query path of GATE-style graph
 * approximate nearest-neighbour search (arXiv 2506.15986) on one GB300
 * (sm_103a).
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are CUDA device pointers on the index's device; other
 *    pointers are host pointers unless stated otherwise.  All device buffers
 *    passed in are owned by the caller and must stay valid until the work
 *    queued on `stream` has finished.  The index owns the device copies of its
 *    base vectors, graph and entry model, and frees them in ann_free_index.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that take a stream are asynchronous: they validate their arguments on the
 *    host, queue kernels and return.
 *  - Errors in the arguments or files are returned synchronously before any
 *    kernel is queued.  Conditions found on the device (visited-set capacity,
 *    a bounded wait that timed out) are OR-ed into the index's device status
 *    word; ann_sync_status returns and clears them.  Queries hit by such a
 *    condition return ids -1 and distance +inf (INT32_MAX for uint8 data).
 *  - Orders are lexicographic on (distance, id): ties go to the smaller id.
 *  - Distances: uint8 data use exact int32 squared L2; floating-point data
 *    accumulate squared L2, or the negated inner product for ANN_IP, in fp32.
 */
#ifndef ANN_H
#define ANN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ANN_OK = 0,
    ANN_ERR_INVALID_ARG = 1,
    ANN_ERR_IO = 2,
    ANN_ERR_FORMAT = 3,
    ANN_ERR_OOM = 4,
    ANN_ERR_CUDA = 5,
    ANN_ERR_CAPACITY = 6,
    ANN_ERR_TIMEOUT = 7,
    ANN_ERR_UNSUPPORTED = 8
} ann_status;

/*
 * Element type of the stored base vectors.  ANN_I8S is int8 with one scale
 * per row (the precision line's int8 storage): a packed row is a 16-byte
 * header (fp32 scale, then 12 zero bytes), the dim int8 codes, and zero bytes
 * up to a multiple of 16 (ann_i8s_row_bytes); the row stands for
 * x_j = scale * code_j.  Queries against every float type, ANN_I8S included,
 * are fp32 rows.
 */
typedef enum { ANN_U8 = 0, ANN_F32 = 1, ANN_F16 = 2, ANN_BF16 = 3, ANN_I8S = 4 } ann_dtype;

/* ANN_L2: squared Euclidean distance; ANN_IP: -<q, x> (maximum inner product) */
typedef enum { ANN_L2 = 0, ANN_IP = 1 } ann_metric;

typedef struct ann_index ann_index;

/* Search flags */
#define ANN_SEARCH_RERANK 1u /* re-score the final pool from the fp32 copy (see ann_index_desc.base_f32) */
#define ANN_SEARCH_FAULT_WAIT 2u /* fault injection for tests of the timeout path (see ann_search_params) */
#define ANN_SEARCH_VISITED_L2 4u /* keep the first-level visited tables resident in L2 (see ann_search_params) */
#define ANN_SEARCH_GROUP_ENTRIES 8u /* run queries grouped by their first seed (see ann_search_params) */

/* Limits of one search */
#define ANN_MAX_L 4096     /* pool size L */
#define ANN_MAX_W 4        /* entries expanded per step */
#define ANN_MAX_STEP_CAND 128 /* W * degree */
#define ANN_MAX_SEEDS 32   /* seed nodes per query (n_entries) */

/*
 * Index description for ann_index_create.  The path searches a fixed-degree
 * proximity graph (Sec. 2.1, Def. 1) over base vectors D.
 *   n, dim       number of base vectors and their dimension; dim * element
 *                size must be a multiple of 16 bytes (16-byte row gathers);
 *                for ANN_I8S, dim must be a multiple of 4
 *   degree       R, slots per adjacency row, 1..ANN_MAX_STEP_CAND (a search
 *                expanding W entries per step needs W * R <= ANN_MAX_STEP_CAND)
 *   dtype,metric see ann_dtype / ann_metric; uint8 supports ANN_L2 only
 *   base         n*dim elements of dtype, row-major (host or device pointer);
 *                for ANN_I8S, n packed rows made by ann_quantize_i8s
 *   graph        n*degree int32 node ids, row-major; -1 marks an unused
 *                slot (host or device pointer)
 *   medoid       entry node used when no per-query entry is given (the
 *                navigating node of Sec. 2.1)
 *   base_f32     optional n*dim fp32 rows (host or device) kept for the exact
 *                rerank of reduced-precision (F16/BF16/I8S) storage; may be
 *                NULL
 * The index copies everything it is given; the caller keeps ownership.
 */
typedef struct {
    int64_t n;
    int32_t dim;
    int32_t degree;
    int32_t dtype;
    int32_t metric;
    const void *base;
    const int32_t *graph;
    int32_t medoid;
    const float *base_f32;
} ann_index_desc;

/*
 * Per-call search parameters (Sec. 2.1, Algorithm 1: pool size l_s = L,
 * result size k).
 *   k         results per query, 1 <= k <= L; also the row stride of the
 *             outputs when d_k is given (then every d_k[i] <= k)
 *   L         pool size, 1 <= L <= ANN_MAX_L; the maximum when d_L is given
 *   W         pool entries expanded per step, 1..ANN_MAX_W, W*degree <= 128
 *   hash_bits log2 of the per-query shared-memory visited-table capacity,
 *             0 = chosen from L; 8..15; -1 = no shared table (the visited set
 *             lives in the global spill tables from the first step)
 *   stage_rows neighbour rows gathered into shared memory per round, 0 =
 *             chosen from the row size; 1..32.  hash_bits and stage_rows change
 *             speed only, never results (see ann_autotune)
 *   team      lanes that compute one distance together (the warp evaluates
 *             32/team staged rows at a time), 0 = chosen from the row size;
 *             1, 2, 4, 8, 16 or 32.  Speed only for uint8 data; for float
 *             data it sets the FP32 summation order, so distances may differ
 *             in the last bits between teams
 *   n_entries seeds per query in d_entry (0 or 1: one), 1..ANN_MAX_SEEDS:
 *             d_entry is then nq x n_entries node ids, -1 marking an unused
 *             slot (at least one per query).  The initial pool holds every
 *             distinct seed, each evaluated once (Algorithm 1 starts from a
 *             set of nodes; one seed is the NSG-style single entry)
 *   spill_bits log2 of the slots of the first global visited table a query
 *             moves to when its shared table fills (the second one has four
 *             times as many), 0 = chosen from L; 10..16.  Speed only, unless
 *             a query outgrows both tables (ANN_ERR_CAPACITY)
 *   flags     ANN_SEARCH_* bits.  ANN_SEARCH_RERANK: after the search, every
 *             id of the final pool (L entries) is re-scored exactly from the
 *             index's fp32 copy of the rows (ann_index_desc.base_f32; without
 *             it the call returns ANN_ERR_UNSUPPORTED) and the k best by
 *             (fp32 distance, id) are returned (the precision line: reduced-
 *             precision storage for traversal, exact scores for the answer).
 *             ANN_SEARCH_VISITED_L2 (speed only): when the first-level visited
 *             tables of all the launch's teams fit the device's persisting-L2
 *             capacity, the search launches with an access-policy window that
 *             keeps them resident in L2 (no write-back, and compare-and-swaps
 *             that hit in L2); otherwise it launches without one.  Such a
 *             call outside stream capture raises the context's persisting-L2
 *             set-aside (cudaLimitPersistingL2CacheSize) to the device maximum
 *             when it is below that.  While the set-aside is raised, accesses
 *             without a persisting window use only the rest of L2, and the
 *             persisting lines outlive the call: ann_release_l2 undoes both.
 *             ANN_SEARCH_GROUP_ENTRIES (speed only): with entries given, the
 *             launch first sorts the work items by a hash of their first seed
 *             (one extra single-CTA kernel, 4 bytes of scratch per item) and
 *             the persistent teams take them in that order, so queries that
 *             start at the same node run side by side and share the rows of
 *             their first steps in L2.  Every item's outputs are written at its
 *             own index and do not depend on the order.  Ignored with the
 *             medoid entry (d_entry NULL).
 *             ANN_SEARCH_FAULT_WAIT: fault injection for testing; every wait
 *             for a round of gathered rows gives up at once, as if its time
 *             limit had passed: each query fails with -1 ids and the call
 *             reports ANN_ERR_TIMEOUT through ann_sync_status.  The copies in
 *             flight still land, so the device and the index stay usable.
 *   gather    how a round of neighbour rows is fetched, 0 = chosen from the
 *             row size; 1: one bulk copy per row; 4: one TMA tensor gather per
 *             four rows (rows of 32-byte multiples up to 1 KiB; other sizes
 *             use 1).  Speed only, never results (see ann_autotune)
 *   d_k, d_L  optional per-query k and L (device int32[nq]); NULL = k, L
 *   d_target  optional per-query target node (device int32[nq]); when given
 *             the search runs in label mode: it stops after the step in which
 *             the target is evaluated and d_stats reports the counters at that
 *             point (INT32_MAX when it never is; Sec. 4.2, Def. 4)
 */
typedef struct {
    int32_t k;
    int32_t L;
    int32_t W;
    int32_t hash_bits;
    int32_t stage_rows;
    int32_t team;
    int32_t spill_bits;
    int32_t n_entries;
    uint32_t flags;
    int32_t gather;
    const int32_t *d_k;
    const int32_t *d_L;
    const int32_t *d_target;
} ann_search_params;

/* Human-readable name of a status code (static storage; never NULL). */
const char *ann_status_string(ann_status s);

/*
 * Create an index on CUDA device `device` from `desc` (copied into memory the
 * index owns).  Validates sizes, dtype/metric and that every graph id is in
 * [-1, n) and the medoid in [0, n).  Returns ANN_ERR_INVALID_ARG on bad
 * arguments, ANN_ERR_OOM / ANN_ERR_CUDA on device failures; *out is set only
 * on success.
 * The index holds the base set D and its proximity graph G of Sec. 2.1
 * (Def. 1).
 */
ann_status ann_index_create(const ann_index_desc *desc, int device, ann_index **out);

/*
 * Bytes of one packed ANN_I8S row of dim codes: 16 + dim rounded up to 16.
 * Layout of the int8 storage of the precision line; pure arithmetic, no
 * error (0 for dim < 1).
 */
int32_t ann_i8s_row_bytes(int32_t dim);

/*
 * Quantise n fp32 rows of dim values (device pointer d_x, row-major) into n
 * packed ANN_I8S rows at d_rows (device, n * ann_i8s_row_bytes(dim) bytes,
 * 16-byte aligned; caller-owned).  Per row, in fp32: scale = max_j |x_j| /
 * 127; code_j = x_j / scale rounded half to even and clipped to [-127, 127];
 * an all-zero row gets scale 0 and zero codes.  dim must be a multiple of 4.
 * Asynchronous on stream.
 * The int8-with-scale storage of the precision line (a storage choice of this
 * library; the paper fixes no precision).
 */
ann_status ann_quantize_i8s(const float *d_x, int64_t n, int32_t dim, void *d_rows, void *stream);

/*
 * Free an index and its device memory (NULL is accepted).  Synchronises the device.
 * Lifetime only (no paper passage); always ANN_OK.
 */
ann_status ann_free_index(ann_index *idx);

/*
 * Read index metadata; any output pointer may be NULL.  has_model reports
 * whether a learned entry model is attached.
 * Metadata of the Sec. 2.1 index; ANN_ERR_INVALID_ARG for a NULL index,
 * else ANN_OK.
 */
ann_status ann_index_info(const ann_index *idx, int64_t *n, int32_t *dim, int32_t *degree,
                          int32_t *dtype, int32_t *metric, int32_t *medoid,
                          int32_t *n_hubs, int32_t *has_model);

/*
 * Write the index (header, base, graph, optional fp32 copy, entry model) to
 * `path` with a 64-bit FNV-1a checksum.  ANN_ERR_IO on a write failure.
 * Persistence of the Sec. 2.1 index and the Sec. 4.3 model (no paper
 * passage).
 */
ann_status ann_save_index(const ann_index *idx, const char *path);

/*
 * Load an index written by ann_save_index onto `device`.  ANN_ERR_IO if the
 * file cannot be read, ANN_ERR_FORMAT if its magic, version, sizes or checksum
 * do not match (a truncated or corrupted file).
 * Persistence of the Sec. 2.1 index and the Sec. 4.3 model (no paper
 * passage).
 */
ann_status ann_load_index(const char *path, int device, ann_index **out);

/*
 * Batched best-first beam search (Sec. 2.1, Algorithm 1; sorted-pool form):
 * for each query, start from its entry node, repeatedly expand the first W
 * unexpanded entries of a pool of the L best nodes seen, evaluate every
 * unvisited neighbour once, and stop when the pool holds no unexpanded entry.
 *   d_queries nq*dim query rows: uint8 for an ANN_U8 index, fp32 otherwise
 *   nq        number of queries (0 is accepted and queues nothing)
 *   d_entry   per-query entry node (device int32[nq]), or nq x p->n_entries
 *             seed nodes when p->n_entries > 1, or NULL for the medoid
 *   p         search parameters (host pointer)
 *   d_ids     out: nq*k int32 node ids, best first; -1 pads missing results
 *   d_dists   out: nq*k distances, int32 for ANN_U8 and fp32 otherwise
 *   d_stats   out (optional): nq*2 int32 {distance evaluations, expansions}
 * One warp serves one query; queries are pulled from a device work queue by
 * a persistent grid sized to the SM count.  Scratch memory is taken from a
 * stream-ordered pool owned by the index, per call: calls on different
 * streams may run concurrently on one index (their outputs must not alias),
 * which lets the next batch's grid fill the SMs that one batch's last
 * queries leave idle.
 * Asynchronous on `stream`. Errors: ANN_ERR_INVALID_ARG for a NULL or
 * misaligned pointer or parameters out of range (returned before any
 * launch); device-side capacity, timeout and bad-input conditions go to the
 * status word (ann_sync_status) and their queries return ids -1.
 */
ann_status ann_search_batch(ann_index *idx, const void *d_queries, int64_t nq,
                            const int32_t *d_entry, const ann_search_params *p,
                            int32_t *d_ids, void *d_dists, int32_t *d_stats, void *stream);

/*
 * Synchronise `stream`, then return and clear the index's device status
 * word: ANN_OK, or the first of ANN_ERR_CAPACITY / ANN_ERR_TIMEOUT raised by
 * kernels since the last call; ANN_ERR_CUDA if a CUDA call failed.
 * The device status word of the Sec. 2.1 search (no paper passage).
 */
ann_status ann_sync_status(ann_index *idx, void *stream);

/*
 * Undoes what searches with ANN_SEARCH_VISITED_L2 left in the L2 of the
 * index's device: every persisting line of this process's context there
 * returns to normal status and the context's persisting-L2 set-aside
 * (cudaLimitPersistingL2CacheSize) returns to zero, so that later work
 * without the flag has the whole L2 again (the next flagged search raises
 * the set-aside again).  Waits for the device first.  A cache-residency
 * control of this implementation (no paper passage); ANN_ERR_CUDA on failure.
 */
ann_status ann_release_l2(ann_index *idx);

/* ---- batching line: CUDA-graph plans and the autotuner -------------------- */

typedef struct ann_plan ann_plan;

/*
 * Capture one batch -- entry selection (entry_mode, L_hub as in
 * ann_select_entry; ANN_ENTRY_MEDOID skips it) followed by ann_search_batch
 * with parameters p -- into a CUDA graph over fixed buffers.  The plan keeps
 * the pointers: queries, per-query arrays of p, d_entry_buf (nq x
 * max(1, p->n_entries) int32, needed unless the mode is ANN_ENTRY_MEDOID;
 * with p->n_entries > 1 the plan selects seed sets with ann_select_entries)
 * and the outputs must stay
 * valid while the plan is used.  Blocking; the index must not be freed
 * before the plan.
 */
ann_status ann_plan_create(ann_index *idx, const void *d_queries, int64_t nq, int32_t entry_mode,
                           int32_t L_hub, const ann_search_params *p, int32_t *d_entry_buf,
                           int32_t *d_ids, void *d_dists, int32_t *d_stats, ann_plan **out);

/*
 * Launch a captured batch on `stream` (asynchronous).
 * The batched serving path: one captured batch of Sec. 4.3 entry
 * selection and Sec. 2.1 search. ANN_ERR_INVALID_ARG for a NULL plan.
 */
ann_status ann_plan_launch(ann_plan *plan, void *stream);

/*
 * Free a plan (NULL is accepted).  Synchronises the device.
 * Lifetime only (no paper passage); always ANN_OK.
 */
ann_status ann_plan_free(ann_plan *plan);

/*
 * Time ann_search_batch over the given batch for a sequence of speed knobs,
 * each stage starting from the fastest combination so far, and return in
 * *best the copy of *p with the fastest combination (*best_ms: its time per
 * batch).  The stages:
 *   1. hash_bits (no shared table, and sizes around and below the default)
 *      x stage_rows 4, 6, 8, 12, 16;
 *   2. team 2 to 32, where a lane gets 1 to 16 16-byte chunks of the row;
 *   3. spill_bits up to two either side of the default;
 *   4. gather 4 (when the index's rows allow TMA tensor gathers) with
 *      stage_rows 8, 12, 16 and team the best or 8;
 *   5. ANN_SEARCH_VISITED_L2 with spill_bits the best and one and two less
 *      (ann_release_l2 after each such trial, and at the end when the chosen
 *      combination has the flag);
 *   6. ANN_SEARCH_GROUP_ENTRIES, when d_entry is given.
 *   reps   timed batches per combination, after one warm-up batch per lane
 *   lanes  1..8 streams the timed batches alternate over (batch r on lane
 *          r mod lanes), so that combinations are timed with consecutive
 *          batches overlapping, as they run when a caller spreads batches over
 *          that many streams; lane 0 is `stream`, the others are created and
 *          destroyed here and write to output buffers from the index's pool
 *   d_ids, d_dists  out: the results of the chosen combination
 * The visited set stays exact (shared table plus global spill), and neither
 * the gather mode nor the work order enters any result; the team size only
 * moves float distances by FP32 rounding.  Blocking.  Errors:
 * ANN_ERR_INVALID_ARG for a NULL index, params or best, nq < 1, reps < 1 or
 * lanes outside 1..8; a search error stops the tuning and is returned.
 * Speed knobs of the Sec. 2.1 search only (the batched serving path).
 */
ann_status ann_autotune(ann_index *idx, const void *d_queries, int64_t nq, const int32_t *d_entry,
                        const ann_search_params *p, int32_t *d_ids, void *d_dists, int32_t reps,
                        int32_t lanes, ann_search_params *best, float *best_ms, void *stream);

/* ---- learned entry selection (Sec. 4.3) ---------------------------------- */

/* How ann_select_entry picks each query's entry node. */
typedef enum {
    ANN_ENTRY_MEDOID = 0,             /* the index's navigating node */
    ANN_ENTRY_LEARNED_NAV = 1,        /* greedy search of the hub graph (Algorithm 1, IP) */
    ANN_ENTRY_LEARNED_EXHAUSTIVE = 2  /* argmax over every hub */
} ann_entry_mode;

/*
 * Two-tower entry model (Sec. 2.2, Sec. 4.3).  Query tower: q_hat =
 * normalise(ReLU(q W1 + b1) W2 + b2); hub tower: e_hat_v = normalise(e_v).
 * The entry of q is the hub node of argmax_v q_hat . e_hat_v (cosine).
 *   in_dim      query dimension; must equal the index dim (<= 512)
 *   hidden      256; out_dim 64 (the only widths supported)
 *   W1 [in_dim][256], b1 [256], W2 [256][64], b2 [64]: fp32, row-major
 *   n_hubs      H >= 2; hub_nodes [H] node ids; hub_emb [H][64] fp32
 *   hub_degree  s, 1..32 and < H: the high-tier graph links every hub to its
 *               s most cosine-similar hubs (Sec. 4.3)
 *   hub_graph   [H][s] int32, or NULL to build it from hub_emb (ties: smaller
 *               hub index)
 *   hub_entry   entry hub of the hub-graph search, or -1 for the hub with the
 *               largest cosine to the mean embedding
 * All arrays may be host or device pointers; they are copied.
 */
typedef struct {
    int32_t in_dim;
    int32_t hidden;
    int32_t out_dim;
    const float *W1;
    const float *b1;
    const float *W2;
    const float *b2;
    int32_t n_hubs;
    const int32_t *hub_nodes;
    const float *hub_emb;
    int32_t hub_degree;
    const int32_t *hub_graph;
    int32_t hub_entry;
} ann_entry_model_desc;

/*
 * Attach (or replace) the entry model of an index.  Builds the BF16 weight
 * and embedding tables, the hub graph when not given, and the hub-graph
 * index.  Blocking.  ANN_ERR_INVALID_ARG on bad sizes or hub node ids.
 */
ann_status ann_set_entry_model(ann_index *idx, const ann_entry_model_desc *model, void *stream);

/*
 * Copy the attached model out (host or device destinations; NULL skips an
 * array).  Sizes as in ann_entry_model_desc.  ANN_ERR_INVALID_ARG without a model.
 * The Sec. 4.3 two-tower model and its hub graph.
 */
ann_status ann_get_entry_model(const ann_index *idx, float *W1, float *b1, float *W2, float *b2,
                               float *hub_emb, int32_t *hub_nodes, int32_t *hub_graph,
                               int32_t *hub_entry);

/*
 * Rebuild the attached model's hub graph (Sec. 4.3: every hub linked to its
 * s most cosine-similar hubs).  Two readings of "connect edges":
 *   max_degree = 0   directed: row i lists hub i's s_nn most similar other
 *                    hubs (what ann_set_entry_model builds); row width s_nn
 *   max_degree >= s  undirected: hubs u and v are linked when either lists
 *                    the other; row i lists its neighbours in decreasing
 *                    cosine (smaller index on ties), at most max_degree of
 *                    them, padded with -1; row width max_degree
 *   s_nn 1..32 and < n_hubs; max_degree 0 or s_nn..32.
 * The similarities are inner products of the normalised FP32 embeddings (the
 * undirected ordering in double on the host).  The hub-graph index is
 * rebuilt; the entry hub and the hub sample (ann_set_hub_seeds) are kept.
 * ann_get_entry_model then returns rows of the new width.  Blocking: waits
 * for the device first.  ANN_ERR_UNSUPPORTED without a model,
 * ANN_ERR_INVALID_ARG for sizes out of range, ANN_ERR_OOM.  After a failure
 * the hub-graph mode reports ANN_ERR_UNSUPPORTED until a rebuild succeeds.
 */
ann_status ann_build_hub_graph(ann_index *idx, int32_t s_nn, int32_t max_degree, void *stream);

/*
 * The sample of hubs the hub-graph search (ANN_ENTRY_LEARNED_NAV) starts
 * from.  Algorithm 1 (Sec. 2.1) starts its pool from a random sample of the
 * graph's nodes; on the high-tier graph of Sec. 4.3 that sample is this list.
 *   seeds  n hub indices in [0, n_hubs) (host or device; copied), drawn by
 *          the caller (the library draws no random numbers); repeats count
 *          once
 *   n      0..ANN_MAX_SEEDS; 0 goes back to the single entry hub
 *          (ann_entry_model_desc.hub_entry)
 * Per query, every distinct sample hub is scored and the L_hub best form the
 * first pool.  The sample belongs to the attached model: ann_set_entry_model
 * (and ann_trainer_attach) start the new model without one.  Blocking: waits
 * for the device, so no entry selection of the index is in flight while the
 * sample changes.  ANN_ERR_UNSUPPORTED without a model, ANN_ERR_INVALID_ARG
 * for n out of range or a hub index out of range.
 */
ann_status ann_set_hub_seeds(ann_index *idx, const int32_t *seeds, int32_t n);

/*
 * Entry node per query (Sec. 4.3: the recommended hub is the entry point).
 *   d_queries  nq*dim rows as for ann_search_batch (16-byte aligned)
 *   mode       ann_entry_mode; the learned modes need an attached model
 *              (ANN_ERR_UNSUPPORTED otherwise)
 *   L_hub      pool size of the hub-graph search (ANN_ENTRY_LEARNED_NAV), 1..ANN_MAX_L
 *   d_entry    out: nq int32 node ids, ready for ann_search_batch
 *   d_qhat     out (optional): nq*64 fp32 normalised query embeddings
 * Asynchronous on `stream`; the query tower and the exhaustive hub scores run
 * as BF16 tcgen05 GEMMs with FP32 accumulation.
 */
ann_status ann_select_entry(ann_index *idx, const void *d_queries, int64_t nq, int32_t mode,
                            int32_t L_hub, int32_t *d_entry, float *d_qhat, void *stream);

/*
 * Seed sets per query: the m_seeds best hubs of each query, best first
 * (Algorithm 1 starts from a set of nodes; Sec. 4.3 scores every hub for the
 * query, so its top hubs are the natural seeds).  ANN_ENTRY_LEARNED_EXHAUSTIVE
 * keeps the top m_seeds of all hub scores (ties to the smaller hub index);
 * ANN_ENTRY_LEARNED_NAV takes the m_seeds best of the hub-graph search's pool
 * (L_hub >= m_seeds); ANN_ENTRY_MEDOID gives the medoid and unused slots.
 *   m_seeds    1..ANN_MAX_ENTRY_HUBS
 *   d_entry    out: nq*m_seeds int32 node ids (-1 = unused slot), ready for
 *              ann_search_batch with ann_search_params.n_entries = m_seeds
 *   other arguments as for ann_select_entry, which is the m_seeds = 1 case.
 */
#define ANN_MAX_ENTRY_HUBS 8
ann_status ann_select_entries(ann_index *idx, const void *d_queries, int64_t nq, int32_t mode, int32_t L_hub,
                              int32_t m_seeds, int32_t *d_entry, float *d_qhat, void *stream);

/*
 * Exhaustive learned entry selection (the ANN_ENTRY_LEARNED_EXHAUSTIVE mode
 * of ann_select_entry) that allocates no device memory.  The paper has no
 * counterpart: this exists for callers that cannot let the library allocate,
 * such as a serving process that has reserved all of HBM up front, a latency
 * critical loop where an allocator call could stall or synchronise the
 * device, or a context (a host callback) where allocating CUDA calls are not
 * allowed.
 *   Scratch: a 16 MiB array that every GPU loading the library holds until the
 *   process exits (136 bytes per query).  Batches larger than
 *   ann_select_entry_noalloc_max_queries() (123,357) are rejected with
 *   ANN_ERR_CAPACITY before anything is queued; split them.
 *   The first call on a device looks up the array's device address on that
 *   device (a one-time set-up), so make the first call on each device before
 *   any stream capture.  The address is kept until the process exits: after
 *   a cudaDeviceReset by the host application it no longer names live
 *   memory, so do not call this entry point on a device that was reset.
 *   All calls on a device share the one array: calls whose work overlaps on
 *   the GPU (for example on two streams) race and must be serialised by the
 *   caller.  Every word is written before it is read, so no clearing is needed.
 *   Arguments and results are those of ann_select_entry in that mode:
 *   d_entry (nq int32 node ids), d_qhat (optional nq*64 fp32).  Needs an
 *   attached entry model (ANN_ERR_UNSUPPORTED otherwise).  Asynchronous.
 */
ann_status ann_select_entry_noalloc(ann_index *idx, const void *d_queries, int64_t nq,
                                    int32_t *d_entry, float *d_qhat, void *stream);

/*
 * Largest nq ann_select_entry_noalloc accepts.
 * A constant of this implementation (no paper passage); no error.
 */
int64_t ann_select_entry_noalloc_max_queries(void);

/* ---- entry-model training (Sec. 4.2 labels, Sec. 4.3 loss, Sec. 5.1 Adam) -- */

typedef struct ann_trainer ann_trainer;

/*
 * Trainer of the two-tower model on one device.  Parameters start from the
 * given fp32 arrays (host or device; W1 [in_dim][256], b1 [256], W2 [256][64],
 * b2 [64], hub_emb [n_hubs][64]); Adam state starts at zero.  n_hubs 2..65536.
 *   max_batch  largest batch (rows of scratch; the paper uses 8,192)
 *   tau        InfoNCE temperature; lr, beta1, beta2, eps: Adam
 * Every GEMM of a step runs on the tensor cores (BF16 operands, FP32
 * accumulators); parameters, gradients and Adam state are fp32.
 * Blocking; ANN_ERR_INVALID_ARG for NULL weights or sizes out of range,
 * ANN_ERR_CUDA for a bad device, ANN_ERR_OOM.
 */
ann_status ann_trainer_create(int device, int32_t in_dim, int32_t n_hubs, const float *W1, const float *b1,
                              const float *W2, const float *b2, const float *hub_emb, int64_t max_batch,
                              float tau, float lr, float beta1, float beta2, float eps, ann_trainer **out);

ann_status ann_trainer_free(ann_trainer *t);

/*
 * One step on the batch of rows d_rows[0..nb) of d_queries (fp32, in_dim
 * columns, 16-byte aligned; d_rows NULL = rows 0..nb-1).  Labels: query row r
 * lists M distinct hub indices d_cand[r*M + j] (-1 = empty slot) with labels
 * d_labels[r*M + j] (+1 positive, -1 negative, 0 unused); every hub not
 * listed for the row is a negative (a hub the label search did not reach
 * from that query, Sec. 4.2).  A dense label matrix is the case M = n_hubs
 * with d_cand[r*M + j] = j.  Computes the loss and the gradients of every
 * parameter; applies the Adam update when apply_update is non-zero.
 * loss_out (host, optional) receives the batch loss.
 * Sec. 4.3 Eq. loss and its gradient, Sec. 5.1 Adam. Blocking when loss_out
 * is given, else asynchronous; ANN_ERR_INVALID_ARG for a NULL or misaligned
 * input, M out of 1..n_hubs or nb out of range.
 */
ann_status ann_trainer_step(ann_trainer *t, const float *d_queries, const int32_t *d_rows, int64_t nb,
                            const int32_t *d_cand, const int8_t *d_labels, int32_t M, int32_t apply_update,
                            float *loss_out, void *stream);

/*
 * Epochs of steps over nt training queries; epoch e visits rows
 * d_order[e*nt .. e*nt+nt) (device, NULL = 0..nt-1) in batches of max_batch.
 * d_cand, d_labels and M as for ann_trainer_step (nt*M entries each).
 * d_losses (device, optional) receives epochs * ceil(nt / max_batch) batch
 * losses.  Blocking.
 * Sec. 4.3 training with Sec. 5.1 Adam.
 */
ann_status ann_trainer_fit(ann_trainer *t, const float *d_queries, int64_t nt, const int32_t *d_cand,
                           const int8_t *d_labels, int32_t M, const int32_t *d_order, int32_t epochs,
                           float *d_losses, void *stream);

/*
 * Copy the current parameters (gradients != 0: the last step's gradients).
 * With a fusion tower, hub_emb receives the rows the model scores, E + F,
 * and its gradient is that of E + F (the same as E's).
 * Sec. 4.3 model parameters. Blocking; ANN_ERR_TIMEOUT if a tensor-core
 * wait of an earlier step gave up, ANN_ERR_INVALID_ARG for a NULL trainer.
 */
ann_status ann_trainer_get(const ann_trainer *t, float *W1, float *b1, float *W2, float *b2, float *hub_emb,
                           int32_t gradients);

/*
 * Topology-aware hub tower (Sec. 4.3, Module I, Eq. fusion): from now on the
 * hub row of hub v is E_v + F_v with
 *     F_v = Concat_j softmax((p_v WQ_j)(U_v WK_j)^T / sqrt(head_dim)) (U_v WV_j)  WO
 * for j = 1..heads, p_v the hub's vector and U_v its T tokens of token_dim
 * (see ann_topo_tokens), trained with the rest by the same Adam.
 *   d_hub_vecs  H x in_dim fp32 (device), copied
 *   d_tokens    H x T x token_dim fp32 (device), copied
 *   WQ  in_dim x (heads*head_dim); WK, WV  token_dim x (heads*head_dim);
 *   WO  (heads*head_dim) x 64: initial weights (host or device), copied
 * Call before the first step; once per trainer.  Blocking.
 * Errors: ANN_ERR_INVALID_ARG (NULL, sizes, a second call or a call after
 * a step), ANN_ERR_OOM.
 */
ann_status ann_trainer_set_fusion(ann_trainer *t, const float *d_hub_vecs, const float *d_tokens, int32_t T,
                                  int32_t token_dim, int32_t heads, int32_t head_dim, const float *WQ, const float *WK,
                                  const float *WV, const float *WO);

/*
 * The fusion weights (gradients != 0: the last step's gradients), as laid out for ann_trainer_set_fusion.
 * Sec. 4.3 Eq. fusion weights. Blocking; ANN_ERR_INVALID_ARG without a
 * fusion tower.
 */
ann_status ann_trainer_get_fusion(const ann_trainer *t, float *WQ, float *WK, float *WV, float *WO, int32_t gradients);

/*
 * Attach the trained model to an index (see ann_set_entry_model).
 * The Sec. 4.3 model and its hub graph (cosine, s neighbours). Blocking;
 * errors as ann_set_entry_model.
 */
ann_status ann_trainer_attach(const ann_trainer *t, ann_index *idx, const int32_t *hub_nodes,
                              int32_t hub_degree, void *stream);

/*
 * One Adam update with bias correction at step `step` (>= 1) over n fp32
 * parameters: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).  Asynchronous.
 * Sec. 5.1 names Adam (Kingma and Ba's update).
 */
ann_status ann_adam_update(float *d_params, const float *d_grads, float *d_m, float *d_v, int64_t n, int64_t step,
                           float lr, float beta1, float beta2, float eps, void *stream);

/* ---- hubs and labels --------------------------------------------------- */

/*
 * Lloyd's k-means (a flat stand-in for the balanced clustering of Sec. 4.1,
 * Algorithm 2) on the sample rows sample_rows[0..m) (host int64) of d_x:
 * centroids start at sample rows init[0..k) (host, indices into the sample);
 * each iteration assigns every sample row to its nearest centroid by
 * (squared L2, centroid index), then moves each centroid to its members'
 * mean; an empty centroid moves onto the sample row farthest from its own
 * centroid (larger distance first, smaller row on ties), each row used once.
 *   d_centroids out: k*dim fp32; objective (host, optional): iters sums of
 *   squared distances of the assignments.  Blocking.
 */
ann_status ann_kmeans(const void *d_x, int64_t n, int32_t dim, int32_t dtype, const int64_t *sample_rows,
                      int64_t m, int32_t k, const int32_t *init, int32_t iters, float *d_centroids,
                      double *objective, void *stream);

/*
 * Per-hop topology tokens of hub nodes (Sec. 4.2, subgraph sampling; a fixed
 * summary in place of Graph2Vec), for the fusion tower.  The guided walk from
 * each hub: MinDeg / MaxDeg are the smallest / largest valid-neighbour counts
 * in the graph; a FIFO queue starts at the hub (hop 0); a dequeued node u at
 * hop < h ranks its deg(u) valid neighbours by (squared L2 to u, id) and
 * samples the ceil(x/2) nearest and floor(x/2) farthest,
 * x = ceil(MinDeg * deg(u) / MaxDeg); a sampled neighbour not yet in the
 * subgraph joins at hop(u)+1 with parent u, in rank order, until max_nodes.
 * Token l = 0..h of a hub (8 floats), s = the hub's mean squared distance to
 * its valid neighbours (1 if none or 0): hop-l nodes / all nodes, their mean
 * degree / MaxDeg, mean and max squared distance to the hub / s, mean squared
 * distance to the parent / s, share sampled as farthest, l / h, 1 (the first
 * six 0 for an empty hop).  float32, each operation rounded on its own,
 * coordinates summed in order and a hop's nodes in joining order.
 *   d_hubs     H node ids (device), checked against n
 *   d_tokens   out: H x (h+1) x 8 fp32
 *   d_nodes    out (optional): H subgraph sizes
 * Needs fp32 rows (an ANN_F32 index, or base_f32 given at creation), degree
 * <= 64 and dim % 4 == 0 (else ANN_ERR_UNSUPPORTED); 1 <= h <= 64,
 * 1 <= max_nodes <= 8192.  Blocking.
 */
ann_status ann_topo_tokens(ann_index *idx, const int32_t *d_hubs, int32_t H, int32_t h, int32_t max_nodes,
                           float *d_tokens, int32_t *d_nodes, void *stream);

/*
 * Hierarchical balanced k-means, HBKM (Sec. 4.1, Def. 2 and Algorithm 2), with
 * the hub of every final cluster (Def. 3).  `levels` levels each split every
 * cluster of the level above (level 0: all n rows) into k children, so
 * k^levels clusters come out; child j of cluster c is cluster c*k + j.  A
 * split runs T iterations; each empties the children, visits the cluster's
 * members in increasing row id and puts row x into
 *     argmin_j ||x - mu_j||^2 + lam * (2 (c_j - m) + 1)   (ties: smaller j)
 * with c_j child j's current size, m = |C|/k, lam = lambda * sigma^2 / m and
 * sigma^2 the members' mean squared distance to C's centroid (the penalty is
 * the increase of Def. 2's size variance sum (|C_j| - m)^2 that the move
 * causes); then every non-empty child moves to its members' mean and an empty
 * one keeps its centroid.  A split starts at its members with the
 * min(k, |C|) smallest (d_keys[id], id), in that order; children beyond |C|
 * stay empty at C's centroid.  All arithmetic is float32 with each operation
 * rounded on its own, distances summed over coordinates 0..dim-1 and sigma^2
 * and means over members in increasing id, so results are reproducible bit
 * for bit.
 *   d_x          n x dim fp32 rows (device, 16-byte aligned), dim % 4 == 0,
 *                4 <= dim <= 4096, 1 <= n < 2^31
 *   k, levels    2 <= k <= 32, levels >= 1, k^levels <= 2^20
 *   lambda       penalty strength >= 0 (0: plain k-means splits)
 *   T            iterations per split, >= 1
 *   d_keys       n uint32 (device): the draw that picks the starting members
 *   d_hubs       out: k^levels int32 row ids, the member nearest each final
 *                centroid (smaller id on ties), -1 for an empty cluster
 *   d_centroids  out (optional): k^levels x dim fp32 final centroids
 *   d_label      out (optional): n int32 final cluster of every row
 * Blocking.  Errors: ANN_ERR_INVALID_ARG for a NULL input or output, bad
 * sizes or alignment; ANN_ERR_UNSUPPORTED when k x dim floats do not fit in
 * one block's shared memory.
 */
ann_status ann_hbkm(const float *d_x, int64_t n, int32_t dim, int32_t k, int32_t levels, double lambda, int32_t T,
                    const uint32_t *d_keys, int32_t *d_hubs, float *d_centroids, int32_t *d_label, void *stream);

/*
 * Hub nodes (Sec. 4.1, Def. 3): assign every base row to its nearest centroid;
 * d_hubs[j] = the member of cluster j nearest its centroid (smaller id on
 * ties), -1 for an empty cluster.  d_assign (optional, n int32).  Blocking.
 */
ann_status ann_assign_hubs(const void *d_base, int64_t n, int32_t dim, int32_t dtype, const float *d_centroids,
                           int32_t k, int32_t *d_hubs, int32_t *d_assign, void *stream);

/*
 * Label-mode search costs (Sec. 4.2, Def. 4): for query i and candidate hub
 * d_cand[i*M + j], search from node d_hub_nodes[d_cand[i*M + j]] with pool L
 * and width W until d_targets[i] (the query's exact nearest neighbour) is
 * evaluated; d_evals / d_hops (nq*M) receive the counters after that step, or
 * INT32_MAX when the target is never evaluated.  Asynchronous.
 */
ann_status ann_hub_costs(ann_index *idx, const void *d_queries, int64_t nq, const int32_t *d_targets,
                         const int32_t *d_cand, int32_t M, const int32_t *d_hub_nodes, int32_t L, int32_t W,
                         int32_t *d_evals, int32_t *d_hops, void *stream);

/*
 * Label rule per query over its M searched hubs: best = argmin (evals, hops,
 * hub index) (-1 if none reached the target); m = min hops; label +1 if
 * hops <= m + t_pos, -1 if hops >= m + t_neg or never reached, 0 otherwise;
 * a query with no reached hub gets -1 for every candidate.  The labels are
 * aligned with the candidate list: d_labels[i*M + j] is the label of hub
 * d_cand[i*M + j].  Hubs a query did not search are not listed and count as
 * negatives wherever these labels are used (ann_trainer_step).
 *   d_labels out: nq*M int8; d_best out (optional): nq int32.  Asynchronous;
 *   ANN_ERR_INVALID_ARG for a NULL input or M < 1.
 * Sec. 4.2, Def. 4 and the labelling rule after it (t_pos, t_neg).
 */
ann_status ann_hub_labels(const int32_t *d_evals, const int32_t *d_hops, const int32_t *d_cand, int64_t nq,
                          int32_t M, int32_t t_pos, int32_t t_neg, int8_t *d_labels, int32_t *d_best, void *stream);

/* ---- base-partitioned search: the exchange step -------------------------- */
/*
 * The base set split into P shards (groups of whole hub clusters, Sec. 4.1,
 * Def. 3), each with its own index searched by ann_search_batch; a query's
 * answer is the k best of the shards' answers under the (distance, id) order
 * of Sec. 2.1, Problem 1.  These two calls are the steps around the exchange
 * of the shards' answers.
 */

/*
 * Shard-local row ids to global ids, in place: d_ids[i] >= 0 becomes
 * d_map[d_ids[i]]; -1 stays -1.  An id >= n_map becomes -1 and sets bit 0 of
 * *d_status (device int32, optional, OR-ed).  Asynchronous;
 * ANN_ERR_INVALID_ARG for a NULL array with count > 0.
 */
ann_status ann_map_ids(int32_t *d_ids, int64_t count, const int32_t *d_map, int64_t n_map, int32_t *d_status,
                       void *stream);

/*
 * Merge of P answer lists per query: d_ids / d_dists hold P blocks of nq x k
 * (block p = shard p's answers, row-major [P][nq][k]), each row sorted by
 * (distance, id) with (-1, +inf) padding, ids global and distinct across
 * the lists (the shards are disjoint).  Writes the k smallest (distance, id)
 * of each query's P*k entries to d_out_ids / d_out_dists (nq x k), padded
 * with (-1, +inf) (INT32_MAX for int distances).
 *   int_dists  non-zero: distances are int32 (uint8 data), else fp32
 *   P          1..32
 * Asynchronous; ANN_ERR_INVALID_ARG for P or k out of range or NULL buffers.
 */
ann_status ann_merge_shards(const int32_t *d_ids, const void *d_dists, int32_t P, int64_t nq, int32_t k,
                            int32_t int_dists, int32_t *d_out_ids, void *d_out_dists, void *stream);

/* ---- offline construction (GPU) ------------------------------------------ */

/*
 * Exact k nearest neighbours (Sec. 2.1, Problem 1; the ground truth R of
 * recall@k): for each of nq query rows, the k base rows with the smallest
 * (distance, id).  Candidate scores come from an fp32 GEMM; the best k + margin
 * candidates per query are re-scored exactly (int32 for uint8, fp32 direct
 * differences otherwise) and sorted.
 *   d_base       n*dim base rows (dtype ANN_U8 or ANN_F32), 16-byte aligned
 *   d_queries    nq*dim rows of the same dtype; equal to d_base when
 *                exclude_self != 0 (then row i never returns id i)
 *   k            1..128 and <= n
 *   d_ids,d_dists out: nq*k int32 ids and distances (int32 for ANN_U8, fp32
 *                otherwise)
 * Blocking: returns after the results are written.  Temporary device memory
 * (about 4 GiB of scores plus fp32 copies of uint8 rows) is allocated on
 * `stream` and released before returning.
 */
ann_status ann_knn(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                   const void *d_queries, int64_t nq, int32_t k, int32_t exclude_self,
                   int32_t *d_ids, void *d_dists, void *stream);

/*
 * Navigating node (Sec. 2.1, NSG): argmin_i ||x_i - mean||^2, smaller id on
 * ties.  uint8 rows are handled exactly in 64-bit integers (n <= 2^20,
 * dim <= 128); fp32 rows in fp32.  Blocking.
 */
ann_status ann_medoid(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t *medoid,
                      void *stream);

/*
 * Proximity graph (Sec. 2.1, Def. 1) under squared L2:
 *  1. the K exact nearest other nodes of every node, by (distance, id);
 *  2. relative-neighbourhood pruning in that order: candidate c is kept unless
 *     a node s kept before it has alpha * delta(s, c) <= delta(p, c); at most
 *     R are kept; -1 pads the row;
 *  3. reachability repair from the navigating node: nodes are taken in id
 *     order; an unreachable node u gets the edge w -> u from the reachable node
 *     w nearest to u (by (distance, id)) whose row has a free slot, and every
 *     node reachable from u becomes reachable before the next node is taken.
 *   d_graph   out: n*R int32 adjacency rows (device)
 *   medoid    in/out: the navigating node; a negative value asks for the medoid
 *   repairs   out (optional): number of edges added in step 3
 * Blocking.  ANN_ERR_CAPACITY if step 3 finds no reachable node with a free
 * slot.  Requires K <= 128 and R <= min(K, 64).
 */
ann_status ann_build_graph(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t K,
                           int32_t R, float alpha, int32_t *d_graph, int32_t *medoid,
                           int64_t *repairs, void *stream);

/*
 * The same kind of graph without the O(N^2 d) candidate search, for base sets
 * of many millions of rows: insertion by search.  The first n_seed rows get
 * the exact graph above; the rest are inserted in id order, in batches of at
 * most `batch` rows and at most a quarter of the rows inserted before them:
 * each row of a batch is searched on the graph built so far (beam
 * search as ann_search_batch, from the seed graph's navigating node, pool
 * max(K, 128), W = 4), its K nearest found become its candidates and are
 * pruned to R as in step 2; then each node those rows point to takes them
 * back, appended while its row has room, else its neighbours and the (at
 * most 32 per batch) newcomers are sorted by (squared L2, id) and pruned to R
 * again.  Finally the navigating node of all rows and the repair of step 3.
 * Rows of one batch do not see each other; which newcomers a busy node keeps
 * can vary from run to run (they arrive through atomics).
 *   dtype must be ANN_F32 (else ANN_ERR_UNSUPPORTED); R <= 32; K + 1 <=
 *   n_seed <= n; batch >= 1; other arguments as for ann_build_graph.
 * Blocking.
 * Sec. 2.1, Def. 1 (the proximity graph); the insertion order is this
 * implementation's.
 */
ann_status ann_build_graph_insert(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t K, int32_t R,
                                  float alpha, int64_t n_seed, int64_t batch, int32_t *d_graph, int32_t *medoid,
                                  int64_t *repairs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ANN_H */
