/*
 * gift.h -- C ABI of the GB300 (sm_103a) implementation of GIFT's on-line
 * query path: multi-view matching through the first inverted file (F-IF),
 * top-k selection, and re-ranking through the second inverted file (S-IF)
 * (Bai et al., "GIFT: A Real-time and Scalable 3D Shape Search Engine",
 * CVPR 2016), with the exact set-to-set match as the plain path.
 *
 * Conventions shared by every call:
 *  - A shape x has a set of view features V(x) = {x_1..x_{N_v}}, each a row of
 *    D floats (Sec. 2.3). Feature matrices are row-major, one view per row,
 *    views of a shape consecutive, shapes in id order.
 *  - The caller owns every buffer it passes; the library owns the memory of an
 *    index and of its per-call scratch. No call keeps a caller pointer after
 *    the work it enqueued has run.
 *  - Work is enqueued on `stream` (0 = legacy default stream). Unless stated
 *    otherwise a call returns once its work is enqueued; results are valid
 *    after the stream is synchronised. Pointers documented as "device or host"
 *    may be either: host memory is staged through the library (pinned host
 *    memory keeps the copies asynchronous).
 *  - Every call returns a gift_status. No exception or abort crosses the ABI.
 *    gift_last_error() gives a message for the last failing call of the
 *    calling thread. GIFT_ECUDA leaves the index usable unless the CUDA
 *    context itself was lost.
 *  - A built index is read-only: calls on one index from several host threads
 *    or streams may run concurrently; each call has its own scratch.
 *  - D must be a positive multiple of 16 (16-byte rows for every storage type).
 */
#ifndef GIFT_H
#define GIFT_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define GIFT_API __attribute__((visibility("default")))
#else
#define GIFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GIFT_OK = 0,
  GIFT_EINVAL = 1,       /* an argument is out of range or inconsistent       */
  GIFT_ENOMEM = 2,       /* device or pinned host memory could not be reserved */
  GIFT_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed        */
  GIFT_ETIMEOUT = 4,     /* a bounded wait ran out (serving loop)             */
  GIFT_EUNSUPPORTED = 5, /* the index was built without what the call needs   */
  GIFT_ESTATE = 6        /* the object is in the wrong state for this call    */
} gift_status;

/* Storage type of the F-IF feature store. */
typedef enum { GIFT_F32 = 0, GIFT_BF16 = 1, GIFT_FP8_E4M3 = 2 } gift_dtype;

/* Matching mode of gift_query. */
typedef enum {
  GIFT_MATCH_EXACT = 0, /* Eq. 3 over all view pairs                           */
  GIFT_MATCH_FIF = 1    /* Eq. 4 through the first inverted file               */
} gift_mode;

/* Maximum query-side multiple assignment. */
#define GIFT_MAX_MA 8

typedef struct {
  int32_t n_shapes;        /* N: database shapes                                 */
  int32_t views_per_shape; /* N_v: views of every database shape                 */
  int32_t dim;             /* D: feature dimension, multiple of 16               */
  int32_t n_codewords;     /* K: size of the vocabulary B (Sec. 2.3)             */
  int32_t storage;         /* gift_dtype of the list-ordered feature store       */
  int32_t query_ma;        /* query views go to this many codewords, 1..8        */
  int32_t sif_k1;          /* k1: neighbour-set size of the S-IF (Sec. 2.4); 0 = no S-IF */
  int32_t rescore_r;       /* FP32 rescore of the top-R F-IF candidates; 0 = off */
  int32_t keep_exact;      /* 1 = keep the FP32 feature master (exact match, rescore) */
  int32_t db_ma;           /* database views go to this many codewords, 1..8 (0 = 1);
                              each view is stored once per list it enters (Sec. 2.3:
                              multiple assignment at the cost of memory)               */
} gift_index_params;

typedef struct gift_index gift_index; /* opaque; owns all its device memory */

/* Sizes of a built index (gift_index_info). */
typedef struct {
  size_t device_bytes;      /* device memory held by the index            */
  int64_t n_rows;           /* N * N_v database views                      */
  int32_t n_lists_nonempty; /* non-empty F-IF lists                        */
  int32_t max_list_len;     /* longest F-IF list                           */
  int64_t n_runs;           /* runs of equal shape id over all lists       */
  int32_t max_runs;         /* most runs in one list                       */
  int32_t max_sif_entry;    /* longest S-IF entry                          */
  int64_t n_entries;        /* F-IF entries: n_rows * db_ma                */
  int32_t sif_shapes;       /* shapes the S-IF covers (0 = no S-IF): N, or the
                               whole database for gift_sif_from_neighbours  */
  int32_t sif_k1;           /* k1 of the S-IF                              */
} gift_index_info_t;

/* Per-stage device times of the last timed gift_query / gift_rerank call
 * (milliseconds, CUDA events on the call's stream), see gift_set_timing. */
typedef struct {
  float assign_ms;   /* quantiser of the query views                        */
  float bucket_ms;   /* grouping of query views by codeword                 */
  float scan_ms;     /* posting-list scan (or the exact all-pairs kernel)   */
  float combine_ms;  /* per-view max over assignments, sum into S           */
  float topk_ms;     /* top-R / top-k selections                            */
  float rescore_ms;  /* FP32 rescore of the candidates                      */
  float rerank_ms;   /* S-IF re-rank (gift_rerank)                          */
  float total_ms;    /* whole call                                          */
  int64_t scan_bytes;   /* algorithmic bytes of the scan: touched list rows
                           + their scales and ids + query rows              */
  int64_t rescore_bytes;/* algorithmic bytes of the rescore                  */
  int64_t scan_pairs;   /* (query view, list entry) pairs scanned           */
  float assign_kernel_ms;  /* tensor-core quantiser kernel alone              */
  float scan_kernel_ms;    /* tensor-core scan kernel alone (BF16 store)      */
  float rescore_kernel_ms; /* tensor-core rescore kernel alone                */
  int64_t assign_rows;     /* rows quantised                                  */
  /* candidate work of the FP32 rescore (F-IF queries with rescore_r > 0): a
     work item is (list, tile of 128 entries, tile of the list's query slots:
     16, 32, 64 or 80 of them when the list has at most 80, else 128)         */
  int64_t rescore_items;      /* work items of the touched lists                */
  int64_t rescore_items_kept; /* items holding a run of one of their slots' query's
                                 candidates: the items the rescore runs (the
                                 FP32-level scan of a BF16 store runs every item) */
  int64_t cand_pairs;         /* (slot, entry) pairs whose entry's shape is a
                                 candidate of the slot's query                  */
  int64_t cand_rows;          /* entries whose shape is a candidate of some slot
                                 of their list: the rows the rescore needs      */
  int64_t rescore_rows_read;  /* entries of the kept items                      */
} gift_timing_t;

/*
 * Build an index (off-line stage, Sec. 3.4 "building two inverted files").
 *  - db_feats: device or host, float [N * N_v * D], database views.
 *  - codebook: device or host, float [K * D], the vocabulary B (Sec. 2.3);
 *    trained by the caller (the paper uses k-means).
 * Steps: quantise every database view to its nearest codeword c(x) (one
 * assignment); F-IF (Fig. 2): per codeword, the (shape id, view feature) of
 * every view assigned to it, in ascending (shape, view) order, features
 * converted to `storage`; S-IF (Fig. 3), when sif_k1 > 0: every database shape
 * is matched as a query (F-IF, FP32 rescore when rescore_r > 0), its first k1
 * neighbours (itself included) give F_p (Eq. 7), and entry i stores ||F_i||_1
 * and the pairs (p, F_p[i]) with F_p[i] != 0, p ascending. Memberships are
 * stored as uint32 fixed point round(S * 2^31).
 * Synchronises `stream`; returns after the build is complete.
 * Errors: EINVAL (sizes, D % 16, query_ma, storage), ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_build_index(const gift_index_params* params, const float* db_feats,
                             const float* codebook, cudaStream_t stream, gift_index** out);

/*
 * Streamed build, for databases whose FP32 views do not fit in host or device
 * memory at once. The same index as gift_build_index (keep_exact must be 0: no
 * FP32 master is kept), built from chunks of whole shapes in three passes; in
 * every pass each shape is added exactly once, chunks in any order:
 *   pass 1  quantise the views (codes, norms);            gift_build_end_pass(1) builds the F-IF lists
 *   pass 2  pack the views into their list positions;    gift_build_end_pass(2)
 *   pass 3  (sif_k1 > 0) run the shapes as queries;      gift_build_end_pass(3) builds the S-IF
 * feats: device or host float [n_shapes * N_v * D], the views of shapes
 * [first_shape, first_shape + n_shapes); gift_build_add returns after the chunk
 * has been consumed, so its buffer may be reused. Queries before the last
 * pass is closed return GIFT_ESTATE.
 * Errors: EINVAL (sizes, order of passes, a pass closed before every shape was
 * added), ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_build_begin(const gift_index_params* params, const float* codebook,
                                      cudaStream_t stream, gift_index** out);
GIFT_API gift_status gift_build_add(gift_index* index, int32_t pass, const float* feats,
                                    int32_t first_shape, int32_t n_shapes, cudaStream_t stream);
GIFT_API gift_status gift_build_end_pass(gift_index* index, int32_t pass, cudaStream_t stream);

/* Release the index and all its device memory (synchronises the device). */
GIFT_API void gift_destroy_index(gift_index* index);

/*
 * Query a batch of B shapes and return each query's top-k database shapes.
 *  - q_feats: device or host, float [sum V_q * D], views of all queries.
 *  - q_view_offsets: HOST int32 [B + 1]; query b owns views
 *    [q_view_offsets[b], q_view_offsets[b+1]); V_q >= 1. (Host side because
 *    the launch is sized from it; no device-to-host read is needed.)
 *  - mode GIFT_MATCH_EXACT: S(x_q, x_p) of Eq. 3 with the cosine similarity,
 *    (1/|V(x_q)|) sum_i max_j s(q_i, p_j), over all N shapes (needs keep_exact,
 *    or a BF16/FP8 index built with rescore_r > 0, whose two-part list store is
 *    then read in list order).
 *    mode GIFT_MATCH_FIF: Eq. 4: each query view is quantised to its query_ma
 *    nearest codewords, only the F-IF lists of those codewords are scanned,
 *    and a shape's view contributes its cosine only when one of its codewords
 *    is among them; every other view contributes 0 to the per-(query view,
 *    shape) maximum, so a negative maximum (signed features) counts only when
 *    every view of the shape is matched. With rescore_r > 0 the top rescore_r
 *    shapes are rescored with FP32 features (same Eq. 4).
 *  - out_ids: device or host int32 [B * topk]; out_scores: device or host
 *    float [B * topk]; each row ordered by (score desc, shape id asc). When
 *    N < topk the tail holds id -1 and score -INFINITY.
 * Errors: EINVAL, EUNSUPPORTED (EXACT without keep_exact; topk > rescore_r
 * when rescoring; topk > 1024), ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_query(gift_index* index, const float* q_feats, const int32_t* q_view_offsets,
                       int32_t B, int32_t mode, int32_t topk, int32_t* out_ids, float* out_scores,
                       cudaStream_t stream);

/*
 * S-IF re-ranking (Sec. 2.4, Eqs. 7, 8, 13, 14).
 *  - cand_ids / cand_scores: device or host [B * n_cand], each row a query's
 *    ranked list from gift_query (score desc, id asc), n_cand >= k1.
 *  - The first k1 entries give F_q (Eq. 7). The numerator of Eq. 8 is taken
 *    over the co-non-zero entries only (Eq. 13) by walking S-IF entry i for
 *    each non-zero F_q[i]; the denominator is ||F_q||_1 + ||F_p||_1 minus the
 *    numerator (Eq. 14). Sums are exact in integer fixed point; S' is divided
 *    in FP32.
 *  - Output rows are ordered by (S' desc, S desc, id asc) over all N shapes,
 *    with S taken from the candidate list (shapes outside it rank after those
 *    inside at equal S').
 *  - out_ids: int32 [B * topk]; out_sprime: float [B * topk] (device or host).
 * Errors: EINVAL, EUNSUPPORTED (index built with sif_k1 == 0 or
 * k1 != sif_k1 is allowed but k1 must be <= n_cand), ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_rerank(gift_index* index, const int32_t* cand_ids, const float* cand_scores,
                        int32_t B, int32_t n_cand, int32_t k1, int32_t topk, int32_t* out_ids,
                        float* out_sprime, cudaStream_t stream);

/*
 * S-IF re-ranking that allocates no memory. The paper has no counterpart: this
 * entry point serves callers that cannot allocate device memory while they
 * re-rank -- a process whose free device memory is held by another allocator
 * (a serving framework's caching pool), where an allocation would fail, or a
 * latency-critical loop that must not enter the CUDA allocator (freeing device
 * memory can synchronise the device).
 *  - Same arguments and results as gift_rerank, but every buffer must be in
 *    device memory (host buffers would need staging memory); returns GIFT_EINVAL
 *    otherwise.
 *  - Scratch: one fixed buffer of GIFT_RERANK_NOALLOC_SCRATCH_BYTES inside the
 *    library, created on every device that uses this call and held until the
 *    process exits. A batch needs about 20 * B * N + 8 * B * (topk + 1) bytes
 *    (N = database shapes; 256-byte alignment per part); a larger batch returns
 *    GIFT_EINVAL with the size it needs -- split it.
 *  - Call it with the index's device current (GIFT_EINVAL otherwise); an index
 *    whose streamed build is still open returns GIFT_ESTATE.
 *  - The first call on a device looks up the buffer's device address with that
 *    device current (the runtime loads the library's module there); make that
 *    first call before any stream capture. Later calls check the remembered
 *    address and look it up again after a device reset.
 *  - Every call uses the same buffer and clears what must start at zero; calls
 *    whose work overlaps on the GPU (several streams or host threads at once)
 *    race on it, so the caller must serialise them.
 *  - No cudaMalloc, cudaFree or other allocating routine is called.
 */
#define GIFT_RERANK_NOALLOC_SCRATCH_BYTES (16u << 20)
GIFT_API gift_status gift_rerank_noalloc(gift_index* index, const int32_t* cand_ids,
                                         const float* cand_scores, int32_t B, int32_t n_cand,
                                         int32_t k1, int32_t topk, int32_t* out_ids,
                                         float* out_sprime, cudaStream_t stream);

/*
 * Second inverted file of a database sharded over several indices (one per
 * GPU, each holding a contiguous range of the N shapes; Sec. 2.4, Fig. 3):
 * install on `index` the S-IF of all n_shapes_total shapes from their ranked
 * neighbour rows, so that gift_rerank on this index re-ranks over the whole
 * database (the S-IF is replicated on every shard; no exchange is needed).
 *  - nbr_ids / nbr_scores: device or host [n_shapes_total * k1]; row p is
 *    N_k1(x_p) over the whole database (global ids, itself included, ranked by
 *    (score desc, id asc)) with the scores S(x_p, x_i) that become F_p (Eq. 7),
 *    e.g. the merged sharded query (gift_merge_topk) of every database shape.
 *  - The index must have been built with sif_k1 == 0 (GIFT_ESTATE otherwise);
 *    afterwards gift_rerank and gift_export_sif use global ids in
 *    [0, n_shapes_total). Synchronises `stream`.
 * Errors: EINVAL (sizes, an id outside [0, n_shapes_total)), ESTATE, ENOMEM,
 * ECUDA.
 */
GIFT_API gift_status gift_sif_from_neighbours(gift_index* index, const int32_t* nbr_ids, const float* nbr_scores,
                                              int32_t n_shapes_total, int32_t k1, cudaStream_t stream);

/*
 * Merge of ranked lists (the exchange step of a database-sharded query, where
 * every shard returns its own top-R): each row of (id, score) pairs, ids
 * distinct within a row and id < 0 marking an empty entry, is reduced to its
 * k best pairs by (score desc, id asc) -- the ranking order of gift_query.
 * Eq. 4 scores of a shape depend on that shape's views only, so merging the
 * shards' top lists gives the ranking of an unsharded index.
 *  - ids, scores: device or host [B * n]; out_ids, out_scores: device or host
 *    [B * k]; rows with fewer than k entries end in id -1, score -INFINITY.
 * Errors: EINVAL (B, n, k outside range: 1 <= k <= 1024), ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_merge_topk(const int32_t* ids, const float* scores, int32_t B, int64_t n, int32_t k,
                                     int32_t* out_ids, float* out_scores, cudaStream_t stream);

/*
 * Re-ranking with two similarity measures (Sec. 2.4: Eqs. 9, 10, 11; the
 * paper's default uses two CNN layers, co-augmentation and alpha = 0.5).
 * measure1 and measure2 are indices of the same N database shapes under two
 * feature sets, both with an S-IF of the same k1; they must outlive the
 * gift_aca object, which reads their ranked neighbour rows N_k1(p).
 *  - Contextual activation of a shape under measure l, by mode:
 *      GIFT_ACA_NONE        its Eq. 7 activation F^(l) (first k1 neighbours);
 *      GIFT_ACA_AUGMENT     Eq. 10: the mean of the Eq. 7 activations F_i^(l)
 *                           of its first k2 neighbours i under measure l;
 *      GIFT_ACA_CO_AUGMENT  Eq. 11: the same mean over its first k2 neighbours
 *                           under the other measure.
 *    The two are fused per coordinate by the generalised mean of Eq. 9 with
 *    exponent alpha (> 0), and S' of Eq. 8 compares fused activations.
 *  - gift_aca_build computes the fused activation of every database shape
 *    and transposes it into a second inverted file of its own (entries in
 *    ascending shape id; memberships uint32 fixed point round(F * 2^31);
 *    norms uint64 in the same fixed point). 1 <= k2 <= k1; k2 * k1 <= 2048
 *    (k1 <= 1024 without augmentation).
 *  - gift_aca_rerank: cand_ids1/cand_scores1 and cand_ids2/cand_scores2 are
 *    the ranked [B, n_cand] results of gift_query on measure1 and measure2
 *    (n_cand >= k1). Output: the top-k of all N shapes by (S' desc, S^(1)
 *    desc, id asc), S^(1) taken from the first list (-inf when absent); ids and
 *    S' [B, topk]; device or host buffers.
 *  - gift_aca_export copies the transposed activations (device or host
 *    buffers; offsets [N + 1], ids and members [pairs], norms [N]); pairs from
 *    gift_aca_pairs.
 * Errors: EINVAL (sizes, k2, alpha, mismatched indices), EUNSUPPORTED (an
 * index without S-IF), ESTATE (an index still being built), ENOMEM, ECUDA.
 */
typedef struct gift_aca gift_aca; /* opaque; owns its device memory */
typedef enum { GIFT_ACA_NONE = 0, GIFT_ACA_AUGMENT = 1, GIFT_ACA_CO_AUGMENT = 2 } gift_aca_mode;
GIFT_API gift_status gift_aca_build(const gift_index* measure1, const gift_index* measure2, int32_t k2,
                                    float alpha, int32_t mode, cudaStream_t stream, gift_aca** out);
GIFT_API gift_status gift_aca_rerank(gift_aca* aca, const int32_t* cand_ids1, const float* cand_scores1,
                                     const int32_t* cand_ids2, const float* cand_scores2, int32_t B,
                                     int32_t n_cand, int32_t topk, int32_t* out_ids, float* out_sprime,
                                     cudaStream_t stream);
GIFT_API gift_status gift_aca_pairs(const gift_aca* aca, int64_t* pairs);
GIFT_API gift_status gift_aca_export(const gift_aca* aca, int64_t* entry_offsets, int32_t* entry_ids,
                                     uint32_t* entry_members, uint64_t* card, cudaStream_t stream);
GIFT_API void gift_aca_destroy(gift_aca* aca);

/*
 * Projection front end (Sec. 2.1): the depth-buffer views of a batch of meshes.
 *  - vertices: device or host float [sum V_m * 3]; triangles: device or host
 *    int32 [sum T_m * 3], vertex indices local to their mesh; vert_off /
 *    tri_off: host int64 [M + 1] offsets (in vertices / triangles) of each mesh.
 *  - Each mesh is normalised: the area-weighted centroid of its surface goes to
 *    the origin and the largest vertex distance from it becomes 1 (scale and
 *    translation only, as in the paper).
 *  - Cameras on the unit sphere at azimuth 2 pi i / n_az and elevation
 *    pi ((j + 1/2) / n_el - 1/2), view v = j * n_az + i, look at the origin:
 *    forward f, right r = f x z / |f x z|, up u = r x f. Orthographic H x W
 *    image over [-1, 1]^2 in (r, u); pixel (y, x) samples its centre
 *    (-1 + (2x + 1) / W, 1 - (2y + 1) / H); a closed triangle covers the samples
 *    where its three edge functions are >= 0; depth = p . f + 1 in [0, 2]
 *    interpolated across the triangle; the nearest depth is kept; 2 where
 *    nothing is seen.
 *  - depth: device or host float [M, n_az * n_el, H, W].
 * Errors: EINVAL (sizes, offsets, a vertex index outside its mesh), ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_render_views(const float* vertices, const int32_t* triangles, const int64_t* vert_off,
                                       const int64_t* tri_off, int32_t M, int32_t n_az, int32_t n_el, int32_t H,
                                       int32_t W, float* depth, cudaStream_t stream);

/*
 * Lloyd's k-means on the GPU: the off-line vocabulary B of Sec. 2.3 (the paper
 * trains it with k-means and gives no details).
 *  - X: device or host float [n * D] (D a multiple of 16); init_rows: host
 *    int32 [K], the rows that start as centres; iters >= 0 iterations.
 *  - Each iteration assigns every row to its nearest centre exactly as
 *    gift_assign does (ties to the lowest index) and moves every centre to the
 *    mean of its rows (float64 sums in ascending row order: deterministic); a
 *    centre left without rows takes the row farthest from the centre it was
 *    assigned to (distance desc, index asc), empty centres in ascending order.
 *  - codebook: device or host float [K * D], written when the call returns.
 * Errors: EINVAL (sizes, rows out of range), ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_kmeans(const float* X, int64_t n, int32_t D, int32_t K, const int32_t* init_rows,
                                 int32_t iters, float* codebook, cudaStream_t stream);

/*
 * The quantiser alone (Sec. 2.3): out_codes[v * ma + a] is the a-th nearest
 * codeword of row v by (squared distance, index), c(x) = argmin_k ||x - b_k||^2.
 *  - feats: device float [n * D]; out_codes: device int32 [n * ma]; 1 <= ma <= 8.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_assign(gift_index* index, const float* feats, int64_t n, int32_t ma,
                        int32_t* out_codes, cudaStream_t stream);

/*
 * Copy the F-IF of a built index to caller buffers (device or host):
 * db_codes int32 [N * N_v] (codeword of each database view), list_offsets
 * int64 [K + 1], list_rows int32 [N * N_v] (row = shape * N_v + view, list
 * order). Any pointer may be NULL to skip it. Synchronises `stream`.
 */
GIFT_API gift_status gift_export_fif(const gift_index* index, int32_t* db_codes, int64_t* list_offsets,
                            int32_t* list_rows, cudaStream_t stream);

/*
 * Copy the S-IF of a built index (device or host): entry_offsets int64 [N + 1],
 * entry_ids int32 [N * k1] (shape p of each pair), entry_members uint32
 * [N * k1] (F_p[i] in fixed point 2^31), card uint64 [N] (||F_i||_1 in the same
 * fixed point), N and k1 as gift_index_info reports them (sif_shapes, sif_k1).
 * Any pointer may be NULL. Synchronises `stream`.
 * Errors: EUNSUPPORTED when the index has no S-IF.
 */
GIFT_API gift_status gift_export_sif(const gift_index* index, int64_t* entry_offsets, int32_t* entry_ids,
                            uint32_t* entry_members, uint64_t* card, cudaStream_t stream);

/* Sizes of a built index. */
GIFT_API gift_status gift_index_info(const gift_index* index, gift_index_info_t* out);

/* Change the FP32 rescore depth R of later gift_query calls (0 = rank by the
 * store's scores alone). R > 0 needs an index built with rescore_r > 0 (the
 * rescore store). Not to be called while another call or a server uses the
 * index. Errors: EINVAL (R outside [0, 1024]), EUNSUPPORTED, ESTATE. */
GIFT_API gift_status gift_set_rescore_depth(gift_index* index, int32_t rescore_r);

/*
 * Per-stage timing of gift_query / gift_rerank calls on this index: when
 * enabled, each call records CUDA events around its stages on its stream;
 * gift_get_timing synchronises on the last call's final event and returns the
 * stage times. Timing is off by default.
 */
GIFT_API gift_status gift_set_timing(gift_index* index, int32_t enable);
GIFT_API gift_status gift_get_timing(gift_index* index, gift_timing_t* out);

/*
 * Set-to-set matching score of Eq. 3 after a linear view projection
 * u = W q (W may be NULL for the identity), for training the projection:
 *   S[b, p] = (1/|V(x_b)|) sum_i max_j s(W q_i, W p_j).
 *  - dtype GIFT_F32 or GIFT_BF16: element type of q, p and W.
 *  - q: device [sum V_q * d_in]; q_view_offsets: HOST int32 [Bq + 1].
 *  - p: device [Np * nv_p * d_in]; W: device [d_out * d_in] or NULL (then
 *    d_out must equal d_in). d_in, d_out multiples of 16.
 *  - S: device float [Bq * Np]; argmax: device int16 [sum V_q * Np], the first
 *    j attaining the max for every (query view, database shape), saved for the
 *    backward pass; nv_p <= 32767.
 * Products run on the tensor cores; the similarity of the projected views is
 * evaluated in FP32-level precision (two-part BF16 operands).
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_match_forward(const void* q, const int32_t* q_view_offsets, int32_t Bq,
                                        const void* p, int32_t Np, int32_t nv_p, const void* W,
                                        int32_t d_in, int32_t d_out, int32_t dtype, float* S,
                                        int16_t* argmax, cudaStream_t stream);

/*
 * Gradient of L = sum_{b,p} grad_S[b,p] * S[b,p] through gift_match_forward,
 * taken through the saved argmax view pair (the max of Eq. 3 is piecewise
 * linear in the selected pair):
 *   dS/du_i = (v_j/|v_j| - s u_i/|u_i|) / |u_i|, dS/dv_j = (u_i/|u_i| - s v_j/|v_j|) / |v_j|,
 * each scaled by grad_S[b,p] / |V(x_b)|; dW = dU^T Q + dV^T P, dQ = dU W, dP = dV W.
 *  - grad_S: device float [Bq * Np]; argmax from the forward call (an entry outside
 *    [0, nv_p) contributes nothing); inputs as in gift_match_forward (same dtype).
 *  - dW: device float [d_out * d_in] or NULL (skipped; must be NULL when W is);
 *    dQ: device float [sum V_q * d_in] or NULL; dP: device float
 *    [Np * nv_p * d_in] or NULL. Outputs are FP32 and overwritten; d_out <= 1024.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
GIFT_API gift_status gift_match_backward(const void* q, const int32_t* q_view_offsets, int32_t Bq,
                                         const void* p, int32_t Np, int32_t nv_p, const void* W,
                                         int32_t d_in, int32_t d_out, int32_t dtype,
                                         const float* grad_S, const int16_t* argmax, float* dW,
                                         float* dQ, float* dP, cudaStream_t stream);

/*
 * Request loop over a resident index (serving). Requests of mixed view counts
 * are queued; a dispatcher thread forms batches from the head of the queue
 * whenever one of `slots` batch slots is free, admits a batch only while the
 * device memory of all batches in flight fits `memory_budget`, and runs each
 * batch (F-IF query, optional S-IF re-rank) on its slot's own stream, so
 * batches overlap on the device. Results and latencies (submission to
 * completion) are per request. Sec. 2 and Table 4 of the paper measure the
 * per-query on-line time; this loop is the batched GPU form of that service.
 */
typedef struct {
  int32_t slots;             /* batches in flight, 1..16                                   */
  int32_t max_batch_queries; /* queries per batch                                          */
  int32_t max_batch_views;   /* views per batch (and per request)                          */
  int32_t topk;              /* results per request (<= rescore depth when rescoring)      */
  int32_t rerank;            /* 1 = results are S-IF re-ranked (needs sif_k1 > 0)          */
  int32_t start_paused;      /* 1 = queue requests until gift_server_resume                */
  int64_t memory_budget;     /* device bytes for slot buffers + batches in flight; 0 = 80%
                                of the free device memory at creation                      */
} gift_server_params;

typedef struct {
  int64_t completed, failed, batches, queued;
  float mean_batch;     /* queries per batch                                             */
  float p50_ms, p99_ms, max_ms;  /* latency, submission to completion                     */
  float queries_per_s;  /* completed / (last completion - first submission)              */
  int64_t admission_waits;      /* dispatcher passes that held a batch back because the
                                   batches in flight left too little of the budget      */
  int64_t peak_in_flight_bytes; /* most admitted bytes of batches in flight at once     */
  int64_t budget_bytes;         /* budget for batches in flight (after slot buffers)    */
  int64_t max_batch_bytes;      /* admission estimate of a batch of the maximum size    */
  int64_t slot_bytes;           /* device and pinned buffers of all slots               */
} gift_server_stats_t;

typedef struct gift_server gift_server;

/* Start a request loop on the current device for `index` (which must outlive it).
 * Errors: EINVAL (limits, budget smaller than one batch), ENOMEM, ECUDA. */
GIFT_API gift_status gift_server_create(gift_index* index, const gift_server_params* params,
                                        gift_server** out);
/* Queue one request: q_feats HOST float [n_views * D] (copied before return).
 * Writes a ticket. Errors: EINVAL (n_views outside [1, max_batch_views]), ESTATE. */
GIFT_API gift_status gift_server_submit(gift_server* server, const float* q_feats, int32_t n_views,
                                        int64_t* ticket);
/* Wait at most timeout_ms for a request; on success copy its topk ids / scores
 * (S' when re-ranking) to HOST buffers and forget the ticket. GIFT_ETIMEOUT when
 * the request is not complete in time (the ticket stays valid). */
GIFT_API gift_status gift_server_wait(gift_server* server, int64_t ticket, int32_t timeout_ms,
                                      int32_t* out_ids, float* out_scores);
/* Start dispatching a server created with start_paused = 1. */
GIFT_API gift_status gift_server_resume(gift_server* server);
GIFT_API gift_status gift_server_stats(gift_server* server, gift_server_stats_t* out);
/* Finish queued and in-flight requests, stop the dispatcher, free the slots. */
GIFT_API void gift_server_destroy(gift_server* server);

/* Number of CUDA kernels this library has launched in the process so far
 * (all threads); the difference across a region counts its launches. */
GIFT_API int64_t gift_launch_count(void);

/* Message of the last failing call on the calling thread ("" if none). */
GIFT_API const char* gift_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
GIFT_API int32_t gift_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GIFT_H */
