/*
 * dt.h — C ABI of libdt.so: weighted-Hamming nearest-neighbour search over
 * 64x64-bit QUICCI descriptors, by brute force and through a Dissimilarity
 * Tree, plus per-object voting for partial-object retrieval.
 *
 * The operations follow arXiv 2107.03368 (van Blokland & Theoharis,
 * "Partial 3D Object Retrieval using Local Binary QUICCI Descriptors and
 * Dissimilarity Tree Indexing"):
 *   distance      Eq. 1 (§2.3), weighted Hamming distance
 *   bf_search     sequential search (§6.2)
 *   dt_build      Dissimilarity Tree construction (§4.1)
 *   dt_search     Dissimilarity Tree query (§4.2)
 *   retrieve_objects   the voting pipeline (§3)
 *
 * Common conventions
 * ------------------
 * Descriptor layout: 64 x uint64 = 4096 bits = 512 bytes, row-major; word r
 *   holds layer r counted from the bottom, bit c of it the circle of radius
 *   index c counted from the innermost (§2.2).  Descriptor arrays are
 *   contiguous [count][64] uint64 and must be 16-byte aligned.
 * Distance: for query q and target t, A = #(q=1, t=0), B = #(q=0, t=1),
 *   P = max(|q|, 1), Z = max(4096 - |q|, 1) and delta = A/P + B/Z (Eq. 1,
 *   with 4096 = N*N bits as the count of possible type B errors).
 *   Results are ranked by the exact value of delta, i.e. by the integer
 *   A*Z + B*P, ties by lowest database index.  Scores are FP32: delta
 *   correctly rounded from the exact rational (A*Z + B*P) / (P*Z).
 * Results: idx[nq][k] (uint32, original database index), score[nq][k]
 *   (float), ab[nq][k][2] (uint16 A then B; optional).  Row i is sorted by
 *   ascending (delta, idx).  When fewer than k descriptors exist, the extra
 *   slots hold idx = 0xFFFFFFFF, score = +inf, A = B = 0xFFFF.
 * Memory: every pointer named d_* is CUDA device memory owned by the caller
 *   and must stay valid until the stream reaches the call's end.  The
 *   library owns dt_index objects and any scratch space it allocates.
 *   Scratch comes from a stream-ordered memory pool that the library
 *   creates for each device on first use and keeps until the process
 *   exits; its release threshold is 16 GiB, so freed scratch stays cached
 *   between calls.  The device's default pool and its settings are left
 *   alone.  Under stream capture scratch is allocated by the graph.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *   enqueue their work and return; outputs are ready when the stream is.
 *   dt_build and calls that return host statistics synchronise the stream.
 * Errors: every call returns DT_OK (0) or a negative status; on error no
 *   output is guaranteed.  dt_status_string() names a status, and
 *   dt_last_error() gives a message for the most recent failure in the
 *   calling thread.
 * Limits: 1 <= k <= DT_MAX_K; database size n <= DT_MAX_N; nq < 2^31.
 */
#ifndef DT_H
#define DT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DT_WORDS 64
#define DT_BITS 4096
#define DT_MAX_K 32
#define DT_MAX_N 2147483647LL

enum {
    DT_OK = 0,
    DT_EINVAL = -1,        /* bad argument: null pointer, size, alignment, k */
    DT_ENOMEM = -2,        /* device allocation failed */
    DT_ECUDA = -3,         /* a CUDA runtime call failed */
    DT_ETIMEOUT = -4,      /* a bounded device wait gave up */
    DT_EUNSUPPORTED = -5,  /* valid request this library or device cannot serve */
    DT_EIO = -6            /* a file could not be opened, read or written */
};

/* Opaque Dissimilarity Tree index; created by dt_build, freed by dt_free. */
typedef struct dt_index dt_index;

typedef struct {
    int32_t leaf_size;      /* a node with at most this many descriptors is a leaf
                               (§4.1; the paper found 32 best); <= 0 means 32 */
    int32_t use_and_image;  /* nonzero: also keep each node's AND (product) image
                               and add its type B term to the bound (§4) */
    int32_t fused_cap;      /* nodes of at most this many descriptors are split by
                               one thread block; larger ones by the multi-block
                               path.  <= 0 means the default (2048).  Both paths
                               compute the same split; this only tunes speed. */
    int32_t reserved;       /* must be 0 */
} dt_build_params;

typedef struct {
    int64_t n_nodes;        /* nodes; breadth first after dt_build (see dt_insert) */
    int64_t n_leaves;
    int32_t depth;          /* deepest level (root = 0) */
    int32_t leaf_size;
    int64_t n;              /* indexed descriptors */
    int32_t use_and_image;
    int32_t reserved;
} dt_index_info;

typedef struct {
    int64_t nodes_visited;     /* nodes whose subtree was entered (inner + leaf) */
    int64_t leaves_visited;    /* leaves scanned */
    int64_t descs_scanned;     /* descriptors whose exact distance was computed */
    int64_t bounds_evaluated;  /* node images read to bound a subtree */
} dt_stats;

/*
 * dt_build — Dissimilarity Tree over n descriptors (§4.1).
 *
 * Each node with more than leaf_size descriptors is split in two.  Bit
 * popularity = how many of the node's descriptors set each bit; bits are
 * taken in ascending popularity (ties: lower bit index first) and every
 * descriptor still in the similar set that has the current bit set moves to
 * the dissimilar set, stopping right after the bit at which the dissimilar
 * set first holds ceil(n/2) descriptors.  If a side would be empty, the
 * node's descriptors (ascending index) are cut at floor(n/2) instead.  Every
 * node stores the OR (sum) image of its descriptors.  Nodes are numbered
 * breadth first, similar child before dissimilar child.
 *
 * d_db: [n][64] uint64 device array (n >= 1), read during the call only: the
 *   index keeps its own tree-ordered copy.  params: nullable (defaults).
 * out: receives the new index.  Synchronises `stream`.
 * Errors: DT_EINVAL (null d_db/out, n < 1, n > DT_MAX_N, misaligned,
 * reserved != 0), DT_ENOMEM, DT_ECUDA.
 */
int dt_build(const uint64_t *d_db, int64_t n, const dt_build_params *params, void *stream,
             dt_index **out);

/*
 * Incremental insertion.  §4.1 suggests that a tree can grow by redoing only
 * the part that new descriptors touch; the rules below are this library's
 * reading of that suggestion.  Appends the m descriptors d_new [m][64]
 * (device, 16-byte aligned, not retained) to the index; they take original
 * indices n .. n+m-1, n being the index's size before the call.
 *   - Each new descriptor descends from the root into the child whose images
 *     it widens least (its set bits outside the child's OR image, plus, with
 *     AND images, its clear bits inside the child's AND image), the similar
 *     child on ties, always against the tree as it was before the call.
 *   - It joins that leaf after the leaf's descriptors (a leaf keeps
 *     ascending original index), and every node on its path takes it into
 *     its images.
 *   - Every leaf left with more than leaf_size descriptors is split again by
 *     dt_build's construction as the root of a new subtree.  New nodes are
 *     numbered after the existing ones, one generation at a time over all
 *     rebuilt subtrees (so the index is no longer numbered breadth first).
 * Searches on the updated index stay exact.  Cost: one pass over the
 * tree-ordered database (rows move to make room), O(m x depth) routing, and
 * the rebuilt subtrees.  Synchronous: returns once the work on `stream` is
 * complete.  The index must not be searched on another stream meanwhile,
 * and the current device must be the one it was built on.  m == 0 is a
 * no-op.
 * Errors: DT_EINVAL (null index, m < 0, n + m > DT_MAX_N - 65536, null or
 * misaligned d_new with m > 0, another current device), DT_ENOMEM, DT_ECUDA.
 * On every error the index is left as it was.  An index that keeps a
 * widened copy (dt_keep_widened) has it rebuilt after the rows move; when
 * the new copy does not fit it is dropped and the call still succeeds
 * (searches stay exact, only slower).
 */
int dt_insert(dt_index *index, const uint64_t *d_new, int64_t m, void *stream);

/*
 * dt_keep_widened — keep (on = 1) or release (on = 0) a resident copy of the
 * index's tree-ordered descriptors widened for the tensor cores.  Not a
 * step of the paper's method: the batched traversal of dt_search (§4.2 with
 * the sequential scan of §6.2 on the tensor cores) multiplies the rows as
 * FP8 E4M3 bytes (one byte per bit), and without a kept copy every call
 * widens the whole database again (about 1.5 ms per million descriptors).
 * Cost: 4,096 bytes per descriptor plus 528 bytes per 128 descriptors of
 * device memory (41 GB at 10M), plain device allocations owned by the
 * index until dt_free, dt_keep_widened(index, 0, ...) or an insertion that
 * no longer leaves room.  Results never change.  The widening runs on
 * `stream` and is complete on return; call it while no search of the index
 * is running.  The current device must be the index's.
 * Errors: DT_EINVAL (null index, on not 0 or 1, another current device),
 * DT_ENOMEM (the copy does not fit; the index is unchanged), DT_ECUDA.
 */
int dt_keep_widened(dt_index *index, int32_t on, void *stream);

/*
 * QUICCI descriptors (§2.2) of oriented points on a triangle mesh, or the
 * modified QUICCI of §5 for partial query meshes (modified != 0).  Bit
 * (layer l, circle c) — bit c of word l of a point's 64 words — is set iff
 * the number of points where circle c meets the mesh differs from that of
 * circle c - 1, by at least 2 when modified (boundaries of a partial mesh
 * change counts by 1, closed surfaces by 2).  Geometry (this library's
 * reading; the paper describes it in words): the point's normal,
 * normalised (a zero normal gives an empty descriptor), is the axis; layer
 * l is the plane at height -R + (2l + 1) R / 64 along it, so the layers
 * evenly fill [-R, R]; circle c has radius (c + 1) R / 64, circle -1 radius
 * 0.  A layer plane cuts a triangle when some vertex lies below it (height
 * < the plane's) and some does not.
 * d_vertices [n_vertices][3] float, d_triangles [n_triangles][3] int32
 * vertex ids, d_points and d_normals [n_points][3] float, all device
 * memory; d_out [n_points][64] uint64 (device, 16-byte aligned).  FP32
 * arithmetic: a bit can differ from exact arithmetic only where a circle
 * passes within rounding distance of a segment's end or closest point, or a
 * layer plane within rounding distance of a vertex.  Triangles are sorted
 * along a Morton curve and grouped by 32; every point tests every group's
 * bounding sphere, then the triangles of the groups that reach its support
 * cylinder.  Waits on the host once, to validate the triangles' vertex ids,
 * then enqueues the sort and the descriptor kernel on `stream` (scratch is
 * released on the stream after them).
 * Errors: DT_EINVAL (null or misaligned pointers, negative or too large
 * sizes, triangles without vertices, support_radius not positive and
 * finite, a vertex id outside [0, n_vertices)), DT_ENOMEM, DT_ECUDA.
 */
int quicci_generate(const float *d_vertices, int64_t n_vertices, const int32_t *d_triangles,
                    int64_t n_triangles, const float *d_points, const float *d_normals,
                    int64_t n_points, float support_radius, int32_t modified, uint64_t *d_out,
                    void *stream);

/*
 * Saving and loading an index (checkpoint / resume).  dt_save writes the
 * tree of `index` — built or grown by dt_insert — to `path`: a 64-byte
 * header (magic "DTINDEX", version 1, n, node and leaf counts, depth,
 * leaf_size, AND images or not), the node records, the OR (and AND) images,
 * the permutation, and a 64-bit checksum of everything after the header;
 * little-endian.  The descriptors are not written: dt_load takes the
 * database d_db [n][64] (device, 16-byte aligned, original-index order, the
 * same rows the index was built and grown over) and rebuilds the
 * tree-ordered copy on the GPU.  Before anything reaches the device,
 * dt_load checks the header, the file size, the checksum, that the nodes
 * form one tree rooted at node 0 whose children split their parent's
 * segment one level below it, that leaves hold at most leaf_size
 * descriptors, the recorded depth and leaf count, and that the permutation
 * is one; images are taken as written.  Both are synchronous.
 * Errors: DT_EINVAL (null arguments, n different from the file's, a
 * rejected file — dt_last_error names the check), DT_EIO (the file cannot
 * be opened, read or written), DT_ENOMEM, DT_ECUDA.
 */
int dt_save(const dt_index *index, const char *path);
int dt_load(const char *path, const uint64_t *d_db, int64_t n, void *stream, dt_index **out);

/* Shape of a built index (host call, no device work). */
int dt_get_info(const dt_index *index, dt_index_info *info);

/*
 * dt_export — copy the flattened tree to host memory (synchronous), for
 * inspection and tests.  Any pointer may be NULL to skip that array.
 *   h_child[n_nodes][2] int64: similar, dissimilar child; -1 at a leaf
 *   h_begin[n_nodes], h_count[n_nodes] int64: the node's segment of h_perm
 *   h_level[n_nodes] int32: depth
 *   h_or[n_nodes][64], h_and[n_nodes][64] uint64: images (h_and requires an
 *     index built with use_and_image)
 *   h_perm[n] int64: tree position -> original database index
 */
int dt_export(const dt_index *index, int64_t *h_child, int64_t *h_begin, int64_t *h_count,
              int32_t *h_level, uint64_t *h_or, uint64_t *h_and, int64_t *h_perm);

/*
 * dt_search — exact k nearest database descriptors of each query by
 * Dissimilarity Tree traversal (§4.2).  A subtree is skipped only when its
 * bound, popc(q & ~OR) * Z (+ popc(~q & AND) * P with AND images), is
 * strictly greater than a key known to be >= the query's k-th result's
 * A*Z + B*P, so the result equals bf_search's, ties included.
 *
 * Two traversals, chosen by batch and index size (dt_search_path picks
 * explicitly):
 *   per query (fewer than 64 queries on an index of fewer than 131,072
 *     descriptors): a warp per query walks the tree
 *     depth first with the bound of every node (dt_stats counts its nodes,
 *     leaves, descriptors and bounds);
 *   batched (64 or more queries, or any batch on a larger index, where one
 *     warp walking most of the rows would take far longer than one shared
 *     scan): every query first descends greedily to one leaf
 *     and scans it, which gives a cap >= its k-th key; queries are sorted
 *     by the position of that leaf and grouped 256 at a time; the tensor
 *     cores bound every (group, run of 128 tree-ordered rows) by the run's
 *     OR image, scan exactly the runs some query of the group may need
 *     (skipping the 128-bit chunks in which the run has no bit) and keep
 *     per query the keys <= its cap.  The AND image is not used there (a
 *     weaker bound, still exact).  dt_stats: nodes_visited and
 *     bounds_evaluated count the descents plus one bound per (query, run);
 *     leaves_visited counts the descents' leaves; descs_scanned counts the
 *     descents' rows plus every (query, row) pair of the runs scanned for
 *     its group.
 *
 * d_q: [nq][64] queries.  d_idx, d_score: [nq][k].  d_ab: [nq][k][2] or NULL.
 * h_stats: NULL, or host struct receiving totals over all queries (this
 * synchronises the stream).  nq = 0 is a no-op.  The current device must
 * be the index's.
 * Errors: DT_EINVAL, DT_ENOMEM, DT_ECUDA; a device wait that gave up is
 * reported by the next dt_sync_status (DT_ETIMEOUT).
 */
int dt_search(const dt_index *index, const uint64_t *d_q, int64_t nq, int32_t k,
              uint32_t *d_idx, float *d_score, uint16_t *d_ab, dt_stats *h_stats,
              void *stream);

/*
 * dt_search_seeded — dt_search with a warm start.  The paper's query (§4.2)
 * starts with an empty result list; here the caller may name, per query,
 * up to n_seed candidate database indices (for instance the answers of the
 * learned proposal).  Their exact keys are computed first, and the k-th
 * smallest of them, which can only be >= the exact k-th result's key, caps
 * the pruning threshold from the first node on.  The result is exactly
 * dt_search's (same indices, scores and (A, B)); only the work changes.
 *
 * d_seed: [nq][n_seed] uint32 original database indices; 0xFFFFFFFF (or any
 * index >= n) means "no candidate"; duplicates count once.  n_seed in
 * [0, 4096]; n_seed = 0 is plain dt_search.  Fewer than k valid distinct
 * candidates give no cap.  Other arguments, outputs and errors as dt_search.
 * In the batched traversal the candidates join the descent's leaf in the
 * cap, so a good proposal prunes runs of rows for whole groups of queries.
 */
int dt_search_seeded(const dt_index *index, const uint64_t *d_q, int64_t nq, int32_t k,
                     const uint32_t *d_seed, int32_t n_seed, uint32_t *d_idx, float *d_score,
                     uint16_t *d_ab, dt_stats *h_stats, void *stream);

/*
 * dt_search_path — dt_search_seeded with the traversal chosen by the
 * caller: path 0 = automatic (as dt_search), 1 = per query, 2 = batched.
 * All paths give identical results.  d_seed may be NULL when n_seed = 0.
 * Errors: as dt_search, and DT_EINVAL for another path.
 */
int dt_search_path(const dt_index *index, const uint64_t *d_q, int64_t nq, int32_t k,
                   const uint32_t *d_seed, int32_t n_seed, uint32_t *d_idx, float *d_score,
                   uint16_t *d_ab, dt_stats *h_stats, int32_t path, void *stream);

/*
 * bf_search — exact k nearest database descriptors by scanning all of them
 * (the sequential search of §6.2).
 *
 * d_db: [n][64] database (n >= 1), d_q: [nq][64] queries; outputs as in
 * dt_search.  path: 1 = popcount kernel (CUDA cores), 2 = tensor-core
 * kernel (tcgen05, the overlap as an FP8 0/1 contraction with exact FP32
 * accumulation in tensor memory), 0 = automatic (2 for 64 or more queries).
 * Both paths give identical results.  Allocates scratch from the
 * stream-ordered allocator.
 * Errors: DT_EINVAL, DT_ENOMEM, DT_ECUDA; a device wait that gave up is
 * reported by the next dt_sync_status (DT_ETIMEOUT).
 */
int bf_search(const uint64_t *d_db, int64_t n, const uint64_t *d_q, int64_t nq, int32_t k,
              uint32_t *d_idx, float *d_score, uint16_t *d_ab, int32_t path, void *stream);

/*
 * bf_search_noalloc — bf_search (path 1, popcount kernel) that allocates no
 * memory at all.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library allocate device memory, for example a
 * serving process that has divided the GPU among models in advance or a host
 * framework that owns all device memory through its own arena.  For them a
 * hidden cudaMalloc / cudaMallocAsync can fail at an arbitrary moment, may
 * synchronise the device, and escapes their memory accounting.
 *
 * The caller passes inputs and outputs exactly as for bf_search.  The only
 * scratch (the per-split top-k lists) lives in a fixed array of
 * DT_NOALLOC_SCRATCH_BYTES compiled into the library; every GPU that loads
 * the library holds that array until the process exits.
 *   Limit: nq * k * 8 <= DT_NOALLOC_SCRATCH_BYTES (nq * k <= 2,097,152);
 *   larger requests return DT_EINVAL without touching the GPU — split the
 *   queries into batches.
 *   Set-up: the first call on a device (with that device current) looks up
 *   the array's device address; make that first call before any stream
 *   capture.
 *   Sharing: all calls on a device share the array; each call first fills
 *   the part it uses with the empty pattern (a stream-ordered memset, no
 *   allocation).  Calls whose work overlaps on the GPU (e.g. on two
 *   unordered streams) race on it; order them on one stream.
 * Results are identical to bf_search's.
 * Errors: DT_EINVAL (bad arguments, or a request larger than the fixed
 * scratch), DT_EUNSUPPORTED (device ordinal 64 or above), DT_ECUDA.  A
 * device wait that gave up is not reported by this call: the kernel raises
 * the same device-side flag as bf_search's popcount path, and the next
 * dt_sync_status returns DT_ETIMEOUT.  That status covers every search
 * enqueued since the previous dt_sync_status, so it cannot tell which call
 * timed out; call dt_sync_status right after this one to attribute it.
 * Nothing in this call touches a memory pool or its settings.
 */
#define DT_NOALLOC_SCRATCH_BYTES (16u << 20)
int bf_search_noalloc(const uint64_t *d_db, int64_t n, const uint64_t *d_q, int64_t nq, int32_t k,
                      uint32_t *d_idx, float *d_score, uint16_t *d_ab, void *stream);

/*
 * retrieve_objects — partial-object retrieval by voting (§3).
 *
 * Query j owns descriptors d_qdesc[d_qoffsets[j] .. d_qoffsets[j+1]).  Its
 * descriptors are drawn in a random order (Fisher-Yates driven by SplitMix64,
 * seeded from `seed` and j); each drawn descriptor's nearest database
 * descriptor (top-1 by the tree) votes for its object d_object_of_desc[idx].
 * With vote_threshold T > 0 drawing stops when an object reaches T votes and
 * that object wins; with T = 0 every descriptor votes and the object with
 * most votes wins (lowest id on ties).  A query without descriptors gets
 * winner -1.
 *
 * d_object_of_desc: [n] uint32, indexed by original database index; ids
 *   outside [0, n_objects) cast no vote.
 * d_qoffsets: [nq+1] int64 device array, non-decreasing, d_qoffsets[0] = 0;
 *   n_qdesc (host) must equal d_qoffsets[nq], the number of query descriptors.
 * d_votes: [nq][n_objects] uint32 — the votes cast.  d_winner: [nq] int32.
 * d_consumed: [nq] int64 descriptors drawn, or NULL.
 * engine selects how the nearest neighbours are found; every engine is
 *   exact, so the outputs do not depend on it: 1 = Dissimilarity Tree
 *   traversal (§4.2), one warp per descriptor, all in one persistent
 *   launch; 2 = tensor-core scan of the index's whole database; 3 = the
 *   batched tree search of dt_search (descriptors of one partial query
 *   share leaves, so their groups skip most of the database); 0 =
 *   automatic (dt_autotune_retrieve's choice when tuned, else 3 when
 *   n_qdesc >= 256 or the index holds 131,072 descriptors or more, else
 *   1).  With T > 0, engines 2 and
 *   3 search the draws in rounds of T, 2T, ... per undecided query, so
 *   mostly only the draws the loop consumes are searched.
 * With T = 0 the call does not synchronise the stream; with T > 0 and
 * engine 2 it reads each round's batch size back (synchronises).
 * Errors: DT_EINVAL, DT_ENOMEM, DT_ECUDA, DT_ETIMEOUT.
 */
int retrieve_objects(const dt_index *index, const uint32_t *d_object_of_desc, int32_t n_objects,
                     const uint64_t *d_qdesc, const int64_t *d_qoffsets, int32_t nq,
                     int64_t n_qdesc, int32_t vote_threshold, uint64_t seed, uint32_t *d_votes,
                     int32_t *d_winner, int64_t *d_consumed, int32_t engine, void *stream);

/*
 * dt_sync_status — wait for `stream`, then report a device-side failure
 * raised by work enqueued since the previous dt_sync_status: DT_ETIMEOUT if
 * a kernel gave up a bounded wait (its outputs are then incomplete), else
 * DT_OK (or DT_ECUDA if the stream itself failed).  Clears the flags.
 */
int dt_sync_status(void *stream);

/*
 * object_scores — object distance scores (§6.4): scores[j][o] = sum over
 * the descriptors of query object j of each one's Eq. 1 distance to its
 * nearest descriptor of database object o (the descriptors t with
 * object_of[t] == o).  +inf where object o has no descriptor (and query j
 * has some); 0 for a query object without descriptors.
 *
 * d_db [n][64], d_object_of [n] uint32 (ids >= n_objects are ignored),
 * d_qdesc [n_qdesc][64] with query j = rows d_qoffsets[j] .. d_qoffsets[j+1]-1
 * (device int64 [nq+1], from 0 to n_qdesc, non-decreasing), d_scores
 * [nq][n_objects] FP64.  Every pair is compared (tensor cores, exact
 * integer keys); each per-object minimum becomes key / (P Z) in FP64 and
 * the sums are taken in FP64.  Reads the offsets to the host and
 * synchronises the stream.  Scratch: a copy of the database grouped by
 * object (n * 512 bytes) plus about 1 GiB.
 * Errors: DT_EINVAL, DT_ENOMEM, DT_ECUDA.
 */
int object_scores(const uint64_t *d_db, int64_t n, const uint32_t *d_object_of, int32_t n_objects,
                  const uint64_t *d_qdesc, const int64_t *d_qoffsets, int32_t nq, int64_t n_qdesc,
                  double *d_scores, void *stream);

/*
 * dt_autotune — pick launch shapes by timing them on the caller's data.
 * The paper has no counterpart; results never depend on the shapes, only
 * speed.  With `index`, the per-query traversal's threads per block and
 * resident blocks per SM, and the batched traversal's database splits and
 * database widening (inside the scan kernel, or once beforehand into
 * scratch) are tuned for (index->n, nq, k); with `d_db`, the database
 * split counts of both brute-force paths and the tensor path's widening
 * are tuned for (n, nq, k).  The winners go into a process-wide table keyed
 * by (kind, log2 n, log2 nq, k, SM count) that later calls of the same
 * shape use.  Runs each candidate twice (synchronises the stream).
 * `report` (nullable, host) receives the chosen shapes and their times.
 * Errors: DT_EINVAL, DT_ENOMEM, DT_ECUDA.
 */
typedef struct {
    int32_t tree_threads, tree_blocks_per_sm;
    int32_t popc_splits, tc_splits;
    float tree_ms, popc_ms, tc_ms;
    int32_t candidates_timed;
    int32_t tc_prewiden;              /* 1: widened in the kernel, 2: beforehand */
    int32_t tree_tc_splits, tree_tc_prewiden;
    float tree_tc_ms;
    int32_t retrieve_engine, retrieve_blocks_per_sm;
    float retrieve_ms;
} dt_tune_report;
int dt_autotune(const dt_index *index, const uint64_t *d_db, int64_t n, const uint64_t *d_q,
                int64_t nq, int32_t k, void *stream, dt_tune_report *report);

/*
 * dt_autotune_retrieve — pick how retrieve_objects finds the nearest
 * neighbours by timing, on the caller's partial queries (the arguments as
 * in retrieve_objects; a sample of the real workload is enough), every
 * engine — for engine 1 also its resident blocks per SM, for engines 2 and
 * 3 the launch of their batched search at this batch size (as dt_autotune)
 * — and keeping the fastest for (index->n, threshold > 0).  Later calls of
 * retrieve_objects with engine 0 use it.  The paper has no counterpart;
 * the votes never depend on the choice.  Synchronises the stream.
 * `report` (nullable) receives retrieve_engine, retrieve_blocks_per_sm and
 * retrieve_ms (and candidates_timed).  Errors: as retrieve_objects.
 */
int dt_autotune_retrieve(const dt_index *index, const uint32_t *d_object_of_desc, int32_t n_objects,
                         const uint64_t *d_qdesc, const int64_t *d_qoffsets, int32_t nq,
                         int64_t n_qdesc, int32_t vote_threshold, void *stream,
                         dt_tune_report *report);

/* Save the tuning table to a text file / load one (returns the number of
 * entries loaded, or a negative status) / forget all entries. */
int dt_tune_save(const char *path);
int dt_tune_load(const char *path);
void dt_tune_clear(void);

/*
 * Learned proposal.  The paper has no learned component; this part proposes
 * candidates with a small trained encoder and ranks them exactly by Eq. 1,
 * so its answers are exact whenever the true neighbours are proposed, and
 * its recall is measured against dt_search / bf_search.
 *
 * Encoder: 64x64 bit image -> conv 3x3/2 (32, 64, 64 channels, ReLU) ->
 * 2x2 average pool -> fc 1024->256 (ReLU) -> fc 256->128 -> unit length.
 * 351,040 FP32 parameters (enc_param_count), flat buffer order w1 b1 w2 b2
 * w3 b3 wf1 bf1 wf2 bf2, conv weights [out][in][3][3], fc weights [out][in].
 */
typedef struct dt_encoder dt_encoder;
int enc_create(uint64_t seed, dt_encoder **out);       /* He-uniform weights, zero biases */
void enc_free(dt_encoder *enc);
int64_t enc_param_count(void);
int enc_get_params(const dt_encoder *enc, float *h_params);  /* host [enc_param_count()] */
int enc_set_params(dt_encoder *enc, const float *h_params);
int enc_get_grads(const dt_encoder *enc, float *h_grads);    /* gradient of the last train step */
/* Embeddings of n descriptors into d_out_bf16 [n][128] (BF16 bits) and/or
 * d_out_f32 [n][128]; at least one output.  Stream-ordered.
 * path: 1 = FP32 arithmetic on CUDA cores (one fused kernel); 2 = tensor
 * cores, the convolutions and dense layers as GEMMs with BF16 operands and
 * FP32 accumulation (agrees with path 1 to about 1e-2); 0 = 2 for
 * n >= 4096, else 1.  The inverted file uses path 0. */
int enc_embed(const dt_encoder *enc, const uint64_t *d_bits, int64_t n, uint16_t *d_out_bf16,
              float *d_out_f32, int32_t path, void *stream);
/* One step of InfoNCE with in-batch negatives on B (query, target) pairs,
 * L = mean_i [ log sum_j exp(<e_qi, e_tj>/tau) - <e_qi, e_ti>/tau ], then Adam
 * (beta 0.9 / 0.999, eps 1e-8) with learning rate lr unless update = 0.
 * h_loss: nullable host float receiving L (synchronises).  2 <= B <= 4096. */
int enc_train_step(dt_encoder *enc, const uint64_t *d_q, const uint64_t *d_t, int32_t B, float lr,
                   float tau, int32_t update, float *h_loss, void *stream);

/* Inverted file over the encoder's embeddings of a database: k-means with
 * n_lists cosine centroids (iters Lloyd iterations from evenly spaced
 * seeds), the database copied list by list.  The centroid sums are exact
 * fixed-point integers, so the same encoder and database give the same
 * lists on every run.  n < 2^32.  Synchronises `stream`. */
typedef struct dt_ivf dt_ivf;
int ivf_build(const dt_encoder *enc, const uint64_t *d_db, int64_t n, int32_t n_lists,
              int32_t iters, void *stream, dt_ivf **out);
void ivf_free(dt_ivf *ivf);
int ivf_offsets(const dt_ivf *ivf, int64_t *h_offsets);      /* host [n_lists + 1] */
/* Top-k of each query among the rows of its n_probe nearest lists (by
 * embedding), ranked exactly by Eq. 1 (A*Z + B*P, ties by original index).
 * d_idx/d_score [nq][k] as in dt_search; d_scanned [nq] rows examined (nullable).
 * With n_probe = n_lists the result is the exact top-k.  n_probe <= 256.
 * path: 1 = one thread block per query scanning its lists on CUDA cores;
 * 2 = the (query, list) pairs regrouped by list, each list's rows scanned
 * once for all its queries on the tensor cores (as bf_search path 2);
 * 0 = 2 when nq * n_probe >= 10 * n_lists (about ten queries per list),
 * else 1.  Both give the same results. */
int ivf_search(const dt_ivf *ivf, const dt_encoder *enc, const uint64_t *d_q, int64_t nq, int32_t k,
               int32_t n_probe, uint32_t *d_idx, float *d_score, int64_t *d_scanned, int32_t path,
               void *stream);

/*
 * Test hooks for failure handling (the paper has no counterpart; both are
 * off by default and affect only this process).
 * dt_debug_fail_allocation(n): the n-th scratch allocation from now on
 *   reports failure (the call returns DT_ENOMEM); n <= 0 switches it off.
 * dt_debug_inject_missing_copy(on): while on, popcount brute-force
 *   launches (bf_search path 1) skip the copy of each thread block's first
 *   database tile and wait for it only a few thousand polls, so the bounded
 *   wait gives up: the results are void and dt_sync_status returns
 *   DT_ETIMEOUT.  Nothing faults, and later calls work normally.
 */
void dt_debug_fail_allocation(int32_t nth);
void dt_debug_inject_missing_copy(int32_t on);

/*
 * Kernel timing (the paper has no counterpart; for measurement).  While
 * switched on, the library records a CUDA event pair around each launch of
 * its main kernels, on the stream of the call (none during stream capture),
 * and totals their durations per kernel name:
 *   "tree_scan"   the batched tree search's scan (tensor cores)
 *   "tree_bound"  its bound pass
 *   "tc_scan"     bf_search's tensor-core scan
 *   "popc_scan"   bf_search's popcount scan
 *   "tree_warp"   the per-query tree traversal
 *   "prewiden"    widening a database into FP8 stage images
 * dt_kernel_timing(on) clears the totals and switches timing on (1) or off
 * (0).  dt_kernel_time(name, &ms, &launches) waits for the recorded events
 * of that kernel and returns their total time in milliseconds and the
 * number of launches (0 and 0 for a name never recorded).
 * Errors: DT_EINVAL (null arguments), DT_ECUDA.
 */
int dt_kernel_timing(int32_t on);
int dt_kernel_time(const char *name, double *ms, int64_t *launches);

/* Release an index (NULL is allowed).  Synchronises the device it lives on. */
void dt_free(dt_index *index);

/* Static name of a status code. */
const char *dt_status_string(int status);

/* Message for the last failing call in this thread ("" if none). */
const char *dt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DT_H */
