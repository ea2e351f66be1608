/*
 * oracle.c — plain CPU oracle for the weighted-Hamming search path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header or table with the CUDA library.
 *
 * Written for clarity, not speed: single descriptors are handled one at a
 * time, bits one at a time where the definition is per bit, FP64 for every
 * real-valued quantity.  Each function names the passage of the paper
 * (arXiv 2107.03368, "Partial 3D Object Retrieval using Local Binary QUICCI
 * Descriptors and Dissimilarity Tree Indexing") that it follows.
 *
 * Readings of the paper taken here (the paper is silent, garbled or
 * inconsistent at these points):
 *   R1  Eq. 1's type-B denominator is max(N*N - |q|, 1): N*N bits can be of
 *       type B at most (the text normalises by the errors that can occur).
 *   R2  The node bound of §4.2 is used in Eq. 1's units with Eq. 1's guards:
 *       scaled by P*Z it is popc(q & ~OR) * Z (+ popc(~q & AND) * P).
 *   R3  The split loop of §4.1 stops right after the first bit (in ascending
 *       popularity order, ties by bit index) whose move makes the dissimilar
 *       set hold at least ceil(n/2) descriptors ("roughly equal" halves).
 *   R4  If a split leaves either side empty, the node's list (ascending
 *       original index) is cut by position: first floor(n/2) similar.
 *   R5  A node is a leaf iff it holds at most leaf_size descriptors.
 *   R5b Every node, leaves included, carries its OR (sum) image; the AND
 *       (product) image is computed and used only when asked for.
 *   R5c Nodes are numbered breadth first, the similar child before the
 *       dissimilar one; each node's descriptors occupy a contiguous segment
 *       of the permutation, similar part first, ascending original index.
 *   R6  Best-first search runs while the queue is non-empty and the smallest
 *       open bound does not exceed the current k-th result.
 *   R7  A child is pruned only if its bound is strictly greater than the
 *       k-th result, so equal-distance lower-index results are never lost.
 *   R8  Results are ordered by (distance, original index) ascending.
 *   R10 "At random" in the voting loop of §3 is a Fisher-Yates permutation
 *       driven by SplitMix64; a vote goes to the object of the top-1 result.
 *   R15 QUICCI geometry (§2.2 describes it in words only): the oriented
 *       point p with unit normal n (normalised here; a zero normal gives an
 *       empty descriptor) is the axis of N = 64 layers and N circles per
 *       layer.  Layer l (word l, bottom = 0) is the plane at height
 *       z_l = -R + (2l + 1) R / N along n, so the layers evenly fill
 *       [-R, R] around p; circle c (bit c) has radius r_c = (c + 1) R / N,
 *       so the largest is the support radius R; the circle one step smaller
 *       than c = 0 has radius 0 and meets nothing.  A circle's
 *       intersection count is the number of points where it meets the
 *       mesh's triangles; a layer plane cuts a triangle in a segment when
 *       some vertex lies below it (height < z_l) and some not.  Bit (l, c)
 *       is set iff the count of circle c differs from that of circle c-1;
 *       the modified QUICCI of §5 sets it only if the two differ by 2 or
 *       more.
 *   R14 Incremental insertion, which §4.1 only suggests (redo the part of
 *       the tree that new descriptors touch): a batch of new descriptors
 *       takes indices n .. n+m-1; each descends, against the tree as it was before the batch, into the
 *       child whose images it would widen least (bits set in it but not in
 *       OR, plus bits clear in it but set in AND when AND images are kept;
 *       the similar child on ties) — the least-enlargement rule of R-tree
 *       insertion (Guttman, 1984); it joins that leaf after the leaf's old
 *       descriptors; images become those of the enlarged sets; a leaf left
 *       over leaf_size is rebuilt by §4.1 as a subtree root, new nodes
 *       numbered from the old node count on, generation by generation.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OW 64          /* 64 words of 64 bits: a 64x64-bit QUICCI image (§6) */
#define OBITS 4096

/* ------------------------------------------------------------------------ */
/* Bits                                                                      */
/* ------------------------------------------------------------------------ */

static int get_bit(const uint64_t *d, int b)
{
    return (int)((d[b >> 6] >> (b & 63)) & 1u);
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 (§2.3): weighted Hamming distance                                   */
/* ------------------------------------------------------------------------ */

/*
 * Eq. 1 for an N x N binary image given one byte per bit (row-major).
 * Type A error: query bit 1, target bit 0.  Type B: query 0, target 1.
 * delta = A / max(|q|, 1) + B / max(N*N - |q|, 1)   (reading R1).
 */
double orc_wh_bytes(const uint8_t *q, const uint8_t *t, int N, int32_t *A_out, int32_t *B_out)
{
    int sq = 0, a = 0, b = 0;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            int qb = q[r * N + c] ? 1 : 0, tb = t[r * N + c] ? 1 : 0;
            sq += qb;
            a += qb * (1 - tb);
            b += (1 - qb) * tb;
        }
    double P = sq > 1 ? (double)sq : 1.0;
    double Z = (N * N - sq) > 1 ? (double)(N * N - sq) : 1.0;
    if (A_out) *A_out = a;
    if (B_out) *B_out = b;
    return (double)a / P + (double)b / Z;
}

/* Eq. 1 on a packed 64x64 descriptor, one bit at a time. */
double orc_wh_bitwise(const uint64_t *q, const uint64_t *t, int32_t *A_out, int32_t *B_out)
{
    int sq = 0, a = 0, b = 0;
    for (int i = 0; i < OBITS; ++i) {
        int qb = get_bit(q, i), tb = get_bit(t, i);
        sq += qb;
        a += qb & (1 - tb);
        b += (1 - qb) & tb;
    }
    double P = sq > 1 ? (double)sq : 1.0;
    double Z = (OBITS - sq) > 1 ? (double)(OBITS - sq) : 1.0;
    if (A_out) *A_out = a;
    if (B_out) *B_out = b;
    return (double)a / P + (double)b / Z;
}

/*
 * The type A and type B error counts of Eq. 1 on packed words: A counts the
 * positions set in q and clear in t, B the positions clear in q and set in t
 * (a library popcount counts the bits of each masked word).
 */
static void error_counts(const uint64_t *q, const uint64_t *t, int *a, int *b)
{
    int sa = 0, sb = 0;
    for (int w = 0; w < OW; ++w) {
        sa += __builtin_popcountll(q[w] & ~t[w]);
        sb += __builtin_popcountll(~q[w] & t[w]);
    }
    *a = sa;
    *b = sb;
}

/* Same value as orc_wh_bitwise, word at a time (used for the large scans). */
double orc_wh(const uint64_t *q, const uint64_t *t, int32_t *A_out, int32_t *B_out)
{
    int sq = 0, a, b;
    for (int w = 0; w < OW; ++w) sq += __builtin_popcountll(q[w]);
    error_counts(q, t, &a, &b);
    double P = sq > 1 ? (double)sq : 1.0;
    double Z = (OBITS - sq) > 1 ? (double)(OBITS - sq) : 1.0;
    if (A_out) *A_out = a;
    if (B_out) *B_out = b;
    return (double)a / P + (double)b / Z;
}

/* ------------------------------------------------------------------------ */
/* Ranked result lists (reading R8)                                          */
/* ------------------------------------------------------------------------ */

/*
 * For one query, P = max(|q|,1) and Z = max(4096-|q|,1) are fixed, so
 * comparing two Eq. 1 values a1/P + b1/Z and a2/P + b2/Z exactly is the same
 * as comparing a1*Z + b1*P and a2*Z + b2*P (both sides multiplied by P*Z>0).
 * The oracle compares these exact integers, never the rounded doubles.
 */
typedef struct { int64_t num; int64_t idx; int32_t a, b; } result_t;

static int res_less(const result_t *x, const result_t *y)
{
    if (x->num != y->num) return x->num < y->num;
    return x->idx < y->idx;
}

/* Insert r into the sorted list res[0..*len) capped at k entries. */
static void res_insert(result_t *res, int *len, int k, result_t r)
{
    if (*len == k && !res_less(&r, &res[k - 1])) return;
    int i = (*len < k) ? (*len)++ : k - 1;
    while (i > 0 && res_less(&r, &res[i - 1])) {
        res[i] = res[i - 1];
        --i;
    }
    res[i] = r;
}

static void res_write(const result_t *res, int len, int k, int64_t P, int64_t Z,
                      int64_t *idx, double *score, int32_t *ab)
{
    for (int j = 0; j < k; ++j) {
        if (j < len) {
            idx[j] = res[j].idx;
            score[j] = (double)res[j].a / (double)P + (double)res[j].b / (double)Z;
            if (ab) { ab[2 * j] = res[j].a; ab[2 * j + 1] = res[j].b; }
        } else {           /* fewer than k descriptors exist */
            idx[j] = -1;
            score[j] = INFINITY;
            if (ab) { ab[2 * j] = -1; ab[2 * j + 1] = -1; }
        }
    }
}

static void query_weights(const uint64_t *q, int64_t *P, int64_t *Z)
{
    int sq = 0;
    for (int w = 0; w < OW; ++w) sq += __builtin_popcountll(q[w]);
    *P = sq > 1 ? sq : 1;
    *Z = (OBITS - sq) > 1 ? (OBITS - sq) : 1;
}

/* ------------------------------------------------------------------------ */
/* Sequential search (§6.2): every database descriptor against the query    */
/* ------------------------------------------------------------------------ */

/*
 * For each of nq queries, the k database descriptors with the smallest Eq. 1
 * distance, ties by lowest index.  Outputs idx[nq][k] (-1 past n), score
 * [nq][k] (FP64 Eq. 1, +inf past n), ab[nq][k][2] = (A, B) (nullable).
 */
void orc_bf_topk(const uint64_t *db, int64_t n, const uint64_t *qs, int64_t nq, int32_t k,
                 int64_t *idx, double *score, int32_t *ab, int32_t nthreads)
{
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
        const uint64_t *q = qs + qi * OW;
        int64_t P, Z;
        query_weights(q, &P, &Z);
        result_t *res = (result_t *)malloc(sizeof(result_t) * (size_t)k);
        int len = 0;
        for (int64_t i = 0; i < n; ++i) {
            int a, b;
            error_counts(q, db + i * OW, &a, &b);
            result_t r = { (int64_t)a * Z + (int64_t)b * P, i, a, b };
            res_insert(res, &len, k, r);
        }
        res_write(res, len, k, P, Z, idx + qi * k, score + qi * k, ab ? ab + qi * k * 2 : NULL);
        free(res);
    }
}

/* ------------------------------------------------------------------------ */
/* Dissimilarity Tree construction (§4.1, construction listing)             */
/* ------------------------------------------------------------------------ */

/*
 * Flattened tree written by both builders (reading R5c):
 *   child[2*i], child[2*i+1]  similar / dissimilar child of node i, -1 at a leaf
 *   begin[i], count[i]        node i's segment of perm
 *   level[i]                  depth of node i (root 0)
 *   or_img[i*64..]            OR (sum) image of node i's descriptors
 *   and_img[i*64..]           AND (product) image (nullable)
 *   perm[n]                   tree position -> original index
 * Capacities: nodes <= 2n-1 (n >= 1).  Returns the node count.
 */
typedef struct {
    int64_t *child, *begin, *count;
    int32_t *level;
    uint64_t *or_img, *and_img;
    int64_t *perm;
} orc_tree_out;

typedef struct { int64_t node, begin, count; int32_t level; } work_t;

typedef struct { int64_t count; int bit; } bitkey_t;

static int cmp_bitkey(const void *x, const void *y)
{
    const bitkey_t *a = (const bitkey_t *)x, *b = (const bitkey_t *)y;
    if (a->count != b->count) return a->count < b->count ? -1 : 1;
    return (a->bit > b->bit) - (a->bit < b->bit);
}

/* Split rule of the literal listing: returns the number of similar
 * descriptors and reorders list[0..n) as similar then dissimilar, each part
 * keeping ascending original index. */
static int64_t split_literal(const uint64_t *db, int64_t *list, int64_t n)
{
    /* popularity of every bit over the node's descriptors (§4.1) */
    int64_t *counts = (int64_t *)calloc(OBITS, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int b = 0; b < OBITS; ++b)
            counts[b] += get_bit(db + list[i] * OW, b);
    /* bitOrder: ascending popularity, ties by bit index (reading R3) */
    bitkey_t *order = (bitkey_t *)malloc(sizeof(bitkey_t) * OBITS);
    for (int b = 0; b < OBITS; ++b) order[b] = (bitkey_t){ counts[b], b };
    qsort(order, OBITS, sizeof(bitkey_t), cmp_bitkey);
    /* move every similar descriptor with the current bit set, bit by bit,
     * until the dissimilar set holds at least ceil(n/2) (reading R3) */
    char *in_similar = (char *)malloc((size_t)n);
    memset(in_similar, 1, (size_t)n);
    int64_t n_dis = 0, target = (n + 1) / 2;
    for (int r = 0; r < OBITS && n_dis < target; ++r) {
        int b = order[r].bit;
        for (int64_t i = 0; i < n; ++i)
            if (in_similar[i] && get_bit(db + list[i] * OW, b)) {
                in_similar[i] = 0;
                ++n_dis;
            }
    }
    int64_t n_sim = n - n_dis;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t s = 0, d = n_sim;
    if (n_sim == 0 || n_dis == 0) {            /* reading R4 */
        n_sim = n / 2;
        memcpy(tmp, list, sizeof(int64_t) * (size_t)n);
    } else {
        for (int64_t i = 0; i < n; ++i) {
            if (in_similar[i]) tmp[s++] = list[i];
            else tmp[d++] = list[i];
        }
    }
    memcpy(list, tmp, sizeof(int64_t) * (size_t)n);
    free(tmp);
    free(in_similar);
    free(order);
    free(counts);
    return n_sim;
}

static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return a < b ? -1 : a > b;
}

/*
 * The same split in closed form.  Give bit b the key (popularity(b), b); the
 * position of b in bitOrder is the rank of its key.  After the listing has
 * processed the first r+1 bits of bitOrder, the dissimilar set is exactly
 * the descriptors whose smallest set-bit key is at most the key of bit r.
 * So the loop stops at the ceil(n/2)-th smallest of these per-descriptor
 * minima, K*, and dissimilar = {d : minkey(d) <= K*} (all non-empty
 * descriptors if fewer than ceil(n/2) exist).  Counting only the set bits
 * makes it fast enough for millions of descriptors.
 */
/* Large nodes (a level with fewer nodes than threads) also spread their
 * per-descriptor loops over threads; both loops are independent per
 * descriptor (the counts are summed, the minima written per descriptor). */
#define ORC_PAR_MIN 200000

static int64_t split_minrank(const uint64_t *db, int64_t *list, int64_t n)
{
    int64_t *counts = (int64_t *)calloc(OBITS, sizeof(int64_t));
#pragma omp parallel for reduction(+ : counts[:OBITS]) if (n >= ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t *d = db + list[i] * OW;
        for (int w = 0; w < OW; ++w) {
            uint64_t x = d[w];
            while (x) {
                counts[w * 64 + __builtin_ctzll(x)]++;
                x &= x - 1;
            }
        }
    }
    const uint64_t NONE = UINT64_MAX;
    uint64_t *mk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t *sorted = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
#pragma omp parallel for if (n >= ORC_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t *d = db + list[i] * OW;
        uint64_t m = NONE;
        for (int w = 0; w < OW; ++w) {
            uint64_t x = d[w];
            while (x) {
                int b = w * 64 + __builtin_ctzll(x);
                uint64_t key = ((uint64_t)counts[b] << 12) | (uint64_t)b;
                if (key < m) m = key;
                x &= x - 1;
            }
        }
        mk[i] = sorted[i] = m;
    }
    qsort(sorted, (size_t)n, sizeof(uint64_t), cmp_u64);
    int64_t target = (n + 1) / 2;
    int64_t n_finite = 0;
    while (n_finite < n && sorted[n_finite] != NONE) ++n_finite;
    uint64_t kstar = n_finite >= target ? sorted[target - 1]
                   : (n_finite > 0 ? sorted[n_finite - 1] : 0);
    int64_t n_dis = 0;
    for (int64_t i = 0; i < n; ++i)
        if (mk[i] != NONE && mk[i] <= kstar) ++n_dis;
    int64_t n_sim = n - n_dis;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (n_sim == 0 || n_dis == 0) {            /* reading R4 */
        n_sim = n / 2;
    } else {
        int64_t s = 0, d = n_sim;
        for (int64_t i = 0; i < n; ++i) {
            if (mk[i] != NONE && mk[i] <= kstar) tmp[d++] = list[i];
            else tmp[s++] = list[i];
        }
        memcpy(list, tmp, sizeof(int64_t) * (size_t)n);
    }
    free(tmp);
    free(sorted);
    free(mk);
    free(counts);
    return n_sim;
}

static void node_images(const uint64_t *db, const int64_t *list, int64_t n,
                        uint64_t *or_img, uint64_t *and_img)
{
    for (int w = 0; w < OW; ++w) {
        uint64_t o = 0, a = n > 0 ? ~0ULL : 0;
        for (int64_t i = 0; i < n; ++i) {
            o |= db[list[i] * OW + w];
            a &= db[list[i] * OW + w];
        }
        or_img[w] = o;
        if (and_img) and_img[w] = a;
    }
}

/*
 * Splits the nodes of the work list cur[0..m) and all their descendants, one
 * generation at a time: a node with more than leaf_size descriptors is split
 * (closed form or literal move loop) and its two children are numbered from
 * next_id on, in the order of their parents, similar child first; every
 * processed node gets its segment, level and images.  The nodes of a
 * generation own disjoint segments of perm, so they are split independently
 * (OpenMP threads over the generation's nodes).  Returns the next free id.
 */
static int64_t grow(const uint64_t *db, int64_t *perm, work_t *cur, int64_t m, int64_t next_id,
                    int64_t cap, int32_t leaf_size, int32_t literal, int32_t nthreads,
                    int64_t *child, int64_t *begin, int64_t *count, int32_t *level,
                    uint64_t *or_img, uint64_t *and_img)
{
    work_t *next = (work_t *)malloc(sizeof(work_t) * (size_t)(cap + 1));
    int64_t *n_sim = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cap + 1));
    int nt = nthreads > 0 ? nthreads : 1;
    while (m > 0) {
        /* few nodes: one at a time, each using all threads inside */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) if (m >= nt)
        for (int64_t i = 0; i < m; ++i) {
            work_t w = cur[i];
            int64_t *list = perm + w.begin;
            begin[w.node] = w.begin;
            count[w.node] = w.count;
            level[w.node] = w.level;
            node_images(db, list, w.count, or_img + w.node * OW,
                        and_img ? and_img + w.node * OW : NULL);
            if (w.count <= leaf_size) {        /* reading R5 */
                n_sim[i] = -1;
                continue;
            }
            n_sim[i] = literal ? split_literal(db, list, w.count)
                               : split_minrank(db, list, w.count);
        }
        int64_t m2 = 0;
        for (int64_t i = 0; i < m; ++i) {
            work_t w = cur[i];
            if (n_sim[i] < 0) {
                child[2 * w.node] = child[2 * w.node + 1] = -1;
                continue;
            }
            int64_t s = next_id++, d = next_id++;
            child[2 * w.node] = s;
            child[2 * w.node + 1] = d;
            next[m2++] = (work_t){ s, w.begin, n_sim[i], w.level + 1 };
            next[m2++] = (work_t){ d, w.begin + n_sim[i], w.count - n_sim[i], w.level + 1 };
        }
        memcpy(cur, next, sizeof(work_t) * (size_t)m2);
        m = m2;
    }
    free(n_sim);
    free(next);
    return next_id;
}

/*
 * Builds the tree one level at a time (breadth first) from the root; the
 * recursion of the listing visits the same nodes with the same splits, only
 * in another order.  literal != 0 selects the bit-by-bit move loop, else the
 * closed form.  Returns the node count.
 */
int64_t orc_build(const uint64_t *db, int64_t n, int32_t leaf_size, int32_t literal,
                  int32_t nthreads, int64_t *child, int64_t *begin, int64_t *count,
                  int32_t *level, uint64_t *or_img, uint64_t *and_img, int64_t *perm)
{
    if (n <= 0) return 0;
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    work_t *cur = (work_t *)malloc(sizeof(work_t) * (size_t)(n + 1));
    cur[0] = (work_t){ 0, 0, n, 0 };
    int64_t n_nodes = grow(db, perm, cur, 1, 1, n, leaf_size, literal, nthreads,
                           child, begin, count, level, or_img, and_img);
    free(cur);
    return n_nodes;
}

/* ------------------------------------------------------------------------ */
/* Incremental insertion (§4.1, reading R14)                                 */
/* ------------------------------------------------------------------------ */

/* How much a node's images would widen if descriptor d joined it. */
static int64_t growth(const uint64_t *d, const uint64_t *or_img, const uint64_t *and_img)
{
    int64_t g = 0;
    for (int i = 0; i < OBITS; ++i) {
        int db = get_bit(d, i);
        if (db && !get_bit(or_img, i)) ++g;
        if (and_img && !db && get_bit(and_img, i)) ++g;
    }
    return g;
}

/*
 * Inserts descriptors n_old .. n_old+m-1 of db into a tree over descriptors
 * 0 .. n_old-1 with n_nodes nodes (arrays as orc_build returns them, with
 * room for n_nodes + 2 * (n_old + m) nodes and n_old + m perm entries).
 *   1. every new descriptor descends from the root, against the tree as it
 *      was before the batch, into the child whose images it widens least,
 *      the similar child on ties, down to a leaf;
 *   2. each leaf's segment becomes its old descriptors followed by those
 *      routed to it in ascending index; leaves keep their order in perm and
 *      every node's segment is the union of its leaves' segments;
 *   3. every node's images are those of its new segment;
 *   4. every leaf that now holds more than leaf_size descriptors, in
 *      ascending id, is split again by the construction of §4.1 as the root
 *      of a subtree; the new nodes get ids from n_nodes on, one generation at
 *      a time over all those subtrees.
 * Returns the new node count.
 */
int64_t orc_insert(const uint64_t *db, int64_t n_old, int64_t m, int32_t leaf_size, int32_t nthreads,
                   int64_t n_nodes, int64_t *child, int64_t *begin, int64_t *count,
                   int32_t *level, uint64_t *or_img, uint64_t *and_img, int64_t *perm)
{
    if (m <= 0) return n_nodes;
    const int64_t n = n_old + m;
    /* 1. routing */
    int64_t *leaf_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    for (int64_t j = 0; j < m; ++j) {
        const uint64_t *d = db + (n_old + j) * OW;
        int64_t v = 0;
        while (child[2 * v] >= 0) {
            int64_t s = child[2 * v], t = child[2 * v + 1];
            int64_t gs = growth(d, or_img + s * OW, and_img ? and_img + s * OW : NULL);
            int64_t gt = growth(d, or_img + t * OW, and_img ? and_img + t * OW : NULL);
            v = gs <= gt ? s : t;
        }
        leaf_of[j] = v;
    }
    /* 2. new segments: walk the leaves in perm order (depth first, similar
     * child first), appending each leaf's new descriptors after its old ones */
    int64_t *routed = (int64_t *)calloc((size_t)n_nodes + 1, sizeof(int64_t));
    for (int64_t j = 0; j < m; ++j) routed[leaf_of[j] + 1]++;
    for (int64_t v = 0; v < n_nodes; ++v) routed[v + 1] += routed[v];
    int64_t *bucket = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int64_t *fill = (int64_t *)calloc((size_t)n_nodes, sizeof(int64_t));
    for (int64_t j = 0; j < m; ++j) bucket[routed[leaf_of[j]] + fill[leaf_of[j]]++] = n_old + j;
    int64_t *old_perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_old);
    memcpy(old_perm, perm, sizeof(int64_t) * (size_t)n_old);
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_nodes + 1));
    int64_t sp = 0, pos = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int64_t v = stack[--sp];
        if (child[2 * v] >= 0) {
            stack[sp++] = child[2 * v + 1];   /* dissimilar after similar */
            stack[sp++] = child[2 * v];
            continue;
        }
        int64_t b = pos;
        for (int64_t i = 0; i < count[v]; ++i) perm[pos++] = old_perm[begin[v] + i];
        for (int64_t i = routed[v]; i < routed[v + 1]; ++i) perm[pos++] = bucket[i];
        begin[v] = b;
        count[v] = pos - b;
    }
    /* children have larger ids than their parent: fill internal nodes last
     * to first from their children */
    for (int64_t v = n_nodes - 1; v >= 0; --v)
        if (child[2 * v] >= 0) {
            begin[v] = begin[child[2 * v]];
            count[v] = count[child[2 * v]] + count[child[2 * v + 1]];
        }
    /* 3. images of the enlarged sets */
    for (int64_t v = 0; v < n_nodes; ++v)
        node_images(db, perm + begin[v], count[v], or_img + v * OW, and_img ? and_img + v * OW : NULL);
    /* 4. overfull leaves become roots of rebuilt subtrees */
    work_t *cur = (work_t *)malloc(sizeof(work_t) * (size_t)(n + 1));
    int64_t n_roots = 0;
    for (int64_t v = 0; v < n_nodes; ++v)
        if (child[2 * v] < 0 && count[v] > leaf_size)
            cur[n_roots++] = (work_t){ v, begin[v], count[v], level[v] };
    int64_t total = grow(db, perm, cur, n_roots, n_nodes, n, leaf_size, 0, nthreads,
                         child, begin, count, level, or_img, and_img);
    free(cur);
    free(stack);
    free(old_perm);
    free(fill);
    free(bucket);
    free(routed);
    free(leaf_of);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Dissimilarity Tree query (§4.2, query listing)                            */
/* ------------------------------------------------------------------------ */

/*
 * Lower bound of Eq. 1 (times P*Z) over every descriptor below a node
 * (§4.2, reading R2): a query bit that is 0 in the node's OR image is a type
 * A error for every descriptor below; a query 0 bit set in the AND image is
 * a type B error for all of them.
 */
static int64_t node_bound(const uint64_t *q, const uint64_t *or_img, const uint64_t *and_img,
                          int64_t P, int64_t Z)
{
    int64_t a = 0, b = 0;
    for (int i = 0; i < OBITS; ++i) {
        int qb = get_bit(q, i);
        if (qb && !get_bit(or_img, i)) ++a;
        if (and_img && !qb && get_bit(and_img, i)) ++b;
    }
    return a * Z + b * P;
}

int64_t orc_node_bound(const uint64_t *q, const uint64_t *or_img, const uint64_t *and_img)
{
    int64_t P, Z;
    query_weights(q, &P, &Z);
    return node_bound(q, or_img, and_img, P, Z);
}

typedef struct { int64_t bound, node; } open_t;

static int open_less(const open_t *x, const open_t *y)
{
    if (x->bound != y->bound) return x->bound < y->bound;
    return x->node < y->node;
}

/* binary min-heap of open nodes */
static void heap_push(open_t *h, int64_t *len, open_t v)
{
    int64_t i = (*len)++;
    h[i] = v;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!open_less(&h[i], &h[p])) break;
        open_t t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static open_t heap_pop(open_t *h, int64_t *len)
{
    open_t top = h[0];
    h[0] = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *len && open_less(&h[l], &h[m])) m = l;
        if (r < *len && open_less(&h[r], &h[m])) m = r;
        if (m == i) break;
        open_t t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return top;
}

/*
 * Best-first search for the k nearest descriptors (readings R6-R8).
 * stats[nq][4] (nullable) = nodes popped, leaves scanned, descriptors
 * scanned, bounds evaluated.
 */
void orc_tree_search(const uint64_t *db, int64_t n_nodes, const int64_t *child,
                     const int64_t *begin, const int64_t *count, const uint64_t *or_img,
                     const uint64_t *and_img, const int64_t *perm, const uint64_t *qs, int64_t nq,
                     int32_t k, int64_t *idx, double *score, int32_t *ab, int64_t *stats,
                     int32_t nthreads)
{
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
        const uint64_t *q = qs + qi * OW;
        int64_t P, Z;
        query_weights(q, &P, &Z);
        result_t *res = (result_t *)malloc(sizeof(result_t) * (size_t)k);
        int len = 0;
        open_t *heap = (open_t *)malloc(sizeof(open_t) * (size_t)(n_nodes + 1));
        int64_t hlen = 0, popped = 0, leaves = 0, scanned = 0, bounds = 0;
        if (n_nodes > 0) {
            heap_push(heap, &hlen, (open_t){ node_bound(q, or_img, and_img, P, Z), 0 });
            ++bounds;
        }
        while (hlen > 0) {
            int64_t worst = len < k ? INT64_MAX : res[k - 1].num;
            if (heap[0].bound > worst) break;  /* reading R6 */
            open_t cur = heap_pop(heap, &hlen);
            ++popped;
            int64_t nd = cur.node;
            if (child[2 * nd] < 0) {           /* leaf: exact distances */
                ++leaves;
                for (int64_t j = 0; j < count[nd]; ++j) {
                    int64_t orig = perm[begin[nd] + j];
                    int a, b;
                    error_counts(q, db + orig * OW, &a, &b);
                    result_t r = { (int64_t)a * Z + (int64_t)b * P, orig, a, b };
                    res_insert(res, &len, k, r);
                    ++scanned;
                }
            } else {
                for (int c = 0; c < 2; ++c) {
                    int64_t ch = child[2 * nd + c];
                    int64_t lb = node_bound(q, or_img + ch * OW,
                                            and_img ? and_img + ch * OW : NULL, P, Z);
                    ++bounds;
                    int64_t w2 = len < k ? INT64_MAX : res[k - 1].num;
                    if (lb <= w2) heap_push(heap, &hlen, (open_t){ lb, ch });  /* R7 */
                }
            }
        }
        res_write(res, len, k, P, Z, idx + qi * k, score + qi * k, ab ? ab + qi * k * 2 : NULL);
        if (stats) {
            stats[qi * 4 + 0] = popped;
            stats[qi * 4 + 1] = leaves;
            stats[qi * 4 + 2] = scanned;
            stats[qi * 4 + 3] = bounds;
        }
        free(heap);
        free(res);
    }
}

/* ------------------------------------------------------------------------ */
/* Voting pipeline (§3)                                                      */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood 2014): state += gamma, then mix. */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/*
 * The random order in which query j's n descriptors are drawn (reading R10):
 * the generator is SplitMix64 seeded with the (j+1)-th output of SplitMix64
 * seeded with `seed`; Fisher-Yates (Durstenfeld) from the last position down,
 * swapping position i with position (draw mod (i+1)).
 */
void orc_permutation(uint64_t seed, int64_t j, int64_t n, int64_t *out)
{
    uint64_t s0 = seed + (uint64_t)j * 0x9e3779b97f4a7c15ULL;
    uint64_t state = orc_splitmix64_next(&s0);
    for (int64_t i = 0; i < n; ++i) out[i] = i;
    for (int64_t i = n - 1; i > 0; --i) {
        uint64_t r = orc_splitmix64_next(&state) % (uint64_t)(i + 1);
        int64_t t = out[i]; out[i] = out[(int64_t)r]; out[(int64_t)r] = t;
    }
}

/*
 * Partial-object retrieval (§3): for query j, draw its descriptors in the
 * random order above, find each one's nearest database descriptor (top-1 by
 * sequential search), vote for that descriptor's object, and stop when an
 * object reaches `threshold` votes (threshold 0: use every descriptor).
 * The winner is the first object to reach the threshold, else the object
 * with most votes (lowest id on ties), -1 when no vote was cast.
 * votes[nq][n_objects] = the votes cast, consumed[nq] = descriptors used.
 */
void orc_retrieve(const uint64_t *db, int64_t n, const uint32_t *object_of, int32_t n_objects,
                  const uint64_t *qdesc, const int64_t *offsets, int32_t nq, int32_t threshold,
                  uint64_t seed, uint32_t *votes, int32_t *winner, int64_t *consumed,
                  int32_t nthreads)
{
    for (int32_t j = 0; j < nq; ++j) {
        int64_t m = offsets[j + 1] - offsets[j];
        uint32_t *v = votes + (int64_t)j * n_objects;
        memset(v, 0, sizeof(uint32_t) * (size_t)n_objects);
        int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        int64_t *nn = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        double *sc = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
        orc_permutation(seed, j, m, order);
        /* nearest neighbour of every descriptor of the query (exact, so the
         * order in which they are computed does not matter) */
        if (m > 0)
            orc_bf_topk(db, n, qdesc + offsets[j] * OW, m, 1, nn, sc, NULL, nthreads);
        int32_t win = -1;
        int64_t used = 0;
        for (int64_t i = 0; i < m; ++i) {
            int64_t t = nn[order[i]];
            uint32_t o = object_of[t];
            ++v[o];
            ++used;
            if (threshold > 0 && v[o] == (uint32_t)threshold) {
                win = (int32_t)o;
                break;
            }
        }
        if (win < 0) {
            uint32_t best = 0;
            for (int32_t o = 0; o < n_objects; ++o)
                if (v[o] > best) { best = v[o]; win = o; }
        }
        winner[j] = win;
        consumed[j] = used;
        free(sc);
        free(nn);
        free(order);
    }
}

/* ------------------------------------------------------------------------ */
/* Object distance score (§6.4)                                              */
/* ------------------------------------------------------------------------ */

/*
 * The distance score of a (query object, complete object) pair is the sum,
 * over the descriptors of the query object, of each one's Eq. 1 distance to
 * its nearest descriptor of the complete object.  scores[j][o] for query j
 * (descriptors offsets[j] .. offsets[j+1]-1 of qdesc) and database object o
 * (the descriptors t with object_of[t] == o): +inf when object o has no
 * descriptor, 0 for a query without descriptors.  Distances in FP64 (Eq. 1
 * as A/P + B/Z); the minimum per object, then the plain sum.
 */
void orc_object_scores(const uint64_t *db, int64_t n, const uint32_t *object_of, int32_t n_objects,
                       const uint64_t *qdesc, const int64_t *offsets, int32_t nq, double *scores,
                       int32_t nthreads)
{
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int32_t j = 0; j < nq; ++j) {
        double *row = scores + (int64_t)j * n_objects;
        double *best = (double *)malloc(sizeof(double) * (size_t)(n_objects > 0 ? n_objects : 1));
        for (int32_t o = 0; o < n_objects; ++o) row[o] = 0.0;
        for (int64_t i = offsets[j]; i < offsets[j + 1]; ++i) {
            const uint64_t *q = qdesc + i * OW;
            for (int32_t o = 0; o < n_objects; ++o) best[o] = INFINITY;
            for (int64_t t = 0; t < n; ++t) {
                const uint32_t o = object_of[t];
                if (o >= (uint32_t)n_objects) continue;
                const double d = orc_wh(q, db + t * OW, NULL, NULL);
                if (d < best[o]) best[o] = d;
            }
            for (int32_t o = 0; o < n_objects; ++o) row[o] += best[o];
        }
        free(best);
    }
}

/* ------------------------------------------------------------------------ */
/* QUICCI (§2.2) and the modified QUICCI for partial queries (§5), R15      */
/* ------------------------------------------------------------------------ */

#define QN 64          /* layers and circles per layer */

/* Number of points where the circle of radius r about the axis meets the
 * segment a + t (b - a), t in [0, 1]; a and b are offsets from the axis
 * within one layer plane.  A tangent point counts once. */
static int circle_hits(const double *a, const double *b, double r)
{
    double d[3] = { b[0] - a[0], b[1] - a[1], b[2] - a[2] };
    double qa = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double qb = 2.0 * (a[0] * d[0] + a[1] * d[1] + a[2] * d[2]);
    double qc = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] - r * r;
    if (qa == 0.0) return qc == 0.0;          /* a single point */
    double disc = qb * qb - 4.0 * qa * qc;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double t1 = (-qb - sq) / (2.0 * qa), t2 = (-qb + sq) / (2.0 * qa);
    int hits = (t1 >= 0.0 && t1 <= 1.0);
    if (disc > 0.0) hits += (t2 >= 0.0 && t2 <= 1.0);
    return hits;
}

/*
 * One 64x64-bit QUICCI per oriented point (points[j], normals[j]) of the
 * mesh (vertices [nv][3], triangles [nt][3] vertex ids), support radius R;
 * modified != 0 gives the modified QUICCI.  out [np][64]: word l = layer l,
 * bit c = circle c (reading R11).  Counts every circle's intersections with
 * every triangle in FP64.
 */
void orc_quicci(const float *vertices, int64_t nv, const int32_t *tris, int64_t nt,
                const float *points, const float *normals, int64_t np, double R,
                int32_t modified, int32_t nthreads, uint64_t *out)
{
    (void)nv;
    int nth = nthreads > 0 ? nthreads : 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
    for (int64_t j = 0; j < np; ++j) {
        uint64_t *img = out + j * OW;
        memset(img, 0, sizeof(uint64_t) * OW);
        double p[3], n[3], len = 0.0;
        for (int k = 0; k < 3; ++k) {
            p[k] = points[j * 3 + k];
            n[k] = normals[j * 3 + k];
            len += n[k] * n[k];
        }
        if (len == 0.0) continue;
        len = sqrt(len);
        for (int k = 0; k < 3; ++k) n[k] /= len;
        int64_t *cnt = (int64_t *)calloc(QN * QN, sizeof(int64_t));
        for (int64_t t = 0; t < nt; ++t) {
            double z[3], q[3][3];
            for (int i = 0; i < 3; ++i) {
                const float *v = vertices + (int64_t)tris[t * 3 + i] * 3;
                double rel[3] = { v[0] - p[0], v[1] - p[1], v[2] - p[2] };
                z[i] = rel[0] * n[0] + rel[1] * n[1] + rel[2] * n[2];
                for (int k = 0; k < 3; ++k) q[i][k] = rel[k] - z[i] * n[k];
            }
            for (int l = 0; l < QN; ++l) {
                double zl = -R + (2.0 * l + 1.0) * R / QN;
                int below[3], nb = 0;
                for (int i = 0; i < 3; ++i) nb += below[i] = z[i] < zl;
                if (nb == 0 || nb == 3) continue;
                double seg[2][3];
                int ns = 0;
                for (int e = 0; e < 3; ++e) {
                    int a = e, b = (e + 1) % 3;
                    if (below[a] == below[b]) continue;
                    double s = (zl - z[a]) / (z[b] - z[a]);
                    for (int k = 0; k < 3; ++k) seg[ns][k] = q[a][k] + s * (q[b][k] - q[a][k]);
                    ++ns;
                }
                for (int c = 0; c < QN; ++c)
                    cnt[l * QN + c] += circle_hits(seg[0], seg[1], (c + 1.0) * R / QN);
            }
        }
        for (int l = 0; l < QN; ++l)
            for (int c = 0; c < QN; ++c) {
                int64_t prev = c > 0 ? cnt[l * QN + c - 1] : 0;
                int64_t d = cnt[l * QN + c] - prev;
                int set = modified ? (d >= 2 || d <= -2) : (d != 0);
                if (set) img[l] |= 1ULL << c;
            }
        free(cnt);
    }
}
