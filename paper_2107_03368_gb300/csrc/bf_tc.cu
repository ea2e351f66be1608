// bf_tc.cu — sequential search (§6.2) with the overlap counted on the
// tensor cores.
//
// O[q][t] = popc(q & t) is the dot product of two 0/1 vectors of length
// 4096, i.e. one row of a dense Q x N x 4096 contraction.  A set bit is
// widened to the FP8 E4M3 value 2^-6 (byte 0x08, the smallest normal) and a
// clear bit to 0; tcgen05.mma (kind::f8f6f4) multiplies with FP32
// accumulation in tensor memory.  Every product is 2^-12 and a row sum is
// O * 2^-12 with O <= 4096, which FP32 holds exactly, so O = 4096 * sum is
// exact.  The epilogue turns O into the Eq. 1 key (A = |q| - O, B = |t| - O)
// and keeps per-query top-k.
//
// Kernel organisation (one persistent CTA per SM).  A work unit is one
// 128-query tile against a run of 128-descriptor database tiles, taken two
// tiles (256 rows) per step, so every MMA is 128 x 256 x 32: per byte the
// tensor cores read from shared memory it does half again the work of a
// 128 x 128 MMA, and operand reads from shared memory are what bound the
// tensor pipe here.  Units come in pairs of query tiles (split mode: the
// pair's tiles scan the same database split on neighbouring CTAs, which
// share the database chunks in L2).  Per 128-bit K chunk a 48 KB stage
// holds the chunk of the query tile and of both database tiles, 128-byte
// swizzled:
//   * database chunks come either pre-widened (one copy of the database as
//     E4M3 stage images, made once per call; a single thread brings each
//     stage in with bulk copies, TMA engine) or are widened in the kernel
//     by 8 producer warps, one database row of the step per thread, which
//     sum |t| on the way; the query tiles are always pre-widened;
//   * one thread issues, per chunk, 4 MMAs of 128 x 256 x 32 into one of
//     two 256-column TMEM accumulators, then commits to free the stage;
//   * the epilogue warps (one thread per query row = TMEM lane, each warp a
//     group of 32-column slices) read the finished accumulator while the
//     next step is multiplied into the other one, and keep top-k.  A slice
//     is first tested as a whole: from its largest overlap and the smallest
//     |t| of its 32 rows follows a lower bound on every key in it, and when
//     that bound exceeds the query's k-th key the slice is skipped.
//     Otherwise every row's key is compared without branches and only the
//     rows that qualify are inserted.
// A four-stage mbarrier ring connects copies/producers and MMA; all waits
// are bounded and a shared abort flag makes every role leave together.
// Work units are (query tile, database split), or come from a unit table
// (list mode); per-split lists are merged afterwards.
#include <algorithm>
#include <mutex>

#include "dt_internal.cuh"
#include "tc_util.cuh"

namespace dtk {
namespace {

constexpr int TM = 128;                 // queries per tile (MMA M)
constexpr int QT = 2;                   // query tiles per unit pair
constexpr int TN = 128;                 // descriptors per database tile
constexpr int NB = 2;                   // database tiles per step
constexpr int BN = NB * TN;             // descriptors per step (MMA N)
constexpr int KC = 128;                 // K bytes (= bits) per chunk
constexpr int NCHUNK = kBits / KC;      // 32
constexpr int STAGES = 4;
constexpr int A_STAGE = TM * KC;        // 16 KB: the query tile's chunk
constexpr int B_STAGE = TN * KC;        // 16 KB per database tile
constexpr int STAGE = A_STAGE + NB * B_STAGE;   // 48 KB
constexpr uint32_t SBO = 8 * KC;        // next 8-row atom (1 KB)
constexpr int SLICES = BN / 32;         // 32-column slices of an accumulator
constexpr int EPI_WARPS = 8, PROD_WARPS = BN / 32;   // producers: one database row per thread
// Warp roles.  In-kernel widening: epilogue 0-7, producers 8-15, MMA 16.
// Pre-widened database (PRE): epilogue 0-15, copy issuer 16, MMA 17.
// Epilogue warp w reads TMEM lanes 32 (w % 4) .. + 31 and the slices of
// group w / 4; a query ends a unit with one sorted list per group (split
// mode), or all slices go to group 0 (list mode: one list per slot).
__host__ __device__ constexpr int epi_warps(bool pre) { return pre ? 2 * EPI_WARPS : EPI_WARPS; }
__host__ __device__ constexpr int mma_warp(bool pre) { return pre ? 17 : 16; }
__host__ __device__ constexpr int kernel_threads(bool pre) { return (mma_warp(pre) + 1) * 32; }
__host__ __device__ constexpr int lists_per_unit(bool pre) { return epi_warps(pre) / 4; }
constexpr uint32_t ACC_COLS = BN;       // one accumulator: 256 columns
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;    // double-buffered: 512
constexpr uint32_t IDESC = idesc_e4m3_f32(TM, BN);
static_assert(PROD_WARPS == 8 && TN % 32 == 0, "one producer thread per row of a step");
static_assert(SLICES % lists_per_unit(true) == 0, "slices split evenly over the groups");

struct TcCtl {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t final_bar;
    uint32_t tmem_base;
    volatile uint32_t abort;
};

constexpr size_t STAGE_BYTES = (size_t)STAGES * STAGE;
// Kernel modes: the plain sequential search (split or list mode), the scan
// pass of the batched tree search (need bitmap, K-chunk masks, caps) and
// its bound pass.  Each is its own instantiation, so the plain search
// carries none of the others' code.
enum { MODE_PLAIN = 0, MODE_TREE = 1, MODE_BOUND = 2 };

// |t| of the rows of the last tp_ring(MODE) steps: the copy issuer or the
// producers write a step's records with its last chunk and the epilogue
// reads them once the step's accumulator is full.  The copies run at most
// STAGES chunks ahead of the MMAs, which run at most one step ahead of the
// slowest epilogue warp (two accumulators).  With whole 32-chunk steps the
// next step's records can be written while the epilogue reads, the one
// after only once the epilogue is done: two entries.  With K chunks skipped
// (tree mode) a step can be a single chunk, so the records of up to
// STAGES + 1 later steps can be written meanwhile: STAGES + 2 entries.
__host__ __device__ constexpr int tp_ring(int mode) { return mode == MODE_TREE ? STAGES + 2 : 2; }
// One record per database tile, contiguous so that a single bulk copy can
// fill it: |t| of every row [TN], then the smallest |t| of each 32 rows
// [TN / 32] (uint32 throughout).  A ring entry holds the NB records of a
// step.
constexpr int SIDE_WORDS = TN + TN / 32;
constexpr uint32_t SIDE_BYTES = SIDE_WORDS * 4;          // 528
static_assert(SIDE_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
__host__ __device__ constexpr size_t smem_bytes(int mode)
{
    return STAGE_BYTES + sizeof(TcCtl) + (size_t)tp_ring(mode) * NB * SIDE_BYTES + 1024;
}

__device__ uint32_t g_tc_error;  // a bounded wait gave up (DT_ETIMEOUT)

// Bit j of each byte of w -> four E4M3 bytes, 0x08 (2^-6) where the bit is
// set: one shift moves bit j of every byte to bit 3 of that byte, one AND
// keeps it (j is a constant at every call, so two instructions a word).
__device__ __forceinline__ uint32_t bitplane_e4m3(uint32_t w, int j)
{
    return (j <= 3 ? (w << (3 - j)) : (w >> (j - 3))) & 0x08080808u;
}

// 32 bits -> 32 E4M3 bytes as two 16-byte pieces.  Output byte 4j + m holds
// bit 8m + j of w.  This reorders the K positions inside a chunk, the same
// way for queries and database, which leaves every dot product unchanged.
__device__ __forceinline__ void widen32(uint32_t w, uint4 &lo, uint4 &hi)
{
    lo = make_uint4(bitplane_e4m3(w, 0), bitplane_e4m3(w, 1), bitplane_e4m3(w, 2),
                    bitplane_e4m3(w, 3));
    hi = make_uint4(bitplane_e4m3(w, 4), bitplane_e4m3(w, 5), bitplane_e4m3(w, 6),
                    bitplane_e4m3(w, 7));
}

// Byte offset of (row, 16-byte piece j of the chunk) in a K-major stage
// with the 128-byte swizzle: row r of 128 bytes in the 1 KB atom r / 8,
// piece j at position j ^ (r % 8) of the row.  The eight rows of an atom
// written by eight threads for the same j fall in eight different bank
// groups.
__device__ __forceinline__ uint32_t core_off(int row, int j)
{
    return (uint32_t)(row >> 3) * SBO + (uint32_t)(row & 7) * KC + (uint32_t)((j ^ (row & 7)) * 16);
}

// Write 128 bits of one row as 128 E4M3 bytes into a stage.
__device__ __forceinline__ void store_row_chunk(unsigned char *stage, int row, uint4 bits)
{
    const uint32_t w[4] = {bits.x, bits.y, bits.z, bits.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint4 lo, hi;
        widen32(w[i], lo, hi);
        *reinterpret_cast<uint4 *>(stage + core_off(row, 2 * i)) = lo;
        *reinterpret_cast<uint4 *>(stage + core_off(row, 2 * i + 1)) = hi;
    }
}

// Queries -> pre-widened tiles a_exp[m_tile][chunk][16 KB stage image], plus |q|.
__global__ void widen_queries_kernel(const uint64_t *__restrict__ q, int64_t nq, int n_mtiles,
                                     unsigned char *__restrict__ a_exp, uint32_t *__restrict__ qpop)
{
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (m_tile, row, chunk)
    const int64_t total = (int64_t)n_mtiles * TM * NCHUNK;
    if (id >= total) return;
    const int c = (int)(id % NCHUNK);
    const int row = (int)((id / NCHUNK) % TM);
    const int64_t mt = id / ((int64_t)NCHUNK * TM);
    const int64_t qi = mt * TM + row;
    uint4 bits = make_uint4(0, 0, 0, 0);
    if (qi < nq) bits = __ldg(reinterpret_cast<const uint4 *>(q + qi * kWords) + c);
    store_row_chunk(a_exp + ((size_t)mt * NCHUNK + c) * A_STAGE, row, bits);
    if (qi < nq && c == 0) {
        uint32_t s = 0;
        const uint4 *r = reinterpret_cast<const uint4 *>(q + qi * kWords);
        for (int j = 0; j < 32; ++j) {
            uint4 v = __ldg(r + j);
            s += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
        qpop[qi] = s;
    }
}

// Gathered query tiles: row r of tile mt is query slot_q[mt * TM + r];
// padding rows (negative) are not written (their accumulator rows are
// never read), nor are tiles at or beyond *n_tiles (all max_tiles tiles
// when n_tiles is null).
__global__ void widen_gather_kernel(const uint64_t *__restrict__ q, const int32_t *__restrict__ slot_q,
                                    const int64_t *__restrict__ n_tiles, int64_t max_tiles,
                                    unsigned char *__restrict__ a_exp, uint32_t *__restrict__ qpop)
{
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (tile, row, chunk)
    if (id >= max_tiles * TM * NCHUNK) return;
    const int c = (int)(id % NCHUNK);
    const int row = (int)((id / NCHUNK) % TM);
    const int64_t mt = id / ((int64_t)NCHUNK * TM);
    if (n_tiles && mt >= *n_tiles) return;
    const int32_t qi = slot_q[mt * TM + row];
    if (qi < 0) return;
    const uint4 bits = __ldg(reinterpret_cast<const uint4 *>(q + (int64_t)qi * kWords) + c);
    store_row_chunk(a_exp + ((size_t)mt * NCHUNK + c) * A_STAGE, row, bits);
    if (c == 0) {
        uint32_t s = 0;
        const uint4 *r = reinterpret_cast<const uint4 *>(q + (int64_t)qi * kWords);
        for (int j = 0; j < 32; ++j) {
            uint4 v = __ldg(r + j);
            s += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
        qpop[mt * TM + row] = s;
    }
}

// |t| records of pre-widened database tiles (one CTA of TN threads per
// tile) from the per-row |t|; rows past n count 0.
__global__ void side_kernel(const uint32_t *__restrict__ rowpop, int64_t n,
                            uint32_t *__restrict__ side)
{
    const int64_t t = blockIdx.x;
    const int row = threadIdx.x, lane = row & 31, w = row >> 5;
    const int64_t i = t * TN + row;
    const uint32_t v = i < n ? rowpop[i] : 0u;
    uint32_t *e = side + t * SIDE_WORDS;
    e[row] = v;
    const uint32_t mn = __reduce_min_sync(0xffffffffu, v);
    if (lane == 0) e[TN + w] = mn;
}

// Bounded wait that also gives up when another role aborted.  The thread
// sleeps inside try_wait (up to 0.5 us per poll) instead of spinning, so
// waiting warps leave the issue slots to the working ones.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, TcCtl *ctl,
                                              uint32_t *err)
{
    for (uint32_t i = 0; i < (kSpinLimit >> 4); ++i) {     // at most ~2 s
        if (mbar_try_wait_sleep(bar, parity, 500u)) return true;
        if (ctl->abort) return false;
    }
    ctl->abort = 1u;
    atomicOr(err, 1u);
    return false;
}

// As wait_or_abort for the two single threads that feed the tensor cores
// (copy issuer, MMA issuer): they poll without sleeping, so a stage is
// refilled or multiplied as soon as its barrier completes.  Bounded by
// elapsed SM clocks (about two seconds).
__device__ __forceinline__ bool wait_spin(uint64_t *bar, uint32_t parity, TcCtl *ctl, uint32_t *err)
{
    const long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (ctl->abort) return false;
        if ((i & 255u) == 255u && clock64() - t0 > (4ll << 30)) break;
    }
    ctl->abort = 1u;
    atomicOr(err, 1u);
    return false;
}

// Bounded wait (about 2 ms of clocks) for the copies of the last issued
// stages [g - STAGES, g) to land, i.e. for their full barriers: after an
// abort no bulk copy may still write into shared memory when the CTA
// leaves.  Immediate when every issued stage was consumed.  A barrier that
// also waits for arrivals that will not come (an aborted partner or
// producer) is given up at the limit.
__device__ __forceinline__ void drain_copies(TcCtl *ctl, uint32_t g)
{
    const long long t0 = clock64();
    for (uint32_t i = g > (uint32_t)STAGES ? g - STAGES : 0u; i < g; ++i) {
        const int s = (int)(i % STAGES);
        while (!mbar_try_wait(&ctl->full[s], (i / STAGES) & 1u))
            if (clock64() - t0 > (1ll << 22)) return;
    }
}

// Warp-uniform version: lane 0 waits, the verdict is broadcast.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, TcCtl *ctl, uint32_t *err,
                                          int lane)
{
    bool ok = true;
    if (lane == 0) ok = wait_or_abort(bar, parity, ctl, err);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// The same with lane 0 polling (wait_spin): for the producer warps, whose
// next stage is on the critical path (18% faster than sleeping at 10M).
__device__ __forceinline__ bool warp_wait_spin(uint64_t *bar, uint32_t parity, TcCtl *ctl,
                                               uint32_t *err, int lane)
{
    bool ok = true;
    if (lane == 0) ok = wait_spin(bar, parity, ctl, err);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

struct TcArgs {
    const uint64_t *db;              // database rows [n][64]
    int64_t n;
    const unsigned char *a_exp;      // pre-widened query tiles
    const uint32_t *qpop;            // |q| per query-tile row
    const uint32_t *idx_map;         // row -> reported index (nullable: identity)
    int64_t nq;
    int k;
    int n_mtiles;                    // query tiles of the whole call
    int n_mpairs;                    // split mode: pairs of query tiles in this launch
    int64_t mp_base;                 // split mode: first pair of this launch
    int64_t n_ntiles;
    int64_t tiles_per_split;
    int n_split;
    // Unit table (list mode): when non-null, units[u] gives the pair of
    // query tiles 2u, 2u + 1 and the pair count is read from *n_units;
    // otherwise units are (query tile, database split) over the whole
    // database, the two tiles of a pair next to each other.
    const TcUnit *units;
    const int64_t *n_units;
    uint64_t *partial;               // split mode: [n_split][nq][k]; list mode: [slot][k]
    uint32_t *err;
    // Batched tree search (split mode only; all null otherwise):
    //   need      bit (pair mp, scan tile g) at need[mp * need_words + g / 32]:
    //             only tiles whose bit is set are multiplied
    //   kmask     per scan tile, the 128-bit K chunks with any bit in the
    //             tile: the others contribute nothing and are skipped
    //   cap       per query row, a key >= its exact k-th result's key: larger
    //             keys are not kept, and in bound mode it is the threshold
    //   need_out  bound pass (MODE_BOUND): the "database" rows are tile
    //             images; bit (mp, g) is set when row g's bound
    //             popc(q & ~image) * Z is <= the cap of some query of pair mp
    const uint32_t *need;
    int64_t need_words;
    const uint32_t *kmask;
    const uint32_t *cap;
    uint32_t *need_out;
    // Split mode: per query, the smallest k-th key of any full list so far
    // (a key >= the exact k-th result's key, as `cap`), shared by all the
    // query's lists while they are built; 0xFFFFFFFF at the start.
    uint32_t *gcap;
    // Pre-widened database (split mode, PRE kernels): stage images
    // b_exp[tile][chunk][B_STAGE] of global tile `tile` (rows 128 tile ..),
    // and per tile its |t| record b_side[tile][SIDE_WORDS].
    const unsigned char *b_exp;
    const uint32_t *b_side;
};

// One work unit: query tile mt (< 0: absent) against database rows
// [r0, r1), taken in tiles of TN rows from r0 and multiplied NB tiles per
// step; query rows >= nvalid are padding.  Unit u is query tile u % 2 of
// pair unit u / 2.  An absent tile has no tiles to multiply, except in
// lock-step kernels (LOCK: both CTAs of a cluster walk the pair's steps
// together), where it multiplies the pair's first tile (mt_a) and keeps
// nothing.
struct Unit {
    int64_t mt, mt_a;
    int64_t r0, r1, ntiles, sp, out_base;
    int64_t mp, t0;                  // split mode: query-tile pair, first global tile
    int nvalid;
};

template <bool LOCK = false>
__device__ __forceinline__ Unit get_unit(const TcArgs &a, int64_t u)
{
    Unit v;
    if (a.units) {
        // list units: the first tiles of all units, then the second ones
        // (mostly absent), so that the CTAs, which take units round-robin,
        // all get present tiles whatever the parity of the grid
        const int64_t nu = __ldg(a.n_units);
        const int qh = u >= nu ? 1 : 0;
        const TcUnit t = a.units[qh ? u - nu : u];
        v.mt = qh ? t.a_tile1 : t.a_tile0;
        v.mt_a = v.mt;
        v.nvalid = qh ? t.nvalid1 : t.nvalid0;
        v.r0 = t.row0;
        v.r1 = t.row1;
        v.sp = 0;
        v.mp = 0;
        v.t0 = 0;
        v.out_base = t.out_base;
    } else {
        const int64_t pu = u >> 1;
        const int qh = (int)(u & 1);
        const int64_t mp = a.mp_base + pu % a.n_mpairs;
        v.sp = pu / a.n_mpairs;
        v.mp = mp;
        v.out_base = 0;
        const int64_t t0 = v.sp * a.tiles_per_split;
        v.t0 = t0;
        v.r0 = t0 * TN;
        v.r1 = a.n;
        const int64_t mt = QT * mp + qh;
        v.mt = mt < a.n_mtiles ? mt : -1;
        v.mt_a = v.mt >= 0 ? v.mt : (LOCK ? QT * mp : -1);
        v.nvalid = mt < a.n_mtiles ? (int)min((int64_t)TM, a.nq - mt * TM) : 0;
    }
    if (v.mt_a < 0) v.ntiles = 0;
    else if (a.units) v.ntiles = (v.r1 - v.r0 + TN - 1) / TN;
    else v.ntiles = min(a.n_ntiles, v.t0 + a.tiles_per_split) - v.t0;
    return v;
}

__device__ __forceinline__ int64_t unit_count(const TcArgs &a)
{
    return 2 * (a.units ? *a.n_units : (int64_t)a.n_mpairs * a.n_split);
}

// The first tile at or after local tile lt of unit uv that is multiplied
// (every tile without a need bitmap); uv.ntiles if none is left.
template <int MODE>
__device__ __forceinline__ int64_t next_tile(const TcArgs &a, const Unit &uv, int64_t lt)
{
    if (MODE != MODE_TREE || !a.need) return lt;
    const uint32_t *row = a.need + uv.mp * a.need_words;
    while (lt < uv.ntiles) {
        const int64_t g = uv.t0 + lt;
        const uint32_t w = __ldg(row + (g >> 5)) >> (g & 31);
        if (w) {
            lt += __ffs(w) - 1;
            break;
        }
        lt += 32 - (g & 31);
    }
    return lt < uv.ntiles ? lt : uv.ntiles;
}

// K chunks of local tile lt that are multiplied (never empty: a tile
// whose image is empty still runs chunk 0, so its accumulator is zeroed).
template <int MODE>
__device__ __forceinline__ uint32_t chunk_mask(const TcArgs &a, const Unit &uv, int64_t lt)
{
    if (MODE != MODE_TREE || !a.kmask) return 0xFFFFFFFFu;
    const uint32_t m = __ldg(a.kmask + uv.t0 + lt);
    return m ? m : 1u;
}

// A step: local tiles lt[0] and lt[1] of a unit (lt[1] < 0: absent), the
// two halves of one 256-row MMA operand.  The first step at or after local
// tile `from` pairs the next two tiles that are multiplied (adjacent ones
// without a need bitmap); lt[0] == uv.ntiles when none is left.
struct Step {
    int64_t lt[NB];
};

template <int MODE>
__device__ __forceinline__ Step first_step(const TcArgs &a, const Unit &uv, int64_t from)
{
    Step st;
    st.lt[0] = next_tile<MODE>(a, uv, from);
    const int64_t l1 = st.lt[0] < uv.ntiles ? next_tile<MODE>(a, uv, st.lt[0] + 1) : uv.ntiles;
    st.lt[1] = l1 < uv.ntiles ? l1 : -1;
    return st;
}

// Local tile after the step: where the next step's search starts.
__device__ __forceinline__ int64_t step_end(const Step &st)
{
    return (st.lt[1] >= 0 ? st.lt[1] : st.lt[0]) + 1;
}

// K chunks multiplied in a step: those of either tile.
template <int MODE>
__device__ __forceinline__ uint32_t step_mask(const TcArgs &a, const Unit &uv, const Step &st)
{
    uint32_t m = chunk_mask<MODE>(a, uv, st.lt[0]);
    if (st.lt[1] >= 0) m |= chunk_mask<MODE>(a, uv, st.lt[1]);
    return m;
}

// The first unit at or after u (in steps of the grid) with a tile to multiply.
template <int MODE>
__device__ __forceinline__ int64_t next_busy(const TcArgs &a, int64_t u, int64_t total, Unit &uv)
{
    for (; u < total; u += gridDim.x) {
        uv = get_unit(a, u);
        if (uv.ntiles > 0 && next_tile<MODE>(a, uv, 0) < uv.ntiles) break;
    }
    return u;
}

// Chunk c (16 bytes) of row `row` of local tile lt of unit uv; zeros past
// the unit's rows or for an absent tile (lt < 0).
__device__ __forceinline__ uint4 load_row(const TcArgs &a, const Unit &uv, int64_t lt, int row, int c)
{
    if (lt < 0) return make_uint4(0, 0, 0, 0);
    const int64_t t = uv.r0 + lt * TN + row;
    if (t >= uv.r1) return make_uint4(0, 0, 0, 0);
    return __ldg(reinterpret_cast<const uint4 *>(a.db + t * kWords) + c);
}

// Insert a candidate into a thread's sorted top-k list (rare once the list
// is full) and return the new k-th entry; kept out of line so the hot
// candidate loop stays small, with the k-th entry held in registers.
__device__ __noinline__ uint64_t list_insert(uint64_t *L, int k, uint32_t key, int64_t ti,
                                             const uint32_t *idx_map, uint64_t worst)
{
    const uint32_t id = idx_map ? __ldg(idx_map + ti) : (uint32_t)ti;
    const uint64_t cand = pack(key, id);
    if (cand >= worst) return worst;
    int p = k - 1;
    while (p > 0 && L[p - 1] > cand) {
        L[p] = L[p - 1];
        --p;
    }
    L[p] = cand;
    return L[k - 1];
}

// PRE: database chunks arrive pre-widened by bulk copies, and CL: the two
// CTAs of a cluster hold a pair's two query tiles and multicast the database
// chunks to each other (split mode; the two always go together).
template <int MODE, bool PRE, bool CL>
__global__ void __launch_bounds__(kernel_threads(PRE), 1) bf_tc_kernel(const TcArgs args)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        ((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // stage s: the query tile's chunk [A_STAGE], then the step's database
    // tiles' chunks [NB][B_STAGE] (rows 0-127 and 128-255 of the operand)
    TcCtl *ctl = reinterpret_cast<TcCtl *>(smem + STAGE_BYTES);
    // |t| ring: entry step % TP_RING (NB records of SIDE_WORDS words)
    static_assert(sizeof(TcCtl) % 16 == 0, "ring entries start 16-byte aligned");
    uint32_t *ring = reinterpret_cast<uint32_t *>(smem + STAGE_BYTES + sizeof(TcCtl));
    constexpr int TP_RING = tp_ring(MODE);
    uint32_t *err = args.err;

    constexpr int EPI = epi_warps(PRE), MMAW = mma_warp(PRE);
    static_assert(PRE == CL, "pre-widened chunks are shared by the CTA pairs");
    // slice groups: one per 4 epilogue warps, each with its own list per
    // query; in list mode (one list per slot) a single group, except for
    // k = 1, where the groups merge into the slot's entry by atomic minimum
    const int ngroups = args.units && args.k > 1 ? 1 : EPI / 4;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            // A (and with PRE, B) bytes + one arrival per producer warp
            mbar_init(&ctl->full[s], PRE ? 1 : 1 + PROD_WARPS);
            // CL: the MMAs of both CTAs of the cluster read the stage
            mbar_init(&ctl->empty[s], CL ? 2 : 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&ctl->acc_full[a], 1);
            mbar_init(&ctl->acc_empty[a], 4 * ngroups);
        }
        mbar_init(&ctl->final_bar, 1);
        ctl->abort = 0u;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&ctl->tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    if (CL) cluster_sync_all();       // the partner's barriers exist before any copy
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    const int64_t total_units = unit_count(args);

    if (PRE && warp == EPI) {
        // ------------------------------------------------ copy issuer (PRE)
        // The database arrives widened.  The two CTAs of a cluster hold the
        // two query tiles of a pair and walk the same steps: per chunk each
        // brings its query tile's chunk, and CTA rank h brings the chunk of
        // the step's database tile h into both CTAs (multicast), so every
        // database chunk is read once per pair.  With a step's last chunk
        // each CTA also copies the tiles' |t| records into its ring (at the
        // same point of the sequence where the producers below write them).
        if (lane == 0) {
            const uint32_t rank = CL ? cluster_rank() : 0u;
            uint32_t g = 0, t = 0;
            // query tiles are read again for every database tile: kept in
            // L2; the widened database streams past once per CTA wave
            const uint64_t keep = l2_keep_policy(), stream = l2_stream_policy();
            for (int64_t u = blockIdx.x; u < total_units && !ctl->abort; u += gridDim.x) {
                const Unit uv = get_unit<CL>(args, u);
                for (Step st = first_step<MODE>(args, uv, 0); st.lt[0] < uv.ntiles;
                     st = first_step<MODE>(args, uv, step_end(st)), ++t) {
                    const int64_t gt0 = uv.t0 + st.lt[0];
                    const int64_t gt1 = st.lt[1] >= 0 ? uv.t0 + st.lt[1] : -1;
                    const uint32_t km = step_mask<MODE>(args, uv, st);
                    const int last_c = 31 - __clz(km);
                    const uint32_t nb = gt1 >= 0 ? 2u : 1u;
                    uint32_t *slot = ring + (t % TP_RING) * (NB * SIDE_WORDS);
                    for (uint32_t m = km; m; m &= m - 1, ++g) {
                        const int c = __ffs(m) - 1;
                        const int s = (int)(g % STAGES);
                        const uint32_t r = g / STAGES;
                        if (!wait_spin(&ctl->empty[s], (r & 1u) ^ 1u, ctl, err)) goto issuer_done;
                        const uint32_t bytes = A_STAGE + nb * B_STAGE + (c == last_c ? nb * SIDE_BYTES : 0u);
                        mbar_arrive_expect_tx(&ctl->full[s], bytes);
                        unsigned char *dst = smem + (size_t)s * STAGE;
                        bulk_g2s_hint(dst, args.a_exp + ((size_t)uv.mt_a * NCHUNK + c) * A_STAGE,
                                      (uint32_t)A_STAGE, &ctl->full[s], keep);
                        const int64_t gt = rank ? gt1 : gt0;
                        if (gt >= 0)
                            bulk_g2s_mc_hint(dst + A_STAGE + rank * B_STAGE,
                                             args.b_exp + ((size_t)gt * NCHUNK + c) * B_STAGE,
                                             (uint32_t)B_STAGE, &ctl->full[s], 0x3, stream);
                        if (c == last_c) {
                            bulk_g2s_hint(slot, args.b_side + (size_t)gt0 * SIDE_WORDS, SIDE_BYTES,
                                          &ctl->full[s], stream);
                            if (gt1 >= 0)
                                bulk_g2s_hint(slot + SIDE_WORDS, args.b_side + (size_t)gt1 * SIDE_WORDS,
                                              SIDE_BYTES, &ctl->full[s], stream);
                        }
                    }
                }
            }
        issuer_done:
            drain_copies(ctl, g);
        }
    } else if (!PRE && warp >= EPI_WARPS && warp < EPI_WARPS + PROD_WARPS) {
        // ------------------------------------------------ producers
        // One database row of the step per thread: warps 8-11 the rows of
        // the step's first tile, 12-15 those of its second.  Chunks are
        // visited in groups of four consecutive chunk indices; a group is
        // loaded (64 bytes a thread) one group ahead of the one being
        // widened, and only the chunks of the step's mask are widened and
        // handed to the MMA.  |t| is summed on the way (skipped chunks hold
        // no bit of any row of either tile) and left in the ring.
        const int p = (warp - EPI_WARPS) * 32 + lane;   // row of the 256-row operand
        const int h = p / TN, row = p % TN, rg = row / 32;
        constexpr int G = 4;                       // chunks per load group
        uint32_t g = 0, t = 0, tp_acc = 0;
        Unit uv{};
        int64_t u = next_busy<MODE>(args, blockIdx.x, total_units, uv);
        Step st{};
        uint32_t km = 0;
        int grp = 0;
        // first group of the mask at or after group gi, or NCHUNK / G
        auto first_group = [](uint32_t m, int gi) {
            if (MODE != MODE_TREE) return gi < NCHUNK / G ? gi : NCHUNK / G;
            const uint32_t rest = gi < NCHUNK / G ? m >> (gi * G) : 0u;
            return rest ? gi + (__ffs(rest) - 1) / G : NCHUNK / G;
        };
        if (u < total_units) {
            st = first_step<MODE>(args, uv, 0);
            km = step_mask<MODE>(args, uv, st);
            grp = first_group(km, 0);
        }
        uint4 nx[G];
#pragma unroll
        for (int i = 0; i < G; ++i)
            nx[i] = u < total_units ? load_row(args, uv, st.lt[h], row, grp * G + i)
                                    : make_uint4(0, 0, 0, 0);
        while (u < total_units) {
            const int64_t mt = uv.mt;
            const int cur_grp = grp;
            const uint32_t cur_km = km;
            const int last_c = MODE == MODE_TREE ? 31 - __clz(cur_km) : NCHUNK - 1;
            uint4 cu[G];
#pragma unroll
            for (int i = 0; i < G; ++i) cu[i] = nx[i];
            // advance (u, step, grp) to the next group with a chunk to
            // multiply and prefetch it
            grp = first_group(km, grp + 1);
            if (grp == NCHUNK / G) {
                st = first_step<MODE>(args, uv, step_end(st));
                if (st.lt[0] == uv.ntiles) {
                    u = next_busy<MODE>(args, u + gridDim.x, total_units, uv);
                    if (u < total_units) st = first_step<MODE>(args, uv, 0);
                }
                if (u < total_units) {
                    km = step_mask<MODE>(args, uv, st);
                    grp = first_group(km, 0);
                }
            }
            if (u < total_units) {
#pragma unroll
                for (int i = 0; i < G; ++i) nx[i] = load_row(args, uv, st.lt[h], row, grp * G + i);
            }
#pragma unroll
            for (int i = 0; i < G; ++i) {
                const int c = cur_grp * G + i;
                if (MODE == MODE_TREE && !((cur_km >> c) & 1u)) continue;
                const int s = (int)(g % STAGES);
                const uint32_t r = g / STAGES;
                if (!warp_wait_spin(&ctl->empty[s], (r & 1u) ^ 1u, ctl, err, lane)) goto producers_done;
                unsigned char *dst = smem + (size_t)s * STAGE;
                if (p == 0) {
                    mbar_arrive_expect_tx(&ctl->full[s], (uint32_t)A_STAGE);
                    bulk_g2s(dst, args.a_exp + ((size_t)mt * NCHUNK + c) * A_STAGE,
                             (uint32_t)A_STAGE, &ctl->full[s]);
                }
                store_row_chunk(dst + A_STAGE, p, cu[i]);
                tp_acc += __popc(cu[i].x) + __popc(cu[i].y) + __popc(cu[i].z) + __popc(cu[i].w);
                if (c == last_c) {                     // row complete: its record for the epilogue
                    uint32_t *e = ring + (t % TP_RING) * (NB * SIDE_WORDS) + h * SIDE_WORDS;
                    e[row] = tp_acc;
                    const uint32_t mn = __reduce_min_sync(0xffffffffu, tp_acc);
                    if (lane == 0) e[TN + rg] = mn;
                    tp_acc = 0;
                    ++t;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->full[s]);
                ++g;
            }
        }
    producers_done:
        if (p == 0) drain_copies(ctl, g);     // the query-tile copies it issued
    } else if (warp == MMAW) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t g = 0, t = 0;
            for (int64_t u = blockIdx.x; u < total_units && !ctl->abort; u += gridDim.x) {
                const Unit uv = get_unit<CL>(args, u);
                for (Step st = first_step<MODE>(args, uv, 0); st.lt[0] < uv.ntiles;
                     st = first_step<MODE>(args, uv, step_end(st)), ++t) {
                    const uint32_t acc = t & 1u, ra = t >> 1;
                    if (!wait_spin(&ctl->acc_empty[acc], (ra & 1u) ^ 1u, ctl, err)) goto mma_done;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + acc * ACC_COLS;
                    uint32_t km = step_mask<MODE>(args, uv, st);
                    bool first = true;
                    for (; km; km &= km - 1, ++g) {
                        const int s = (int)(g % STAGES);
                        const uint32_t r = g / STAGES;
                        if (!wait_spin(&ctl->full[s], r & 1u, ctl, err)) goto mma_done;
                        tc_fence_after();
                        const uint32_t a_base = smem_u32(smem + (size_t)s * STAGE);
                        const uint32_t b_base = a_base + A_STAGE;
#pragma unroll
                        for (int kk = 0; kk < KC / 32; ++kk)
                            mma_e4m3(d_tmem, smem_desc_sw128(a_base + kk * 32u, SBO),
                                     smem_desc_sw128(b_base + kk * 32u, SBO), IDESC,
                                     (!first || kk != 0) ? 1u : 0u);
                        first = false;
                        // CL: the stage holds chunks the partner brought in
                        // and is refilled by both CTAs: free it in both
                        if (CL) mma_commit_mc(&ctl->empty[s], 0x3);
                        else mma_commit(&ctl->empty[s]);
                    }
                    mma_commit(&ctl->acc_full[acc]);
                }
            }
        mma_done:
            mma_commit(&ctl->final_bar);          // every MMA issued here has completed
            wait_or_abort(&ctl->final_bar, 0u, ctl, err);
        }
        __syncwarp();
    } else if (warp < EPI && (warp >> 2) < ngroups) {
        // ------------------------------------------------ epilogue
        // Warp w reads TMEM lanes 32 (w % 4) .. + 31 (its sub-partition)
        // and slices cs0 .. cs1 - 1 of each accumulator; slice cs covers
        // rows 32 (cs % 4) .. + 31 of the step's tile cs / 4.
        const int quarter = warp & 3, grp = warp >> 2;
        const int cs0 = grp * (SLICES / ngroups), cs1 = cs0 + SLICES / ngroups;
        const int row = quarter * 32 + lane;         // TMEM lane = query row of the tile
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        const int k = args.k;
        const int64_t nq = args.nq;
        uint64_t L[kMaxK];
        uint32_t t = 0;
        for (int64_t u = blockIdx.x; u < total_units; u += gridDim.x) {
            const Unit uv = get_unit<CL>(args, u);
            const int64_t qi = uv.mt * TM + row;      // query (split mode) or pair slot (list mode)
            const bool valid = uv.mt >= 0 && row < uv.nvalid;
            const QueryWeights w = query_weights(valid ? args.qpop[qi] : 0u);
            // a cap known to be >= the exact k-th key: nothing above it is kept
            const uint32_t capk =
                (MODE != MODE_PLAIN && args.cap && valid) ? __ldg(args.cap + qi) : 0xFFFFFFFFu;
            uint64_t capw = capk == 0xFFFFFFFFu ? kEmpty : pack(capk, 0xFFFFFFFFu);
            uint32_t published = capk;        // the largest key not worth publishing
            // key = A*Z + B*P = (|q| - O) Z + (|t| - O) P = |t| P + |q| Z - O (Z + P).
            // The bit pattern F of 4096 * sum + 2^23 is 0x4B000000 + O, so
            // key = |t| P + (|q| Z + 0x4B000000 (Z + P)) - F (Z + P) in
            // 32-bit arithmetic, which wraps back to the exact key.
            const uint32_t qz = w.pop * w.Z, zp = w.Z + w.P;
            const uint32_t qzc = qz + 0x4B000000u * zp, nzp = 0u - zp;
            for (int j = 0; j < k; ++j) L[j] = kEmpty;
            uint64_t worst = capw;
            uint32_t wkey = capk;             // key part of `worst`
            for (Step st = first_step<MODE>(args, uv, 0); st.lt[0] < uv.ntiles;
                 st = first_step<MODE>(args, uv, step_end(st)), ++t) {
                const uint32_t acc = t & 1u, ra = t >> 1;
                if (MODE != MODE_BOUND && args.gcap && valid) {
                    // the query's other lists may have found closer rows:
                    // nothing above their k-th key can be in the result
                    const uint32_t gc = __ldcg(args.gcap + qi);
                    if (gc < wkey) {
                        capw = pack(gc, 0xFFFFFFFFu);
                        worst = worst < capw ? worst : capw;
                        wkey = (uint32_t)(worst >> 32);
                        published = gc;
                    }
                }
                if (!warp_wait(&ctl->acc_full[acc], ra & 1u, ctl, err, lane)) goto done;
                tc_fence_after();
                const uint32_t *side = ring + (t % TP_RING) * (NB * SIDE_WORDS);
                for (int cs = cs0; cs < cs1; ++cs) {
                    const int h = cs / (TN / 32), cb = cs % (TN / 32);
                    const int64_t lt = st.lt[h];
                    if (lt < 0) continue;
                    const int64_t b0 = uv.r0 + lt * TN + cb * 32;
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(lane_base + acc * ACC_COLS + (uint32_t)cs * 32, v);
                    tmem_ld_wait();
                    if constexpr (MODE == MODE_BOUND) {
                        // bound pass: row j of the slice is the image of scan
                        // tile b0 + j; a bit per tile some valid query may need
                        const int m = (int)(uv.r1 - b0 < 32 ? (uv.r1 - b0 > 0 ? uv.r1 - b0 : 0) : 32);
                        uint32_t bits = 0;
                        if (valid) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const uint32_t o =
                                    __float_as_uint(fmaf(__uint_as_float(v[j]), 4096.0f, 8388608.0f)) -
                                    0x4B000000u;
                                const uint32_t lb = (w.pop - o) * w.Z;   // popc(q & ~image) * Z
                                if (j < m && lb <= capk) bits |= 1u << j;
                            }
                        }
                        bits = __reduce_or_sync(0xffffffffu, bits);
                        if (lane == 0 && bits)
                            atomicOr(args.need_out + uv.mp * args.need_words + (b0 >> 5), bits);
                        continue;
                    }
                    const uint32_t *tp = side + h * SIDE_WORDS;   // |t| [TN], minima [TN / 32]
                    // Slice filter: every key here is >= |t|min P + |q| Z - Omax (Z + P);
                    // when that exceeds the k-th key no row of the slice can enter
                    // the list.  The values are non-negative floats, ordered as
                    // their bit patterns.
                    if (wkey != 0xFFFFFFFFu) {
                        uint32_t mx = 0;
#pragma unroll
                        for (int j = 0; j < 32; j += 2) mx = __vimax3_u32(mx, v[j], v[j + 1]);
                        const uint32_t omax =
                            __float_as_uint(fmaf(__uint_as_float(mx), 4096.0f, 8388608.0f)) - 0x4B000000u;
                        const uint32_t tmin = tp[TN + cb];
                        if ((int64_t)omax * zp < (int64_t)qz + (int64_t)tmin * w.P - (int64_t)wkey)
                            continue;
                    }
                    // every row's key, without branches; v[j] becomes the key
                    const uint4 *tp4 = reinterpret_cast<const uint4 *>(tp + cb * 32);
                    uint32_t bits = 0;
#pragma unroll
                    for (int j4 = 0; j4 < 8; ++j4) {
                        const uint4 t4 = tp4[j4];
                        const uint32_t tt[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int j = 4 * j4 + i;
                            const uint32_t f =
                                __float_as_uint(fmaf(__uint_as_float(v[j]), 4096.0f, 8388608.0f));
                            v[j] = f * nzp + (tt[i] * w.P + qzc);
                            bits |= (v[j] <= wkey ? 1u : 0u) << j;
                        }
                    }
                    const int64_t m = uv.r1 - b0;        // rows of the slice that exist
                    if (m < 32) bits &= m > 0 ? (1u << m) - 1u : 0u;
                    if (bits) {                          // rare once the list has filled
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if ((bits >> j) & 1u) {
                                worst = list_insert(L, k, v[j], b0 + j, args.idx_map, worst);
                                worst = worst < capw ? worst : capw;
                                wkey = (uint32_t)(worst >> 32);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->acc_empty[acc]);
                if (MODE != MODE_BOUND && args.gcap && valid && wkey < published &&
                    L[k - 1] != kEmpty) {
                    // a full list: its k-th key bounds the query's result
                    atomicMin(args.gcap + qi, wkey);
                    published = wkey;
                }
            }
            if (MODE != MODE_BOUND && valid) {
                uint64_t *out = args.units ? args.partial + (uv.out_base + qi) * k
                                           : args.partial + ((uv.sp * ngroups + grp) * nq + qi) * k;
                if (args.units && ngroups > 1)      // k == 1: the groups share the entry
                    atomicMin(reinterpret_cast<unsigned long long *>(out), (unsigned long long)L[0]);
                else
                    for (int j = 0; j < k; ++j) out[j] = L[j];
            }
        }
    }
done:
    tc_fence_before();
    __syncthreads();
    // CL: no CTA leaves while its partner may still copy into it or
    // release its stages
    if (CL) cluster_sync_all();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// One warp per query: the smallest entry over the split lists -> its index.
__global__ void merge_top1_kernel(const uint64_t *__restrict__ partial, int n_split, int64_t nq,
                                  uint32_t *__restrict__ nn)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    uint64_t best = kEmpty;
    for (int s = lane; s < n_split; s += 32) {
        uint64_t v = partial[(int64_t)s * nq + q];
        best = v < best ? v : best;
    }
    best = warp_min_u64(best);
    if (lane == 0) nn[q] = best == kEmpty ? 0xFFFFFFFFu : (uint32_t)best;
}

// Split-mode scans run over at most this many pairs of query tiles per
// launch: 96 pre-widened query tiles (48 MB) stay resident in L2 while the
// database streams past, instead of being fetched from HBM again for every
// database tile when a call has more queries than L2 holds.
constexpr int kBatchPairs = 48;

// Pre-widened kernels run as clusters of two CTAs (the two query tiles of
// a pair).  Launch configuration, and how many such clusters the device
// holds at once (queried once per device and kernel mode; 0 when none
// fits, and then the in-kernel widening is used).
template <int MODE>
cudaLaunchConfig_t pre_config(int grid, cudaStream_t s, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t c{};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    c.gridDim = dim3((unsigned)grid);
    c.blockDim = dim3((unsigned)kernel_threads(true));
    c.dynamicSmemBytes = smem_bytes(MODE);
    c.stream = s;
    c.attrs = attr;
    c.numAttrs = 1;
    return c;
}

template <int MODE>
int pre_clusters()
{
    static std::mutex mu;
    static int cached[64];
    static bool known[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!known[dev]) {
        int n = 0;
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t c = pre_config<MODE>(2, nullptr, attr);
        if (allow_smem((const void *)bf_tc_kernel<MODE, true, true>, (int)smem_bytes(MODE)) != cudaSuccess ||
            cudaOccupancyMaxActiveClusters(&n, (const void *)bf_tc_kernel<MODE, true, true>, &c) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        cached[dev] = n;
        known[dev] = true;
    }
    return cached[dev];
}

// Launch a pre-widened kernel over `units` units (an even number: pairs).
template <int MODE>
cudaError_t launch_pre(const TcArgs &a, int64_t units, cudaStream_t s)
{
    const int ncl = pre_clusters<MODE>();
    if (ncl < 1) return cudaErrorLaunchOutOfResources;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t c =
        pre_config<MODE>((int)(2 * std::min<int64_t>(ncl, (units + 1) / 2)), s, attr);
    return cudaLaunchKernelEx(&c, bf_tc_kernel<MODE, true, true>, a);
}

// Should a split-mode scan of n rows by nq queries read a pre-widened copy
// of the rows (kernel variant PRE)?  The copy costs one pass writing
// n * 4 KB (8x the rows) and that much scratch; it spares every unit the
// producers' widening.  forced: 1 never, 2 always, 0 from eight query
// tiles on when the copy fits in half the free device memory.
bool want_prewiden(int64_t n, int64_t nq, int forced)
{
    if (forced == 1) return false;
    if (pre_clusters<MODE_PLAIN>() < 1 || pre_clusters<MODE_TREE>() < 1) return false;
    if (forced == 2) return true;
    if (nq < 8 * TM) return false;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t bytes = (size_t)((n + TN - 1) / TN) * ((size_t)NCHUNK * B_STAGE + SIDE_BYTES);
    return bytes <= free_b / 2;
}

// Database splits for `per` units per split on `ctas` persistent CTAs that
// take units round-robin: the fewest splits whose units fill the last wave
// best, so that every CTA runs the same number of units (10M x 10k top-10:
// 19 splits, ten full waves, 5% faster than 7 splits and a 92% last wave);
// at most 64 splits and at least 8 tiles (4 steps) per split.
int pick_tc_splits(int64_t per, int64_t n_tiles, int ctas)
{
    const int max_s = (int)std::max<int64_t>(1, std::min<int64_t>(64, n_tiles / 8));
    int best = 1;
    double best_eff = -1.0;
    for (int sp = 1; sp <= max_s; ++sp) {
        const double waves = (double)per * sp / ctas;
        const double eff = waves / std::ceil(waves);
        if (eff > best_eff + 0.004) {
            best_eff = eff;
            best = sp;
        }
    }
    return best;
}

// Tiles per split when n_tiles tiles are cut into `splits` splits, rounded
// up to whole steps so that no split ends with a half-empty step.
int64_t step_tiles(int64_t n_tiles, int splits)
{
    const int64_t t = (n_tiles + splits - 1) / splits;
    return (t + NB - 1) / NB * NB;
}

// Stage images and |t| records of rows [0, n) of db, tiled by TN rows
// (rows past n are zero), from `scratch`.
// Widen rows [0, n) into b_exp / b_side (sized as in prewiden_rows).
int widen_rows_into(const uint64_t *db, int64_t n, unsigned char *b_exp, uint32_t *b_side,
                    Scratch &scratch, cudaStream_t s)
{
    const int64_t n_tiles = (n + TN - 1) / TN;
    uint32_t *rowpop = nullptr;
    DT_CUDA_TRY(scratch.alloc(&rowpop, (size_t)n_tiles * TN * 4));
    static_assert(TN == TM && B_STAGE == A_STAGE, "database tiles widen like query tiles");
    const int64_t items = n_tiles * TN * NCHUNK;
    {
        KernelTimer timer("prewiden", s);
        widen_queries_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(db, n, (int)n_tiles, b_exp,
                                                                             rowpop);
        side_kernel<<<(unsigned)n_tiles, TN, 0, s>>>(rowpop, n, b_side);
    }
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

int prewiden_rows(const uint64_t *db, int64_t n, Scratch &scratch, cudaStream_t s,
                  unsigned char **b_exp, uint32_t **b_side)
{
    const int64_t n_tiles = (n + TN - 1) / TN;
    DT_CUDA_TRY(scratch.alloc(b_exp, (size_t)n_tiles * NCHUNK * B_STAGE));
    DT_CUDA_TRY(scratch.alloc(b_side, (size_t)n_tiles * SIDE_BYTES));
    return widen_rows_into(db, n, *b_exp, *b_side, scratch, s);
}

// Per-split top-k lists of every query over db (rows reported through
// idx_map when given).  *partial is allocated on the stream; the caller frees it.
int tc_partial_topk(const uint64_t *db, int64_t n, const uint32_t *idx_map, const uint64_t *q,
                    int64_t nq, int k, cudaStream_t s, Scratch &scratch, uint64_t **partial_out,
                    int *n_split_out, const TuneCfg *cfg)
{
    DT_CUDA_TRY(allow_smem((const void *)bf_tc_kernel<MODE_PLAIN, false, false>, (int)smem_bytes(MODE_PLAIN)));
    DT_CUDA_TRY(allow_smem((const void *)bf_tc_kernel<MODE_PLAIN, true, true>, (int)smem_bytes(MODE_PLAIN)));
    const int n_mtiles = (int)((nq + TM - 1) / TM);
    const int n_mpairs = (n_mtiles + QT - 1) / QT;
    const int64_t n_ntiles = (n + TN - 1) / TN;
    const int sms = sm_count();
    TuneCfg c{0, 0};
    if (cfg) c = *cfg;
    else tune_lookup(TUNE_TC, n, nq, k, &c);
    const bool pre = want_prewiden(n, nq, c.b);
    const int batch_pairs = std::min(n_mpairs, kBatchPairs);
    const int splits = c.a > 0 ? (int)std::min<int64_t>(c.a, n_ntiles)
                               : pick_tc_splits(2 * batch_pairs, n_ntiles, sms);
    const int64_t tiles_per_split = step_tiles(n_ntiles, splits);
    const int n_split = (int)((n_ntiles + tiles_per_split - 1) / tiles_per_split);

    unsigned char *a_exp = nullptr;
    uint32_t *qpop = nullptr, *err = nullptr;
    uint64_t *partial = nullptr;
    const size_t a_bytes = (size_t)n_mtiles * NCHUNK * A_STAGE;
    DT_CUDA_TRY(scratch.alloc(&a_exp, a_bytes));
    DT_CUDA_TRY(scratch.alloc(&qpop, (size_t)nq * 4));
    const int n_lists = n_split * lists_per_unit(pre);
    DT_CUDA_TRY(scratch.alloc(&partial, (size_t)n_lists * nq * k * 8));
    // lists start empty: a block that gives up on a wait leaves valid lists
    DT_CUDA_TRY(cudaMemsetAsync(partial, 0xFF, (size_t)n_lists * nq * k * 8, s));
    uint32_t *gcap = nullptr;
    DT_CUDA_TRY(scratch.alloc(&gcap, (size_t)nq * 4));
    DT_CUDA_TRY(cudaMemsetAsync(gcap, 0xFF, (size_t)nq * 4, s));
    DT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_tc_error));
    const int64_t items = (int64_t)n_mtiles * TM * NCHUNK;
    widen_queries_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(q, nq, n_mtiles, a_exp, qpop);
    DT_CUDA_TRY(cudaGetLastError());
    TcArgs a{};
    a.db = db;
    a.n = n;
    a.a_exp = a_exp;
    a.qpop = qpop;
    a.idx_map = idx_map;
    a.nq = nq;
    a.k = k;
    a.n_mtiles = n_mtiles;
    a.n_mpairs = n_mpairs;
    a.n_ntiles = n_ntiles;
    a.tiles_per_split = tiles_per_split;
    a.n_split = n_split;
    a.units = nullptr;
    a.n_units = nullptr;
    a.partial = partial;
    a.err = err;
    a.gcap = gcap;
    if (pre) {
        unsigned char *b_exp = nullptr;
        uint32_t *b_side = nullptr;
        if (int r = prewiden_rows(db, n, scratch, s, &b_exp, &b_side)) return r;
        a.b_exp = b_exp;
        a.b_side = b_side;
    }
    for (int p0 = 0; p0 < n_mpairs; p0 += kBatchPairs) {     // L2-sized batches of queries
        a.mp_base = p0;
        a.n_mpairs = std::min(kBatchPairs, n_mpairs - p0);
        const int grid = (int)std::min<int64_t>(2 * (int64_t)a.n_mpairs * n_split, sms);
        KernelTimer timer("tc_scan", s);
        if (pre)
            DT_CUDA_TRY(launch_pre<MODE_PLAIN>(a, 2 * (int64_t)a.n_mpairs * n_split, s));
        else
            bf_tc_kernel<MODE_PLAIN, false, false><<<grid, kernel_threads(false), smem_bytes(MODE_PLAIN), s>>>(a);
        DT_CUDA_TRY(cudaGetLastError());
    }
    *partial_out = partial;
    *n_split_out = n_lists;
    return DT_OK;
}

}  // namespace

int take_tc_error(bool *raised)
{
    uint32_t v = 0, zero = 0;
    DT_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(v)));
    if (v) DT_CUDA_TRY(cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(zero)));
    *raised = v != 0;
    return DT_OK;
}

int launch_tc_units(const uint64_t *db, int64_t n, const uint32_t *idx_map, const uint64_t *q,
                    const int32_t *slot_q, const TcUnit *units, const int64_t *n_units,
                    const int64_t *n_tiles, int64_t max_tiles, int k, uint64_t *partial,
                    cudaStream_t s)
{
    DT_CUDA_TRY(allow_smem((const void *)bf_tc_kernel<MODE_PLAIN, false, false>, (int)smem_bytes(MODE_PLAIN)));
    if (max_tiles <= 0) return DT_OK;
    unsigned char *a_exp = nullptr;
    uint32_t *qpop = nullptr, *err = nullptr;
    Scratch scratch(s);
    DT_CUDA_TRY(scratch.alloc(&a_exp, (size_t)max_tiles * NCHUNK * A_STAGE));
    DT_CUDA_TRY(scratch.alloc(&qpop, (size_t)max_tiles * TM * 4));
    DT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_tc_error));
    const int64_t items = max_tiles * TM * NCHUNK;
    widen_gather_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(q, slot_q, n_tiles,
                                                                        max_tiles, a_exp, qpop);
    DT_CUDA_TRY(cudaGetLastError());
    TcArgs a{};
    a.db = db;
    a.n = n;
    a.a_exp = a_exp;
    a.qpop = qpop;
    a.idx_map = idx_map;
    a.nq = max_tiles * TM;
    a.k = k;
    a.units = units;
    a.n_units = n_units;
    a.partial = partial;
    a.err = err;
    const int grid = (int)std::min<int64_t>(max_tiles, sm_count());   // units <= tiles
    bf_tc_kernel<MODE_PLAIN, false, false><<<grid, kernel_threads(false), smem_bytes(MODE_PLAIN), s>>>(a);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

size_t tc_tile_bytes() { return (size_t)NCHUNK * A_STAGE; }

int launch_widen_queries(const uint64_t *q, int64_t nq, unsigned char *a_exp, uint32_t *qpop,
                         cudaStream_t s)
{
    if (nq <= 0) return DT_OK;
    const int n_mtiles = (int)((nq + TM - 1) / TM);
    const int64_t items = (int64_t)n_mtiles * TM * NCHUNK;
    widen_queries_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(q, nq, n_mtiles, a_exp, qpop);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

int launch_tc_units_pre(const uint64_t *db, int64_t n, const uint32_t *idx_map,
                        const unsigned char *a_exp, const uint32_t *qpop, const TcUnit *units,
                        const int64_t *n_units, int64_t max_units, int k, uint64_t *partial,
                        cudaStream_t s)
{
    DT_CUDA_TRY(allow_smem((const void *)bf_tc_kernel<MODE_PLAIN, false, false>, (int)smem_bytes(MODE_PLAIN)));
    if (max_units <= 0) return DT_OK;
    uint32_t *err = nullptr;
    DT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_tc_error));
    TcArgs a{};
    a.db = db;
    a.n = n;
    a.a_exp = a_exp;
    a.qpop = qpop;
    a.idx_map = idx_map;
    a.nq = 0;
    a.k = k;
    a.units = units;
    a.n_units = n_units;
    a.partial = partial;
    a.err = err;
    const int grid = (int)std::min<int64_t>(2 * max_units, sm_count());
    bf_tc_kernel<MODE_PLAIN, false, false><<<grid, kernel_threads(false), smem_bytes(MODE_PLAIN), s>>>(a);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

int launch_tree_tc(const dt_index *ix, const uint64_t *q, int64_t nq, const int32_t *slot_q,
                   const uint32_t *cap_slot, int n_mtiles, int k, Scratch &scratch, cudaStream_t s,
                   uint64_t **partial_out, int *n_split_out, std::vector<uint32_t> *need_host,
                   int64_t *need_words_out)
{
    static_assert(TN == kScanTileRows, "scan tiles are tensor-core tiles");
    DT_CUDA_TRY(allow_smem((const void *)bf_tc_kernel<MODE_BOUND, false, false>, (int)smem_bytes(MODE_BOUND)));
    DT_CUDA_TRY(allow_smem((const void *)bf_tc_kernel<MODE_TREE, false, false>, (int)smem_bytes(MODE_TREE)));
    DT_CUDA_TRY(allow_smem((const void *)bf_tc_kernel<MODE_TREE, true, true>, (int)smem_bytes(MODE_TREE)));
    const int64_t n = ix->n;
    const int64_t n_tt = (n + TN - 1) / TN;             // scan tiles
    const int64_t need_words = (n_tt + 31) / 32;
    const int n_mpairs = (n_mtiles + QT - 1) / QT;
    const int sms = sm_count();
    unsigned char *a_exp = nullptr;
    uint32_t *qpop = nullptr, *need = nullptr, *err = nullptr;
    uint64_t *partial = nullptr;
    DT_CUDA_TRY(scratch.alloc(&a_exp, (size_t)n_mtiles * NCHUNK * A_STAGE));
    DT_CUDA_TRY(scratch.alloc(&qpop, (size_t)n_mtiles * TM * 4));
    DT_CUDA_TRY(scratch.alloc(&need, (size_t)n_mpairs * need_words * 4));
    DT_CUDA_TRY(cudaMemsetAsync(need, 0, (size_t)n_mpairs * need_words * 4, s));
    DT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_tc_error));
    const int64_t items = (int64_t)n_mtiles * TM * NCHUNK;
    widen_gather_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(q, slot_q, nullptr, n_mtiles,
                                                                        a_exp, qpop);
    DT_CUDA_TRY(cudaGetLastError());

    // pass 1: every (pair of slot tiles, tile image) bound; the images are
    // the rows of a small database of n_tt rows
    TcArgs b{};
    b.db = ix->tile_or;
    b.n = n_tt;
    b.a_exp = a_exp;
    b.qpop = qpop;
    b.nq = nq;
    b.k = k;
    b.n_mtiles = n_mtiles;
    b.n_mpairs = n_mpairs;
    b.n_ntiles = (n_tt + TN - 1) / TN;
    const int batch_pairs = std::min(n_mpairs, kBatchPairs);
    {
        const int splits = pick_tc_splits(2 * batch_pairs, b.n_ntiles, sms);
        b.tiles_per_split = step_tiles(b.n_ntiles, splits);
        b.n_split = (int)((b.n_ntiles + b.tiles_per_split - 1) / b.tiles_per_split);
    }
    b.cap = cap_slot;
    b.need_out = need;
    b.need_words = need_words;
    b.err = err;
    for (int p0 = 0; p0 < n_mpairs; p0 += kBatchPairs) {     // L2-sized batches of queries
        b.mp_base = p0;
        b.n_mpairs = std::min(kBatchPairs, n_mpairs - p0);
        KernelTimer timer("tree_bound", s);
        bf_tc_kernel<MODE_BOUND, false, false><<<(int)std::min<int64_t>(2 * (int64_t)b.n_mpairs * b.n_split, sms),
                                           kernel_threads(false), smem_bytes(MODE_BOUND), s>>>(b);
    }
    DT_CUDA_TRY(cudaGetLastError());

    // pass 2: the needed scan tiles of each pair, zero K chunks skipped
    TcArgs a{};
    a.db = ix->db_tree;
    a.n = n;
    a.a_exp = a_exp;
    a.qpop = qpop;
    a.idx_map = ix->perm;
    a.nq = nq;
    a.k = k;
    a.n_mtiles = n_mtiles;
    a.n_mpairs = n_mpairs;
    a.n_ntiles = n_tt;
    TuneCfg c{0, 0};
    tune_lookup(TUNE_TREE_TC, n, nq, k, &c);
    const int splits = c.a > 0 ? (int)std::min<int64_t>(c.a, n_tt) : pick_tc_splits(2 * batch_pairs, n_tt, sms);
    a.tiles_per_split = step_tiles(n_tt, splits);
    a.n_split = (int)((n_tt + a.tiles_per_split - 1) / a.tiles_per_split);
    a.need = need;
    a.need_words = need_words;
    a.kmask = ix->tile_kmask;
    a.cap = cap_slot;
    a.err = err;
    // a resident widened copy costs nothing per call: use it unless forced off
    const bool pre = ix->scan_exp && c.b != 1 && pre_clusters<MODE_TREE>() > 0
                         ? true
                         : want_prewiden(n, nq, c.b);
    const int n_lists = a.n_split * lists_per_unit(pre);
    DT_CUDA_TRY(scratch.alloc(&partial, (size_t)n_lists * nq * k * 8));
    DT_CUDA_TRY(cudaMemsetAsync(partial, 0xFF, (size_t)n_lists * nq * k * 8, s));
    a.partial = partial;
    uint32_t *gcap = nullptr;
    DT_CUDA_TRY(scratch.alloc(&gcap, (size_t)n_mtiles * TM * 4));
    DT_CUDA_TRY(cudaMemsetAsync(gcap, 0xFF, (size_t)n_mtiles * TM * 4, s));
    a.gcap = gcap;
    if (pre && ix->scan_exp) {
        a.b_exp = ix->scan_exp;
        a.b_side = ix->scan_side;
    } else if (pre) {
        unsigned char *b_exp = nullptr;
        uint32_t *b_side = nullptr;
        if (int r = prewiden_rows(ix->db_tree, n, scratch, s, &b_exp, &b_side)) return r;
        a.b_exp = b_exp;
        a.b_side = b_side;
    }
    for (int p0 = 0; p0 < n_mpairs; p0 += kBatchPairs) {     // L2-sized batches of queries
        a.mp_base = p0;
        a.n_mpairs = std::min(kBatchPairs, n_mpairs - p0);
        const int grid = (int)std::min<int64_t>(2 * (int64_t)a.n_mpairs * a.n_split, sms);
        KernelTimer timer("tree_scan", s);
        if (pre)
            DT_CUDA_TRY(launch_pre<MODE_TREE>(a, 2 * (int64_t)a.n_mpairs * a.n_split, s));
        else
            bf_tc_kernel<MODE_TREE, false, false><<<grid, kernel_threads(false), smem_bytes(MODE_TREE), s>>>(a);
        DT_CUDA_TRY(cudaGetLastError());
    }
    DT_CUDA_TRY(cudaGetLastError());
    if (need_host) {
        need_host->resize((size_t)n_mpairs * need_words);
        DT_CUDA_TRY(cudaMemcpyAsync(need_host->data(), need, need_host->size() * 4,
                                    cudaMemcpyDeviceToHost, s));
    }
    *partial_out = partial;
    *n_split_out = n_lists;
    *need_words_out = need_words;
    return DT_OK;
}

// Keep (on) or release (off) the index's resident widened copy of its
// tree-ordered rows.  The arrays are plain device allocations owned by the
// index; the widening runs on stream s and is complete on return.
int index_keep_widened(dt_index *ix, bool on, cudaStream_t s)
{
    if (!on) {
        if (ix->scan_exp || ix->scan_side) {
            DT_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(ix->scan_exp);
            cudaFree(ix->scan_side);
            ix->scan_exp = nullptr;
            ix->scan_side = nullptr;
        }
        return DT_OK;
    }
    if (ix->scan_exp) return DT_OK;
    const int64_t n_tiles = (ix->n + TN - 1) / TN;
    const size_t exp_bytes = (size_t)n_tiles * NCHUNK * B_STAGE, side_bytes = (size_t)n_tiles * SIDE_BYTES;
    unsigned char *e = nullptr;
    uint32_t *sd = nullptr;
    if (cudaMalloc(&e, exp_bytes) != cudaSuccess) {
        cudaGetLastError();
        return DT_ENOMEM;
    }
    if (cudaMalloc(&sd, side_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(e);
        return DT_ENOMEM;
    }
    int rc = DT_OK;
    {
        Scratch scratch(s);
        rc = widen_rows_into(ix->db_tree, ix->n, e, sd, scratch, s);
    }
    if (rc == DT_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = DT_ECUDA;
    if (rc != DT_OK) {
        cudaFree(e);
        cudaFree(sd);
        return rc;
    }
    ix->scan_exp = e;
    ix->scan_side = sd;
    return DT_OK;
}

int launch_bf_tc_cfg(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                     uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s, const TuneCfg *cfg)
{
    Scratch scratch(s);
    uint64_t *partial = nullptr;
    int n_split = 0;
    if (int r = tc_partial_topk(db, n, nullptr, q, nq, k, s, scratch, &partial, &n_split, cfg))
        return r;
    return launch_merge_partials(partial, n_split, db, n, q, nq, k, idx, score, ab, s);
}

int launch_bf_tc(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                 uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s)
{
    return launch_bf_tc_cfg(db, n, q, nq, k, idx, score, ab, s, nullptr);
}

int launch_tc_top1(const uint64_t *db, int64_t n, const uint32_t *idx_map, const uint64_t *q,
                   int64_t nq, uint32_t *nn, cudaStream_t s)
{
    Scratch scratch(s);
    uint64_t *partial = nullptr;
    int n_split = 0;
    if (int r = tc_partial_topk(db, n, idx_map, q, nq, 1, s, scratch, &partial, &n_split, nullptr))
        return r;
    merge_top1_kernel<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(partial, n_split, nq, nn);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

}  // namespace dtk
