// index_io.cu — saving a built (or grown) Dissimilarity Tree to a file and
// loading it back.
//
// The file holds the tree, not the descriptors: the caller keeps the
// database (in original-index order) and passes it to dt_load, which
// rebuilds the tree-ordered copy on the GPU.  Layout, little-endian:
//   header (IndexFileHeader below, 64 bytes)
//   node records   [n_nodes] x {first_child, begin, count, level} int32
//   OR images      [n_nodes][64] uint64
//   AND images     [n_nodes][64] uint64, only when the header says so
//   permutation    [n] uint32 (tree position -> original index)
//   checksum       uint64 over every byte after the header (below)
// dt_load checks everything a search relies on before anything reaches the
// GPU: sizes, the checksum, that the nodes form one tree whose children
// partition their parent's segment and sit one level below it, that leaves
// hold at most leaf_size descriptors, the recorded depth and leaf count, and
// that the permutation is one.  Once the tree-ordered rows are on the GPU,
// one more pass checks the images against them (check_images_kernel): a
// file loaded over a database other than the one it was built over (other
// rows, or the same rows in another order) is rejected, because its images
// would no longer bound their subtrees and searches could silently miss
// results.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dt_internal.cuh"

namespace dtk {
namespace {

struct IndexFileHeader {
    char magic[8];          // "DTINDEX" and a zero byte
    uint32_t version;       // 1
    uint32_t header_bytes;  // sizeof(IndexFileHeader)
    int64_t n, n_nodes, n_leaves;
    int32_t depth, leaf_size, use_and, reserved;
    int64_t reserved2;
};
static_assert(sizeof(IndexFileHeader) == 64, "header layout");
static_assert(sizeof(NodeRec) == 16, "node record layout");

constexpr char kMagic[8] = {'D', 'T', 'I', 'N', 'D', 'E', 'X', 0};
constexpr uint32_t kVersion = 1;

// Checksum of a byte stream: each 8-byte little-endian word (the last one
// zero-padded) is mixed in by xor, multiply and shift.
struct Checksum {
    uint64_t h = 0x9e3779b97f4a7c15ull;
    uint64_t pending = 0;
    int have = 0;
    void word(uint64_t w)
    {
        h ^= w;
        h *= 0x100000001b3ull;
        h ^= h >> 29;
    }
    void bytes(const void *p, size_t len)
    {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < len; ++i) {
            pending |= (uint64_t)b[i] << (8 * have);
            if (++have == 8) {
                word(pending);
                pending = 0;
                have = 0;
            }
        }
    }
    uint64_t finish()
    {
        if (have) word(pending);
        have = 0;
        pending = 0;
        return h;
    }
};

struct File {
    std::FILE *f = nullptr;
    ~File()
    {
        if (f) std::fclose(f);
    }
};

int io_error(const std::string &what, const char *path)
{
    set_error(what + ": " + path);
    return DT_EIO;
}

int save_index(const dt_index *ix, const char *path)
{
    const int64_t nn = ix->n_nodes, n = ix->n;
    std::vector<NodeRec> node((size_t)nn);
    std::vector<uint64_t> img((size_t)nn * kWords);
    std::vector<uint64_t> aimg(ix->use_and ? (size_t)nn * kWords : 0);
    std::vector<uint32_t> perm((size_t)n);
    DT_CUDA_TRY(cudaMemcpy(node.data(), ix->node, node.size() * sizeof(NodeRec), cudaMemcpyDeviceToHost));
    DT_CUDA_TRY(cudaMemcpy(img.data(), ix->or_img, img.size() * 8, cudaMemcpyDeviceToHost));
    if (ix->use_and)
        DT_CUDA_TRY(cudaMemcpy(aimg.data(), ix->and_img, aimg.size() * 8, cudaMemcpyDeviceToHost));
    DT_CUDA_TRY(cudaMemcpy(perm.data(), ix->perm, perm.size() * 4, cudaMemcpyDeviceToHost));

    IndexFileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = sizeof(h);
    h.n = n;
    h.n_nodes = nn;
    h.n_leaves = ix->n_leaves;
    h.depth = ix->depth;
    h.leaf_size = ix->leaf_size;
    h.use_and = ix->use_and;

    File f;
    f.f = std::fopen(path, "wb");
    if (!f.f) return io_error("cannot open for writing", path);
    Checksum ck;
    auto put = [&](const void *p, size_t len, bool sum) {
        if (sum) ck.bytes(p, len);
        return len == 0 || std::fwrite(p, 1, len, f.f) == len;
    };
    bool ok = put(&h, sizeof(h), false) && put(node.data(), node.size() * sizeof(NodeRec), true) &&
              put(img.data(), img.size() * 8, true) && put(aimg.data(), aimg.size() * 8, true) &&
              put(perm.data(), perm.size() * 4, true);
    const uint64_t sum = ck.finish();
    ok = ok && put(&sum, 8, false);
    ok = std::fclose(f.f) == 0 && ok;
    f.f = nullptr;
    if (!ok) return io_error("write failed", path);
    return DT_OK;
}

// A host copy of a tree read from a file.
struct LoadedIndex {
    IndexFileHeader h;
    std::vector<NodeRec> node;
    std::vector<uint64_t> img, aimg;
    std::vector<uint32_t> perm;
};

int bad_file(const std::string &why)
{
    set_error("index file rejected: " + why);
    return DT_EINVAL;
}

// One tree rooted at node 0 over positions [0, n): every other node is the
// child of exactly one node with a smaller id, children split their
// parent's segment (similar part first) one level below it, leaves hold at
// most leaf_size descriptors; depth and leaf count as recorded.
int check_tree(const LoadedIndex &L)
{
    const IndexFileHeader &h = L.h;
    const int64_t nn = h.n_nodes;
    const NodeRec &root = L.node[0];
    if (root.begin != 0 || root.count != h.n || root.level != 0) return bad_file("root");
    std::vector<uint8_t> parented((size_t)nn, 0);
    int64_t leaves = 0;
    int32_t depth = 0;
    for (int64_t i = 0; i < nn; ++i) {
        const NodeRec &r = L.node[(size_t)i];
        if (i > 0 && !parented[(size_t)i]) return bad_file("a node without a parent");
        if (r.count < 1 || r.begin < 0 || (int64_t)r.begin + r.count > h.n)
            return bad_file("a node segment out of range");
        depth = std::max(depth, r.level);
        if (r.first_child < 0) {
            if (r.first_child != -1 || r.count > h.leaf_size) return bad_file("a leaf");
            ++leaves;
            continue;
        }
        const int64_t c = r.first_child;
        if (c <= i || c + 1 >= nn) return bad_file("a child id");
        if (parented[(size_t)c] || parented[(size_t)c + 1]) return bad_file("a node with two parents");
        parented[(size_t)c] = parented[(size_t)c + 1] = 1;
        const NodeRec &s = L.node[(size_t)c], &d = L.node[(size_t)c + 1];
        if (s.level != r.level + 1 || d.level != r.level + 1) return bad_file("a child level");
        if (s.begin != r.begin || (int64_t)d.begin != (int64_t)r.begin + s.count ||
            (int64_t)s.count + d.count != r.count)
            return bad_file("children that do not split their parent");
    }
    if (depth != h.depth) return bad_file("depth");
    if (leaves != h.n_leaves) return bad_file("leaf count");
    std::vector<uint8_t> seen((size_t)h.n, 0);
    for (uint32_t v : L.perm) {
        if ((int64_t)v >= h.n || seen[v]) return bad_file("permutation");
        seen[v] = 1;
    }
    return DT_OK;
}

// Reads and checks an index file into *L.  No device work.
int read_index(const char *path, int64_t n, LoadedIndex *L)
{
    File f;
    f.f = std::fopen(path, "rb");
    if (!f.f) return io_error("cannot open for reading", path);
    IndexFileHeader &h = L->h;
    if (std::fread(&h, sizeof(h), 1, f.f) != 1) return bad_file("short header");
    if (std::memcmp(h.magic, kMagic, 8) != 0) return bad_file("not an index file");
    if (h.version != kVersion || h.header_bytes != sizeof(h)) return bad_file("version");
    if (h.reserved != 0 || h.reserved2 != 0) return bad_file("reserved fields");
    if (h.n != n) return bad_file("built over " + std::to_string(h.n) + " descriptors, not " + std::to_string(n));
    if (h.n < 1 || h.n > DT_MAX_N - 65536) return bad_file("size");
    if (h.n_nodes < 1 || h.n_nodes > 2 * h.n) return bad_file("node count");
    if (h.leaf_size < 1 || h.leaf_size > 4096 || (h.use_and != 0 && h.use_and != 1))
        return bad_file("parameters");
    if (h.depth < 0 || h.depth >= h.n_nodes || h.n_leaves < 1 || h.n_leaves > h.n_nodes)
        return bad_file("shape");
    const int64_t nn = h.n_nodes;
    const int64_t payload = nn * (int64_t)sizeof(NodeRec) + nn * kWords * 8 * (1 + h.use_and) + h.n * 4;
    if (std::fseek(f.f, 0, SEEK_END) != 0) return io_error("cannot seek", path);
    const long long size = (long long)std::ftell(f.f);
    if (size != (long long)(sizeof(h) + payload + 8)) return bad_file("file size");
    if (std::fseek(f.f, (long)sizeof(h), SEEK_SET) != 0) return io_error("cannot seek", path);
    L->node.resize((size_t)nn);
    L->img.resize((size_t)nn * kWords);
    L->aimg.resize(h.use_and ? (size_t)nn * kWords : 0);
    L->perm.resize((size_t)h.n);
    Checksum ck;
    auto get = [&](void *p, size_t len) {
        if (len && std::fread(p, 1, len, f.f) != len) return false;
        ck.bytes(p, len);
        return true;
    };
    uint64_t sum = 0;
    if (!get(L->node.data(), L->node.size() * sizeof(NodeRec)) || !get(L->img.data(), L->img.size() * 8) ||
        !get(L->aimg.data(), L->aimg.size() * 8) || !get(L->perm.data(), L->perm.size() * 4) ||
        std::fread(&sum, 8, 1, f.f) != 1)
        return io_error("read failed", path);
    if (ck.finish() != sum) return bad_file("checksum");
    return check_tree(*L);
}

// One warp per node (a lane owns 16 bytes of each image): a leaf's stored
// images must equal the OR and AND of its rows of the tree-ordered
// database, an inner node's the OR and AND of its two children's stored
// images.  By induction from the leaves every image is then exactly that of
// its node's descriptors.  The tree's shape was checked on the host, so
// every segment and child id is in range.  Sets *bad on any difference.
__global__ void check_images_kernel(const NodeRec *__restrict__ node, int64_t n_nodes,
                                    const uint64_t *__restrict__ db_tree,
                                    const uint64_t *__restrict__ or_img,
                                    const uint64_t *__restrict__ and_img, uint32_t *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; i < n_nodes; i += stride) {
        const NodeRec r = node[i];
        uint4 o, a;
        if (r.first_child < 0) {
            o = make_uint4(0u, 0u, 0u, 0u);
            a = make_uint4(~0u, ~0u, ~0u, ~0u);
            for (int j = 0; j < r.count; ++j) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(db_tree + ((int64_t)r.begin + j) * kWords) + lane);
                o.x |= v.x; o.y |= v.y; o.z |= v.z; o.w |= v.w;
                a.x &= v.x; a.y &= v.y; a.z &= v.z; a.w &= v.w;
            }
        } else {
            const int64_t c = r.first_child;
            const uint4 s0 = __ldg(reinterpret_cast<const uint4 *>(or_img + c * kWords) + lane);
            const uint4 s1 = __ldg(reinterpret_cast<const uint4 *>(or_img + (c + 1) * kWords) + lane);
            o = make_uint4(s0.x | s1.x, s0.y | s1.y, s0.z | s1.z, s0.w | s1.w);
            if (and_img) {
                const uint4 t0 = __ldg(reinterpret_cast<const uint4 *>(and_img + c * kWords) + lane);
                const uint4 t1 = __ldg(reinterpret_cast<const uint4 *>(and_img + (c + 1) * kWords) + lane);
                a = make_uint4(t0.x & t1.x, t0.y & t1.y, t0.z & t1.z, t0.w & t1.w);
            }
        }
        const uint4 so = __ldg(reinterpret_cast<const uint4 *>(or_img + i * kWords) + lane);
        bool diff = so.x != o.x || so.y != o.y || so.z != o.z || so.w != o.w;
        if (and_img) {
            const uint4 sa = __ldg(reinterpret_cast<const uint4 *>(and_img + i * kWords) + lane);
            diff = diff || sa.x != a.x || sa.y != a.y || sa.z != a.z || sa.w != a.w;
        }
        if (__any_sync(0xffffffffu, diff) && lane == 0) atomicOr(bad, 1u);
    }
}

int check_images(const dt_index *ix, cudaStream_t s)
{
    Scratch scratch(s);
    uint32_t *bad = nullptr;
    DT_CUDA_TRY(scratch.alloc(&bad, 4));
    DT_CUDA_TRY(cudaMemsetAsync(bad, 0, 4, s));
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((ix->n_nodes + 7) / 8, (int64_t)sm_count() * 16));
    check_images_kernel<<<(unsigned)blocks, 256, 0, s>>>(ix->node, ix->n_nodes, ix->db_tree, ix->or_img,
                                                         ix->and_img, bad);
    DT_CUDA_TRY(cudaGetLastError());
    uint32_t h = 0;
    DT_CUDA_TRY(cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, s));
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) return bad_file("node images do not match the database rows (a different database, "
                           "or its rows in another order, than the index was built over)");
    return DT_OK;
}

int upload_index(const LoadedIndex &L, const uint64_t *d_db, cudaStream_t s, dt_index **out)
{
    dt_index *ix = new dt_index();
    struct Guard {
        dt_index *&p;
        ~Guard()
        {
            if (p) dt_free(p);
        }
    } guard{ix};
    const IndexFileHeader &h = L.h;
    DT_CUDA_TRY(cudaGetDevice(&ix->device));
    ix->n = h.n;
    ix->n_nodes = h.n_nodes;
    ix->n_leaves = h.n_leaves;
    ix->depth = h.depth;
    ix->leaf_size = h.leaf_size;
    ix->use_and = h.use_and;
    DT_CUDA_TRY(cudaMalloc((void **)&ix->node, L.node.size() * sizeof(NodeRec)));
    DT_CUDA_TRY(cudaMemcpy(ix->node, L.node.data(), L.node.size() * sizeof(NodeRec), cudaMemcpyHostToDevice));
    DT_CUDA_TRY(cudaMalloc((void **)&ix->or_img, L.img.size() * 8));
    DT_CUDA_TRY(cudaMemcpy(ix->or_img, L.img.data(), L.img.size() * 8, cudaMemcpyHostToDevice));
    if (h.use_and) {
        DT_CUDA_TRY(cudaMalloc((void **)&ix->and_img, L.aimg.size() * 8));
        DT_CUDA_TRY(cudaMemcpy(ix->and_img, L.aimg.data(), L.aimg.size() * 8, cudaMemcpyHostToDevice));
    }
    DT_CUDA_TRY(cudaMalloc((void **)&ix->perm, L.perm.size() * 4));
    DT_CUDA_TRY(cudaMemcpy(ix->perm, L.perm.data(), L.perm.size() * 4, cudaMemcpyHostToDevice));
    int rc = fill_index_rows(d_db, ix, s);
    if (rc != DT_OK) return rc;
    rc = check_images(ix, s);
    if (rc != DT_OK) return rc;
    *out = ix;
    ix = nullptr;                      // ownership passes to the caller
    return DT_OK;
}

bool device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (p == nullptr || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace dtk

using namespace dtk;

extern "C" {

int dt_save(const dt_index *index, const char *path)
{
    DT_CHECK_ARG(index != nullptr && path != nullptr, "index and path must not be NULL");
    return save_index(index, path);
}

int dt_load(const char *path, const uint64_t *d_db, int64_t n, void *stream, dt_index **out)
{
    DT_CHECK_ARG(out != nullptr && path != nullptr, "path and out must not be NULL");
    *out = nullptr;
    DT_CHECK_ARG(n >= 1 && n <= DT_MAX_N - 65536, "n out of range");
    LoadedIndex L;
    const int rc = read_index(path, n, &L);
    if (rc != DT_OK) return rc;
    DT_CHECK_ARG(device_pointer(d_db) && aligned16(d_db), "d_db must be a non-null device pointer");
    return upload_index(L, d_db, (cudaStream_t)stream, out);
}

}  // extern "C"
