// quicci.cu — QUICCI descriptors (§2.2) of oriented points on a triangle
// mesh, and the modified QUICCI of §5 for partial query meshes.
//
// Geometry: the point p and its unit normal n define an axis; layer l is the
// plane at height z_l = -R + (2l + 1) R / 64 along n, circle c of a layer
// has radius r_c = (c + 1) R / 64 about the axis, and the circle below c = 0
// has radius 0.  Bit (l, c) is set iff the number of points where circle c
// meets the mesh differs from that of circle c - 1 (by at least 2 for the
// modified QUICCI).
//
// A layer plane cuts a triangle in a segment (from the two edges whose ends
// lie on different sides; "below" is height < z_l).  With a and b the
// segment's ends as offsets from the axis, the distance from the axis along
// the segment is convex, smallest (dm) at the closest point; circle r meets
// the segment once on each side of that point with dm < r <= that side's end
// distance.  So a segment changes the count of circle c by +1 at the first
// circle beyond dm and by -1 at the first circle beyond each end distance:
// the first circle with radius > x is c(x) = floor(x * 64 / R).
// A CTA owns one point and accumulates these signed changes, per (layer,
// circle), in shared memory; the bit is then just "change != 0" (or
// |change| >= 2).
//
// Work: every triangle is tested against every point, in two levels.  The
// triangles are packed (three vertices and a bounding sphere, 64 bytes) and
// sorted along a Morton curve of their centroids, so that each run of 32
// consecutive triangles (a group) is a compact patch with a bounding sphere
// of its own; a warp rejects a whole group against the point's support
// cylinder with one test, and only the groups that pass are tested triangle
// by triangle, one per lane.  Counts are integer sums, so the order in which
// triangles are visited changes nothing.  Arithmetic is FP32.
#include <algorithm>
#include <climits>
#include <cmath>

#include "dt_internal.cuh"
#include "sort_util.cuh"

namespace dtk {
namespace {

constexpr int QN = 64;            // layers, circles per layer
constexpr int kQThreads = 128;    // threads per CTA, one CTA per point
constexpr int kQWarps = kQThreads / 32;
constexpr int kQBlocksPerSm = 8;  // 64 registers per thread
constexpr int kQueue = 64;        // surviving triangles waiting per warp
constexpr size_t kQSmem = (size_t)QN * QN * sizeof(int) + (size_t)kQWarps * kQueue * sizeof(int);
constexpr int kGroup = 32;        // triangles per group (one per lane)

struct PackedTri {
    float4 v0, v1, v2;            // xyz, w unused
    float4 sphere;                // centre xyz, radius (negative: a bad vertex id, call rejected)
};

// Gathers each triangle's vertices and bounding sphere; flags ids out of range.
__global__ void pack_triangles_kernel(const float *__restrict__ vertices, int64_t nv,
                                      const int32_t *__restrict__ tris, int64_t nt,
                                      PackedTri *__restrict__ out, int *__restrict__ bad)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; t < nt; t += stride) {
        float3 v[3];
        bool ok = true;
        for (int i = 0; i < 3; ++i) {
            const int32_t id = tris[t * 3 + i];
            if (id < 0 || id >= nv) {
                ok = false;
                v[i] = make_float3(0.f, 0.f, 0.f);
                continue;
            }
            const float *vp = vertices + (int64_t)id * 3;
            v[i] = make_float3(vp[0], vp[1], vp[2]);
        }
        PackedTri p;
        p.v0 = make_float4(v[0].x, v[0].y, v[0].z, 0.f);
        p.v1 = make_float4(v[1].x, v[1].y, v[1].z, 0.f);
        p.v2 = make_float4(v[2].x, v[2].y, v[2].z, 0.f);
        const float cx = (v[0].x + v[1].x + v[2].x) / 3.f, cy = (v[0].y + v[1].y + v[2].y) / 3.f,
                    cz = (v[0].z + v[1].z + v[2].z) / 3.f;
        float r2 = 0.f;
        for (int i = 0; i < 3; ++i) {
            const float dx = v[i].x - cx, dy = v[i].y - cy, dz = v[i].z - cz;
            r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
        }
        // widened by a relative margin so rounding never rejects a triangle
        // that reaches the support cylinder
        p.sphere = make_float4(cx, cy, cz, ok ? sqrtf(r2) * 1.0001f + 1e-3f : -1.f);
        out[t] = p;
        if (!ok) atomicExch(bad, 1);
    }
}

// Order-preserving map of a float to a signed int (for atomic min / max).
__device__ __forceinline__ int ordered(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void box_init_kernel(int *box)
{
    if (threadIdx.x < 3) box[threadIdx.x] = INT_MAX;
    else if (threadIdx.x < 6) box[threadIdx.x] = INT_MIN;
}

// Bounding box of the triangle centres: box[0..2] min, box[3..5] max, as
// ordered ints (box_init_kernel sets the starting values).
__global__ void centre_box_kernel(const PackedTri *__restrict__ tris, int64_t nt, int *__restrict__ box)
{
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; t < nt; t += stride) {
        const float4 c = tris[t].sphere;
        const int o[3] = {ordered(c.x), ordered(c.y), ordered(c.z)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = min(lo[k], o[k]);
            hi[k] = max(hi[k], o[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], d));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], d));
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            atomicMin(&box[k], lo[k]);
            atomicMax(&box[3 + k], hi[k]);
        }
}

// Spreads the low 10 bits of x to every third bit (bit i -> bit 3i).
__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// Morton key (8 bits per axis, 24 in all) of each triangle centre within the box.
__global__ void morton_kernel(const PackedTri *__restrict__ tris, int64_t nt, const int *__restrict__ box,
                              uint32_t *__restrict__ key, uint32_t *__restrict__ val)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float lo[3], scale[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = unordered(box[k]);
        const float ext = unordered(box[3 + k]) - lo[k];
        scale[k] = ext > 0.f ? 255.f / ext : 0.f;
    }
    for (; t < nt; t += stride) {
        const float4 c = tris[t].sphere;
        const float cc[3] = {c.x, c.y, c.z};
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float f = fminf(fmaxf((cc[k] - lo[k]) * scale[k], 0.f), 255.f);
            m |= spread3((uint32_t)f) << k;
        }
        key[t] = m;
        val[t] = (uint32_t)t;
    }
}

__global__ void gather_tris_kernel(const PackedTri *__restrict__ in, const uint32_t *__restrict__ order,
                                   int64_t nt, PackedTri *__restrict__ out)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; t < nt; t += stride) out[t] = in[order[t]];
}

// A warp per group of kGroup consecutive triangles: a sphere holding all of
// their spheres (centre: mean of their centres).
__global__ void group_sphere_kernel(const PackedTri *__restrict__ tris, int64_t nt, int64_t n_groups,
                                    float4 *__restrict__ groups)
{
    const int lane = threadIdx.x & 31;
    int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; g < n_groups; g += nw) {
        const int64_t t = g * kGroup + lane;
        const bool have = t < nt;
        const float4 c = have ? tris[t].sphere : make_float4(0.f, 0.f, 0.f, 0.f);
        float sx = c.x, sy = c.y, sz = c.z, cntf = have ? 1.f : 0.f;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, d);
            sy += __shfl_xor_sync(0xffffffffu, sy, d);
            sz += __shfl_xor_sync(0xffffffffu, sz, d);
            cntf += __shfl_xor_sync(0xffffffffu, cntf, d);
        }
        const float cx = sx / cntf, cy = sy / cntf, cz = sz / cntf;
        float r = 0.f;
        if (have) {
            const float dx = c.x - cx, dy = c.y - cy, dz = c.z - cz;
            r = sqrtf(dx * dx + dy * dy + dz * dz) + c.w;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, d));
        // widened like the triangles' spheres, so rounding never rejects a
        // group that reaches the support cylinder
        if (lane == 0) groups[g] = make_float4(cx, cy, cz, r * 1.0001f + 1e-3f);
    }
}

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 axpy3(float s, float3 x, float3 y)
{
    return make_float3(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z));
}

// One of three values by index, without indexing an array (which would
// place the array in local memory).
template <class T> __device__ __forceinline__ T pick3(int i, T a, T b, T c)
{
    return i == 0 ? a : (i == 1 ? b : c);
}

// First circle with radius > x (QN: none).
__device__ __forceinline__ int circle_after(float x, float inv_step)
{
    const float f = floorf(x * inv_step);
    return f >= (float)QN ? QN : (int)f;
}

__device__ __forceinline__ void add_branch(int *row, float dm, float end, float inv_step)
{
    if (!(end > dm)) return;
    const int c0 = circle_after(dm, inv_step);
    if (c0 >= QN) return;
    atomicAdd(&row[c0], 1);
    const int c1 = circle_after(end, inv_step);
    if (c1 < QN) atomicAdd(&row[c1], -1);
}

// Whether a sphere (centre xyz, radius w) reaches the support cylinder of the
// point p with unit axis n: |height| <= R + radius and distance from the
// axis <= R + radius.
__device__ __forceinline__ bool reaches(float4 sp, float3 p, float3 n, float R, float R2)
{
    const float3 rc = sub3(make_float3(sp.x, sp.y, sp.z), p);
    const float zc = dot3(rc, n);
    if (fabsf(zc) - sp.w > R) return false;
    const float3 qc = axpy3(-zc, n, rc);
    const float rad = sqrtf(dot3(qc, qc)) - sp.w;
    return !(rad > 0.f && rad * rad > R2);
}

// Adds the count changes of triangle t's layer segments to the counters.
__device__ __forceinline__ void add_triangle(const PackedTri *__restrict__ tris, int64_t t, float3 p,
                                             float3 n, float R, float step, float inv_step, int *cnt)
{
    const float4 a4 = __ldg(&tris[t].v0), b4 = __ldg(&tris[t].v1), c4 = __ldg(&tris[t].v2);
    float z[3];
    float3 q[3];
    const float3 rel[3] = {sub3(make_float3(a4.x, a4.y, a4.z), p), sub3(make_float3(b4.x, b4.y, b4.z), p),
                           sub3(make_float3(c4.x, c4.y, c4.z), p)};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        z[i] = dot3(rel[i], n);
        q[i] = axpy3(-z[i], n, rel[i]);
    }
    const float zmin = fminf(z[0], fminf(z[1], z[2])), zmax = fmaxf(z[0], fmaxf(z[1], z[2]));
    // layers with z_l in (zmin, zmax]: z_l > zmin iff l > x0 and z_l <= zmax
    // iff l <= x1; where rounding could put x0 or x1 on the wrong side of an
    // integer the range takes one more layer, and the exact side test below
    // decides
    const float x0 = (zmin + R) * (0.5f * inv_step) - 0.5f;
    const float x1 = (zmax + R) * (0.5f * inv_step) - 0.5f;
    const float f0 = floorf(x0), f1 = floorf(x1);
    int l0 = (int)f0 + (x0 - f0 > 1e-3f ? 1 : 0);
    int l1 = (int)f1 + (x1 - f1 > 1.f - 1e-3f ? 1 : 0);
    l0 = max(l0, 0);
    l1 = min(l1, QN - 1);
    for (int l = l0; l <= l1; ++l) {
        const float zl = -R + (2.f * l + 1.f) * step;
        const bool b0 = z[0] < zl, b1 = z[1] < zl, b2 = z[2] < zl;
        const int nb = (int)b0 + (int)b1 + (int)b2;
        if (nb == 0 || nb == 3) continue;
        // the two crossing edges both start at the vertex alone on its side
        const int solo = (b0 != b1) ? ((b0 != b2) ? 0 : 1) : 2;
        const int o1 = solo == 2 ? 0 : solo + 1, o2 = solo == 0 ? 2 : solo - 1;
        const float zs = pick3(solo, z[0], z[1], z[2]);
        const float3 qs = pick3(solo, q[0], q[1], q[2]);
        const float s1 = (zl - zs) / (pick3(o1, z[0], z[1], z[2]) - zs);
        const float s2 = (zl - zs) / (pick3(o2, z[0], z[1], z[2]) - zs);
        const float3 e0 = axpy3(s1, sub3(pick3(o1, q[0], q[1], q[2]), qs), qs);
        const float3 e1 = axpy3(s2, sub3(pick3(o2, q[0], q[1], q[2]), qs), qs);
        const float3 d = sub3(e1, e0);
        const float dd = dot3(d, d);
        const float d0 = sqrtf(dot3(e0, e0)), d1 = sqrtf(dot3(e1, e1));
        float ts = dd > 0.f ? -dot3(e0, d) / dd : 0.f;
        ts = fminf(fmaxf(ts, 0.f), 1.f);
        const float3 cp = axpy3(ts, d, e0);
        const float dm = fminf(sqrtf(dot3(cp, cp)), fminf(d0, d1));
        int *row = cnt + l * QN;
        add_branch(row, dm, d0, inv_step);
        add_branch(row, dm, d1, inv_step);
    }
}

// One CTA per oriented point (persistent over points).  Each warp takes 32
// triangle groups at a time, one per lane (interleaved with the other
// warps' groups), and tests them against the support cylinder; for every
// group that passed (a warp-wide ballot), its lanes test the group's
// triangles, one each, and push the survivors onto the warp's queue in
// shared memory; whenever 32 are waiting, every lane takes one and adds its
// segments' count changes to the point's 64 x 64 counters, so the costly
// part runs on full warps.  The four warps then turn 16 layers each into
// descriptor words.
__global__ void __launch_bounds__(kQThreads, kQBlocksPerSm)
quicci_kernel(const PackedTri *__restrict__ tris, int64_t nt, const float4 *__restrict__ groups,
              int64_t n_groups, const float *__restrict__ points, const float *__restrict__ normals,
              int64_t np, float R, int modified, uint64_t *__restrict__ out)
{
    extern __shared__ __align__(16) int cnt[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int *queue = cnt + QN * QN + w * kQueue;
    const uint32_t below = (1u << lane) - 1u;
    const float step = R / QN, inv_step = QN / R;
    const float R2 = R * R;
    for (int64_t j = blockIdx.x; j < np; j += gridDim.x) {
        for (int i = tid; i < QN * QN / 4; i += kQThreads) reinterpret_cast<int4 *>(cnt)[i] = make_int4(0, 0, 0, 0);
        __syncthreads();
        const float3 p = make_float3(points[j * 3], points[j * 3 + 1], points[j * 3 + 2]);
        float3 n = make_float3(normals[j * 3], normals[j * 3 + 1], normals[j * 3 + 2]);
        const float len = sqrtf(dot3(n, n));
        int qn = 0;                      // triangles waiting in this warp's queue
        if (len > 0.f) {
            n = make_float3(n.x / len, n.y / len, n.z / len);
            // lane i of warp w tests group g0 + i * kQWarps + w: neighbouring
            // groups (often reached together) go to different warps
            for (int64_t g0 = 0; g0 < n_groups; g0 += (int64_t)kQWarps * 32) {
                const int64_t g = g0 + (int64_t)lane * kQWarps + w;
                const bool hit = g < n_groups && reaches(__ldg(&groups[g]), p, n, R, R2);
                uint32_t mask = __ballot_sync(0xffffffffu, hit);
                while (mask) {
                    const int b = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int64_t t = (g0 + (int64_t)b * kQWarps + w) * kGroup + lane;
                    const bool live = t < nt && reaches(__ldg(&tris[t].sphere), p, n, R, R2);
                    const uint32_t lm = __ballot_sync(0xffffffffu, live);
                    if (live) queue[qn + __popc(lm & below)] = (int)t;
                    qn += __popc(lm);
                    __syncwarp();
                    if (qn >= 32) {
                        add_triangle(tris, queue[lane], p, n, R, step, inv_step, cnt);
                        qn -= 32;
                        __syncwarp();
                        const int moved = lane < qn ? queue[32 + lane] : 0;
                        __syncwarp();
                        if (lane < qn) queue[lane] = moved;
                        __syncwarp();
                    }
                }
            }
            if (lane < qn) add_triangle(tris, queue[lane], p, n, R, step, inv_step, cnt);
        }
        __syncthreads();
        // warp w: layers 16w .. 16w + 15, lanes hold circles lane and lane + 32
        for (int l = w * (QN / kQWarps); l < (w + 1) * (QN / kQWarps); ++l) {
            const int v0 = cnt[l * QN + lane], v1 = cnt[l * QN + 32 + lane];
            const bool s0 = modified ? (v0 >= 2 || v0 <= -2) : v0 != 0;
            const bool s1 = modified ? (v1 >= 2 || v1 <= -2) : v1 != 0;
            const uint32_t lo = __ballot_sync(0xffffffffu, s0), hi = __ballot_sync(0xffffffffu, s1);
            if (lane == 0) out[j * QN + l] = ((uint64_t)hi << 32) | lo;
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace dtk

namespace dtk {

int launch_quicci(const float *d_vertices, int64_t n_vertices, const int32_t *d_triangles,
                  int64_t n_triangles, const float *d_points, const float *d_normals,
                  int64_t n_points, float support_radius, int modified, uint64_t *d_out,
                  cudaStream_t s)
{
    Scratch scratch(s);
    PackedTri *packed = nullptr;
    int *bad = nullptr;
    DT_CUDA_TRY(scratch.alloc(&bad, sizeof(int)));
    DT_CUDA_TRY(scratch.alloc(&packed, (size_t)std::max<int64_t>(n_triangles, 1) * sizeof(PackedTri)));
    DT_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (n_triangles > 0) {
        pack_triangles_kernel<<<(unsigned)std::min<int64_t>((n_triangles + 255) / 256, 65535), 256, 0, s>>>(
            d_vertices, n_vertices, d_triangles, n_triangles, packed, bad);
        DT_CUDA_TRY(cudaGetLastError());
    }
    int h_bad = 0;
    DT_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    DT_CHECK_ARG(!h_bad, "a triangle vertex id is outside [0, n_vertices)");
    // spatial order: Morton keys of the centres, stable radix sort, gather
    const int64_t n_groups = (n_triangles + kGroup - 1) / kGroup;
    PackedTri *sorted = nullptr;
    float4 *groups = nullptr;
    uint32_t *key = nullptr, *val = nullptr, *key2 = nullptr, *val2 = nullptr, *hist = nullptr;
    int *box = nullptr;
    if (n_triangles > 0) {
        const int64_t nt = n_triangles;
        DT_CUDA_TRY(scratch.alloc(&sorted, (size_t)nt * sizeof(PackedTri)));
        DT_CUDA_TRY(scratch.alloc(&groups, (size_t)n_groups * sizeof(float4)));
        DT_CUDA_TRY(scratch.alloc(&key, (size_t)nt * 4));
        DT_CUDA_TRY(scratch.alloc(&val, (size_t)nt * 4));
        DT_CUDA_TRY(scratch.alloc(&key2, (size_t)nt * 4));
        DT_CUDA_TRY(scratch.alloc(&val2, (size_t)nt * 4));
        DT_CUDA_TRY(scratch.alloc(&hist, (size_t)radix_tiles(nt) * 256 * 4));
        DT_CUDA_TRY(scratch.alloc(&box, 6 * sizeof(int)));
        box_init_kernel<<<1, 32, 0, s>>>(box);
        const unsigned gb = (unsigned)std::min<int64_t>((nt + 255) / 256, 4096);
        centre_box_kernel<<<gb, 256, 0, s>>>(packed, nt, box);
        morton_kernel<<<gb, 256, 0, s>>>(packed, nt, box, key, val);
        DT_CUDA_TRY(cudaGetLastError());
        DT_CUDA_TRY(radix_sort_pairs(&key, &val, &key2, &val2, nt, 24, hist, s));
        gather_tris_kernel<<<gb, 256, 0, s>>>(packed, val, nt, sorted);
        group_sphere_kernel<<<(unsigned)std::min<int64_t>((n_groups + 7) / 8, 8192), 256, 0, s>>>(
            sorted, nt, n_groups, groups);
        DT_CUDA_TRY(cudaGetLastError());
    }
    DT_CUDA_TRY(allow_smem((const void *)quicci_kernel, (int)kQSmem));
    const int64_t blocks = std::min<int64_t>(n_points, (int64_t)sm_count() * kQBlocksPerSm);
    quicci_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), kQThreads, kQSmem, s>>>(
        sorted, n_triangles, groups, n_groups, d_points, d_normals, n_points, support_radius,
        modified ? 1 : 0, d_out);
    DT_CUDA_TRY(cudaGetLastError());
    // the packed triangles are freed on the stream after the kernel
    return DT_OK;
}

}  // namespace dtk
