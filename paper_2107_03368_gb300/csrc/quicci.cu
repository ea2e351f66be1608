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
// Work: every triangle is tested against every point (cheap rejection by the
// triangle's bounding sphere against the support cylinder); triangles are
// pre-packed as three vertices plus a bounding sphere, 64 bytes, and read
// through the read-only cache by all warps.  Arithmetic is FP32.
#include <algorithm>
#include <cmath>

#include "dt_internal.cuh"

namespace dtk {
namespace {

constexpr int QN = 64;            // layers, circles per layer
constexpr int kQThreads = 128;    // threads per CTA, one CTA per point
constexpr int kQWarps = kQThreads / 32;
constexpr int kQBlocksPerSm = 8;  // 64 registers per thread
constexpr size_t kQSmem = (size_t)QN * QN * sizeof(int);

struct PackedTri {
    float4 v0, v1, v2;            // xyz, w unused
    float4 sphere;                // centre xyz, radius (negative: skip)
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

// One CTA per oriented point (persistent over points): its threads take the
// triangles in turn and add their segments' count changes to the point's
// 64 x 64 counters in shared memory; the four warps then turn 16 layers each
// into descriptor words.
__global__ void __launch_bounds__(kQThreads, kQBlocksPerSm)
quicci_kernel(const PackedTri *__restrict__ tris, int64_t nt, const float *__restrict__ points,
              const float *__restrict__ normals, int64_t np, float R, int modified,
              uint64_t *__restrict__ out)
{
    extern __shared__ __align__(16) int cnt[];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const float step = R / QN, inv_step = QN / R;
    const float R2 = R * R;
    for (int64_t j = blockIdx.x; j < np; j += gridDim.x) {
        for (int i = tid; i < QN * QN / 4; i += kQThreads) reinterpret_cast<int4 *>(cnt)[i] = make_int4(0, 0, 0, 0);
        __syncthreads();
        const float3 p = make_float3(points[j * 3], points[j * 3 + 1], points[j * 3 + 2]);
        float3 n = make_float3(normals[j * 3], normals[j * 3 + 1], normals[j * 3 + 2]);
        const float len = sqrtf(dot3(n, n));
        if (len > 0.f) {
            n = make_float3(n.x / len, n.y / len, n.z / len);
            for (int64_t t = tid; t < nt; t += kQThreads) {
                const float4 sp = __ldg(&tris[t].sphere);
                if (sp.w < 0.f) continue;
                const float3 rc = sub3(make_float3(sp.x, sp.y, sp.z), p);
                const float zc = dot3(rc, n);
                if (fabsf(zc) - sp.w > R) continue;
                const float3 qc = axpy3(-zc, n, rc);
                const float rad = sqrtf(dot3(qc, qc)) - sp.w;
                if (rad > 0.f && rad * rad > R2) continue;
                const float4 a4 = __ldg(&tris[t].v0), b4 = __ldg(&tris[t].v1), c4 = __ldg(&tris[t].v2);
                float z[3];
                float3 q[3];
                const float3 rel[3] = {sub3(make_float3(a4.x, a4.y, a4.z), p),
                                       sub3(make_float3(b4.x, b4.y, b4.z), p),
                                       sub3(make_float3(c4.x, c4.y, c4.z), p)};
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    z[i] = dot3(rel[i], n);
                    q[i] = axpy3(-z[i], n, rel[i]);
                }
                const float zmin = fminf(z[0], fminf(z[1], z[2])), zmax = fmaxf(z[0], fmaxf(z[1], z[2]));
                // layers with z_l in (zmin, zmax], widened by one on each side;
                // the exact side test below decides
                int l0 = (int)floorf((zmin + R) * (0.5f * inv_step) - 0.5f);
                int l1 = (int)ceilf((zmax + R) * (0.5f * inv_step) - 0.5f);
                l0 = max(l0, 0);
                l1 = min(l1, QN - 1);
                for (int l = l0; l <= l1; ++l) {
                    const float zl = -R + (2.f * l + 1.f) * step;
                    const bool b0 = z[0] < zl, b1 = z[1] < zl, b2 = z[2] < zl;
                    const int nb = (int)b0 + (int)b1 + (int)b2;
                    if (nb == 0 || nb == 3) continue;
                    // the two crossing edges, in edge order (0,1), (1,2), (2,0);
                    // the vertex alone on its side starts both of them
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
    DT_CUDA_TRY(allow_smem((const void *)quicci_kernel, (int)kQSmem));
    const int64_t blocks = std::min<int64_t>(n_points, (int64_t)sm_count() * kQBlocksPerSm);
    quicci_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), kQThreads, kQSmem, s>>>(
        packed, n_triangles, d_points, d_normals, n_points, support_radius, modified ? 1 : 0, d_out);
    DT_CUDA_TRY(cudaGetLastError());
    // the packed triangles are freed on the stream after the kernel
    return DT_OK;
}

}  // namespace dtk
