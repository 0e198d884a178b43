// bvh_build.cu -- GPU BVH builder (Morton order, PLOC clustering) collapsed to an 8-wide BVH.
//
// The paper (§6) traced its scenes with OptiX and says nothing about the
// acceleration structure; this builder serves the scene S(n) of §2, Eq. 1.
// Steps, all on the device:
//  1. primitive boxes and centroids; scene and centroid bounds (atomic min/max
//     on order-preserving integer images of the floats);
//  2. 30-bit Morton codes of the centroids (10 bits per axis, in the cube of
//     the largest extent);
//  3. radix sort of (code, primitive) pairs (radix_sort.cu);
//  4. binary tree by PLOC (Meister and Bittner 2018): the primitives in
//     Morton order are clusters; each round every cluster finds the cluster
//     within 16 array positions whose union box has the least surface area,
//     mutual pairs merge (the new node gets the union box), and the array is
//     compacted by a prefix sum, until one cluster is left;
//  5. leaves renumbered in depth-first order, so that every subtree's
//     primitives are contiguous;
//  6. collapse to 8-wide nodes, one launch per level. Subtrees of <= LEAF_MAX
//     (3) primitives become leaves. Which binary nodes are opened into a wide
//     node's 8 slots follows the scene's policy: RCP_COLLAPSE_AREA repeatedly
//     opens the child of largest surface area that holds more than LEAF_MAX
//     primitives; RCP_COLLAPSE_SAH shares the slots out by a bottom-up dynamic
//     program over the binary tree that minimises the surface-area cost. Children
//     are placed in slots so that slot order approximates front-to-back order
//     per ray octant; child boxes are float32 bounds with a small outward pad
//     (tri_pad). Leaf primitives are copied into 48-byte records, contiguous
//     per node. Optionally (split_max > 1) long thin triangles first enter
//     as several clipped references (early split clipping, below); each keeps
//     its part of the triangle, so that a refit after a vertex update bounds
//     it by that part of the moved triangle.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "rcp_internal.cuh"
#include "scene.h"

namespace rcp {

size_t radix_sort_scratch_bytes(int64_t n);
rcp_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* alt_keys, uint32_t* alt_vals,
                            int64_t n, int bits, void* scratch, int* d_error, cudaStream_t stream);

namespace {

constexpr int BUILD_BLOCK = 256;
// Most primitives in one leaf slot. A leaf's meta byte holds count << 5 |
// offset with bit 7 clear (bit 7 marks an internal child), so count <= 3.
constexpr int LEAF_MAX = 3;
static_assert(LEAF_MAX >= 1 && LEAF_MAX <= 3, "a leaf's count must leave the meta byte's top bit clear");

__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bounds layout: [0..2] centroid min, [3..5] centroid max, [6..8] box min, [9..11] box max
__global__ void k_init_bounds(uint32_t* b) {
    const int i = threadIdx.x;
    if (i < 12) b[i] = ((i % 6) < 3) ? 0xffffffffu : 0u;
}

__device__ __forceinline__ void prim_box(const float* __restrict__ tri, const float* __restrict__ sph, int64_t T,
                                         int64_t id, float3& lo, float3& hi) {
    if (id < T) {
        const float* v = tri + 9 * id;
        lo = make_float3(fminf(fminf(v[0], v[3]), v[6]), fminf(fminf(v[1], v[4]), v[7]), fminf(fminf(v[2], v[5]), v[8]));
        hi = make_float3(fmaxf(fmaxf(v[0], v[3]), v[6]), fmaxf(fmaxf(v[1], v[4]), v[7]), fmaxf(fmaxf(v[2], v[5]), v[8]));
    } else {
        const float* s = sph + 4 * (id - T);
        const float r = fabsf(s[3]);
        lo = make_float3(__fsub_rd(s[0], r), __fsub_rd(s[1], r), __fsub_rd(s[2], r));
        hi = make_float3(__fadd_ru(s[0], r), __fadd_ru(s[1], r), __fadd_ru(s[2], r));
    }
}

// Outward pad of a triangle's stored boxes: 2^-12 of its box's extent plus
// 2^-18 of its coordinates' magnitude. The float ray-triangle test accepts
// hits up to a rounding error outside the true edges and vertices; a box that
// is exact at a vertex or an edge would let the walk skip such a hit that a
// test of every primitive accepts. The build's decisions (Morton codes,
// clustering, collapse) use the exact boxes; the boxes stored in the tree
// (leaf slots, and every node's box, refitted from the padded leaves) carry
// the pad. The scene's bounds (and its diameter) are those of the exact
// vertices.
// Float arithmetic rounded upwards (the pad) and outwards (the padded box):
// refits run it for every record of every frame, and double arithmetic is
// slow on this GPU.
__device__ __forceinline__ float tri_pad(const float3& lo, const float3& hi) {
    const float ext = __fadd_ru(__fadd_ru(__fsub_ru(hi.x, lo.x), __fsub_ru(hi.y, lo.y)), __fsub_ru(hi.z, lo.z));
    const float mag = fmaxf(fmaxf(fmaxf(fabsf(lo.x), fabsf(hi.x)), fmaxf(fabsf(lo.y), fabsf(hi.y))),
                            fmaxf(fabsf(lo.z), fabsf(hi.z)));
    return __fadd_ru(__fmul_ru(ext, 0x1p-12f), __fmul_ru(mag, 0x1p-18f));
}

__device__ __forceinline__ void pad_box(float pad, float3& lo, float3& hi) {
    lo = make_float3(__fsub_rd(lo.x, pad), __fsub_rd(lo.y, pad), __fsub_rd(lo.z, pad));
    hi = make_float3(__fadd_ru(hi.x, pad), __fadd_ru(hi.y, pad), __fadd_ru(hi.z, pad));
}

// The stored (padded) box of reference `ref`: its exact box (plo/phi),
// padded by the pad of its primitive when that is a triangle. ref_prim maps
// references to primitives (nullptr: references are the primitives).
__device__ __forceinline__ void padded_ref_box(const float4* plo, const float4* phi, const uint32_t* ref_prim,
                                               const float* tri, const float* sph, int64_t T, uint32_t ref,
                                               float3& lo, float3& hi) {
    const float4 l = plo[ref], h = phi[ref];
    lo = make_float3(l.x, l.y, l.z);
    hi = make_float3(h.x, h.y, h.z);
    const uint32_t prim = ref_prim ? ref_prim[ref] : ref;
    if ((int64_t)prim < T) {
        float3 tl, th;
        prim_box(tri, sph, T, prim, tl, th);
        pad_box(tri_pad(tl, th), lo, hi);
    }
}

__global__ void __launch_bounds__(BUILD_BLOCK) k_prim_bounds(const float* __restrict__ tri,
                                                             const float* __restrict__ sph, int64_t T, int64_t N,
                                                             float4* __restrict__ plo, float4* __restrict__ phi,
                                                             uint32_t* __restrict__ bounds) {
    __shared__ uint32_t sb[12];
    if (threadIdx.x < 12) sb[threadIdx.x] = ((threadIdx.x % 6) < 3) ? 0xffffffffu : 0u;
    __syncthreads();
    uint32_t mine[12];
    for (int a = 0; a < 12; ++a) mine[a] = ((a % 6) < 3) ? 0xffffffffu : 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float3 lo, hi;
        prim_box(tri, sph, T, i, lo, hi);
        plo[i] = make_float4(lo.x, lo.y, lo.z, 0.f);
        phi[i] = make_float4(hi.x, hi.y, hi.z, 0.f);
        const float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
        const float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
        for (int a = 0; a < 3; ++a) {
            mine[a] = min(mine[a], f2ord(c[a]));
            mine[3 + a] = max(mine[3 + a], f2ord(c[a]));
            mine[6 + a] = min(mine[6 + a], f2ord(l[a]));
            mine[9 + a] = max(mine[9 + a], f2ord(h[a]));
        }
    }
    for (int a = 0; a < 12; ++a) {
        if ((a % 6) < 3) atomicMin(&sb[a], mine[a]);
        else atomicMax(&sb[a], mine[a]);
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        if ((threadIdx.x % 6) < 3) atomicMin(&bounds[threadIdx.x], sb[threadIdx.x]);
        else atomicMax(&bounds[threadIdx.x], sb[threadIdx.x]);
    }
}

// 10 bits of each axis interleaved as ...x2y2z2 x1y1z1 x0y0z0 (x highest).
// Every axis is scaled by the box's largest extent (a cube over lo), not by
// its own: a flat scene (terrain, a forest floor) then keeps its thin axis in
// the low bits, so the top of the hierarchy splits the long axes and no node
// near the root spans the whole scene along them.
__device__ __forceinline__ uint32_t morton30(float x, float y, float z, const float* lo, const float* hi) {
    const float c[3] = {x, y, z};
    const float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        float u = ext > 0.f ? (c[a] - lo[a]) / ext : 0.f;
        int v = (int)(u * 1024.f);
        q[a] = (uint32_t)min(max(v, 0), 1023);
    }
    uint32_t code = 0;
    for (int b = 0; b < 10; ++b)
        code |= (((q[0] >> b) & 1u) << (3 * b + 2)) | (((q[1] >> b) & 1u) << (3 * b + 1)) | (((q[2] >> b) & 1u) << (3 * b));
    return code;
}

__global__ void k_morton(const float4* __restrict__ plo, const float4* __restrict__ phi, int64_t N,
                         const uint32_t* __restrict__ bounds, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = ord2f(bounds[a]);
        hi[a] = ord2f(bounds[3 + a]);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 l = plo[i], h = phi[i];
        keys[i] = morton30(0.5f * (l.x + h.x), 0.5f * (l.y + h.y), 0.5f * (l.z + h.z), lo, hi);
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_morton_points(const float* __restrict__ xyz, int64_t n, float l0, float l1, float l2, float h0,
                                float h1, float h2, uint32_t* __restrict__ codes) {
    const float lo[3] = {l0, l1, l2}, hi[3] = {h0, h1, h2};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        codes[i] = morton30(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lo, hi);
}

// ---- early split clipping (Ernst and Greiner 2007) ----
// A triangle whose box is large against its own area (long thin triangles,
// such as a cone's sides from apex to base) enters the build as several
// references: its box is halved at the midpoint of the longest axis, the
// triangle is clipped to each half, and the halves whose clipped part is
// still large are halved again, up to split_max references per triangle.
// Each reference is bounded by the box of its clipped part, rounded outwards,
// so the references' boxes together cover the triangle (stored with the pad
// of the whole triangle); every reference's leaf record is the whole
// triangle, so hits are exactly those of one record.
constexpr float SPLIT_RATIO = 4.f;  // split while box half-area > 4 x triangle area
constexpr int SPLIT_MAX = 8;

// Clipping below runs in float with explicit round-to-nearest intrinsics (no
// contraction left to the compiler), so that the counting and the writing
// kernels, and any other caller, compute bit-identical pieces. Its rounding,
// about 2^-23 of the coordinates and edges, sits far inside the pad that every
// stored box carries (2^-12 of the triangle's extent plus 2^-18 of its
// coordinates' magnitude). Double arithmetic runs at a small fraction of the
// float rate on this GPU: the double version took 58 % of the forest's build.

// Box of triangle v (3 vertices) clipped to [lo, hi] (Sutherland-Hodgman).
// False when the triangle misses the box.
__device__ bool clip_triangle_box(const float (&v)[3][3], const float lo[3], const float hi[3], float3& olo,
                                  float3& ohi) {
    float poly[10][3], tmp[10][3];
    int n = 3;
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) poly[i][a] = v[i][a];
    for (int a = 0; a < 3; ++a)
        for (int side = 0; side < 2; ++side) {
            const float b = side ? hi[a] : lo[a];
            int m = 0;
            for (int i = 0; i < n; ++i) {
                const float* p = poly[i];
                const float* q = poly[(i + 1) % n];
                const bool pin = side ? p[a] <= b : p[a] >= b;
                const bool qin = side ? q[a] <= b : q[a] >= b;
                if (pin) {
                    for (int c = 0; c < 3; ++c) tmp[m][c] = p[c];
                    ++m;
                }
                if (pin != qin) {  // p[a] != q[a]: they lie on either side of b
                    const float t = __fdiv_rn(__fsub_rn(b, p[a]), __fsub_rn(q[a], p[a]));
                    for (int c = 0; c < 3; ++c) tmp[m][c] = __fmaf_rn(t, __fsub_rn(q[c], p[c]), p[c]);
                    tmp[m][a] = b;  // on the plane exactly
                    ++m;
                }
            }
            n = m;
            if (n == 0) return false;
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) poly[i][c] = tmp[i][c];
        }
    float l[3] = {poly[0][0], poly[0][1], poly[0][2]}, h[3] = {poly[0][0], poly[0][1], poly[0][2]};
    for (int i = 1; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            l[c] = fminf(l[c], poly[i][c]);
            h[c] = fmaxf(h[c], poly[i][c]);
        }
    olo = make_float3(l[0], l[1], l[2]);
    ohi = make_float3(h[0], h[1], h[2]);
    return true;
}

// The references of triangle `id` (exact boxes, in emission order); returns
// their number. With rlo/rhi null it only counts; otherwise it writes at most
// `cap` of them. Counting and writing run the same steps, so they agree.
__device__ int split_triangle(const float* __restrict__ tri, uint32_t id, int max_refs, float4* __restrict__ rlo,
                              float4* __restrict__ rhi, int cap) {
    const float* f = tri + 9 * (int64_t)id;
    float v[3][3];
    for (int i = 0; i < 3; ++i)
        for (int a = 0; a < 3; ++a) v[i][a] = f[3 * i + a];
    // The split test compares areas in double, a few operations per triangle
    // and per piece: in float, the cross product of a long thin triangle's
    // edges loses digits and moves the decisions (measured: forest 2.7 %
    // slower). Only the clipping, the bulk of the work, runs in float.
    const double e1[3] = {(double)v[1][0] - v[0][0], (double)v[1][1] - v[0][1], (double)v[1][2] - v[0][2]};
    const double e2[3] = {(double)v[2][0] - v[0][0], (double)v[2][1] - v[0][1], (double)v[2][2] - v[0][2]};
    const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                 cz = e1[0] * e2[1] - e1[1] * e2[0];
    const double tri_area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    float sl[SPLIT_MAX][3], sh[SPLIT_MAX][3];
    int sp = 0, n_out = 0;
    for (int a = 0; a < 3; ++a) {
        sl[0][a] = fminf(fminf(f[a], f[3 + a]), f[6 + a]);
        sh[0][a] = fmaxf(fmaxf(f[a], f[3 + a]), f[6 + a]);
    }
    sp = 1;
    while (sp > 0) {
        --sp;
        const float l[3] = {sl[sp][0], sl[sp][1], sl[sp][2]}, h[3] = {sh[sp][0], sh[sp][1], sh[sp][2]};
        const double dx = (double)h[0] - l[0], dy = (double)h[1] - l[1], dz = (double)h[2] - l[2];
        const double box_area = dx * dy + dy * dz + dz * dx;
        // a split adds at most one box to the outstanding ones: keep <= max_refs
        if (tri_area <= 0.0 || n_out + sp + 2 > max_refs || box_area <= SPLIT_RATIO * tri_area) {
            if (rlo && n_out < cap) {
                rlo[n_out] = make_float4(l[0], l[1], l[2], 0.f);
                rhi[n_out] = make_float4(h[0], h[1], h[2], 0.f);
            }
            ++n_out;
            continue;
        }
        const int ax = (dx >= dy && dx >= dz) ? 0 : (dy >= dz ? 1 : 2);
        const float mid = __fmul_rn(0.5f, __fadd_rn(l[ax], h[ax]));
        const int sp0 = sp;
        for (int half = 1; half >= 0; --half) {
            float cl[3] = {l[0], l[1], l[2]}, ch[3] = {h[0], h[1], h[2]};
            if (half) cl[ax] = mid;
            else ch[ax] = mid;
            float3 ol, oh;
            if (clip_triangle_box(v, cl, ch, ol, oh)) {
                sl[sp][0] = ol.x, sl[sp][1] = ol.y, sl[sp][2] = ol.z;
                sh[sp][0] = oh.x, sh[sp][1] = oh.y, sh[sp][2] = oh.z;
                ++sp;
            }
        }
        if (sp == sp0) {  // neither half kept a part (rounding): keep the box itself
            if (rlo && n_out < cap) {
                rlo[n_out] = make_float4(l[0], l[1], l[2], 0.f);
                rhi[n_out] = make_float4(h[0], h[1], h[2], 0.f);
            }
            ++n_out;
        }
    }
    return n_out;
}

// References per primitive (spheres: 1).
__global__ void k_split_count(const float* __restrict__ tri, int64_t T, int64_t N, int max_refs,
                              unsigned long long* __restrict__ counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        counts[i] = i < T ? (unsigned long long)split_triangle(tri, (uint32_t)i, max_refs, nullptr, nullptr, 0) : 1ull;
}

// Write the references at their offsets (exclusive prefix sum of the counts,
// R in all). A primitive writes at most the slots its count gave it; a count
// that differs sets *err and the build fails.
__global__ void k_split_write(const float* __restrict__ tri, int64_t T, int64_t N, int max_refs,
                              const unsigned long long* __restrict__ offsets, int64_t R,
                              const float4* __restrict__ plo, const float4* __restrict__ phi,
                              float4* __restrict__ rlo, float4* __restrict__ rhi, uint32_t* __restrict__ rprim,
                              int* __restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)offsets[i];
        const int cap = (int)((i + 1 < N ? (int64_t)offsets[i + 1] : R) - o);
        int n = 1;
        if (i < T) {
            n = split_triangle(tri, (uint32_t)i, max_refs, rlo + o, rhi + o, cap);
            if (n != cap) {
                atomicAdd(err, 1);
                n = min(n, cap);
            }
        } else {
            rlo[o] = plo[i];
            rhi[o] = phi[i];
        }
        for (int k = 0; k < n; ++k) rprim[o + k] = (uint32_t)i;
    }
}

// ---- parts of split references, for refits ----
// A reference of a split triangle stands for the part of the triangle inside
// its box. That part is kept as a convex polygon in the triangle's own
// coordinates (u, v), with p = v0 + u (v1 - v0) + v (v2 - v0). Every point of
// the triangle moves with its (u, v) when the vertices change, so a refit
// maps the polygon through the moved vertices and bounds the reference by
// exactly its part of the moved triangle; the parts of a triangle still cover
// it, whatever the motion.
// A vertex is stored as u and v in 16-bit fixed point (u = q / 65535), one
// 32-bit word: u in the low half. Rounding to nearest moves a mapped vertex by
// at most 2^-17 of each edge, 2^-16 of the triangle's extent, well inside the
// 2^-12 extent pad of the triangle's boxes. A record's part fills PART_MAX
// words; the word PART_END (u = v = 1, impossible in a triangle) ends a part
// of fewer vertices, and a first word PART_END means no part (the whole
// primitive).
constexpr int PART_MAX = 9;  // a triangle clipped by the 6 planes of a box has <= 9 vertices
constexpr uint32_t PART_END = 0xffffffffu;

__device__ __forceinline__ uint32_t quantize_uv(float u, float v) {
    const float su = __fmul_rn(fminf(fmaxf(u, 0.f), 1.f), 65535.f), sv = __fmul_rn(fminf(fmaxf(v, 0.f), 1.f), 65535.f);
    return __float2uint_rn(su) | (__float2uint_rn(sv) << 16);
}

// The part of triangle v inside [lo, hi] (Sutherland-Hodgman in float as
// above, the vertices carrying their (u, v)), written to out[0..PART_MAX) with
// its end marker; returns the vertex count (0: no area left, nothing written).
__device__ int clip_triangle_uv(const float (&v)[3][3], const float lo[3], const float hi[3],
                                uint32_t* __restrict__ out) {
    float poly[PART_MAX + 1][5], tmp[PART_MAX + 1][5];
    for (int i = 0; i < 3; ++i) {
        for (int a = 0; a < 3; ++a) poly[i][a] = v[i][a];
        poly[i][3] = i == 1 ? 1.f : 0.f;
        poly[i][4] = i == 2 ? 1.f : 0.f;
    }
    int n = 3;
    for (int a = 0; a < 3; ++a)
        for (int side = 0; side < 2; ++side) {
            const float b = side ? hi[a] : lo[a];
            int m = 0;
            for (int i = 0; i < n; ++i) {
                const float* p = poly[i];
                const float* q = poly[(i + 1) % n];
                const bool pin = side ? p[a] <= b : p[a] >= b;
                const bool qin = side ? q[a] <= b : q[a] >= b;
                if (pin) {
                    for (int c = 0; c < 5; ++c) tmp[m][c] = p[c];
                    ++m;
                }
                if (pin != qin) {
                    const float t = __fdiv_rn(__fsub_rn(b, p[a]), __fsub_rn(q[a], p[a]));
                    for (int c = 0; c < 5; ++c) tmp[m][c] = __fmaf_rn(t, __fsub_rn(q[c], p[c]), p[c]);
                    tmp[m][a] = b;
                    ++m;
                }
            }
            n = m;
            if (n < 3) return 0;
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 5; ++c) poly[i][c] = tmp[i][c];
        }
    for (int i = 0; i < n; ++i) out[i] = quantize_uv(poly[i][3], poly[i][4]);
    if (n < PART_MAX) out[n] = PART_END;
    return n;
}

// The part of every record of a split build, at part_uv[PART_MAX r ...], and
// the record's primitive id (with its sphere flag, as in the record) at
// rec_id[r]. A record whose reference box holds its whole triangle, a sphere,
// and a part that clipping left without area (which a refit then bounds by
// the whole moved triangle) get no part.
__global__ void k_record_parts(const float4* __restrict__ prims, int64_t R, const float4* __restrict__ rec_box,
                               const float* __restrict__ tri, int64_t T, uint32_t* __restrict__ part_uv,
                               uint32_t* __restrict__ rec_id) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t idb = __float_as_uint(prims[3 * r + 2].y);
        rec_id[r] = idb;
        int n = 0;
        if (!(idb & SPHERE_BIT) && (int64_t)idb < T) {
            float3 tl, th;
            prim_box(tri, nullptr, T, idb, tl, th);
            const float4 l = rec_box[2 * r], h = rec_box[2 * r + 1];
            if (l.x > tl.x || l.y > tl.y || l.z > tl.z || h.x < th.x || h.y < th.y || h.z < th.z) {
                const float* f = tri + 9 * (int64_t)idb;
                float v[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int a = 0; a < 3; ++a) v[i][a] = f[3 * i + a];
                const float lo[3] = {l.x, l.y, l.z}, hi[3] = {h.x, h.y, h.z};
                n = clip_triangle_uv(v, lo, hi, part_uv + PART_MAX * r);
            }
        }
        if (n == 0) part_uv[PART_MAX * r] = PART_END;
    }
}

// ---- PLOC: parallel locally-ordered clustering (Meister and Bittner, 2018) ----
// Clusters start as the primitives in Morton order. Every iteration each
// cluster finds, among the PLOC_R clusters on either side of it in the array,
// the one whose union box has the smallest surface area; mutual nearest
// neighbours merge into a new binary node, and the array is compacted (the
// merged cluster takes the lower position). Pairs are ordered by (area, index
// gap, parity of the lower index, lower index), a total order, so the
// globally smallest pair is always mutual: every iteration merges at least
// one pair, and a run of equal boxes pairs up (0,1), (2,3), ... at once.
// Node indices count down: the last merge creates the root, node 0.
constexpr int PLOC_R = 16;
constexpr int PLOC_BLOCK = 256;

__device__ __forceinline__ float union_area(float4 alo, float4 ahi, float4 blo, float4 bhi) {
    const float dx = fmaxf(ahi.x, bhi.x) - fminf(alo.x, blo.x);
    const float dy = fmaxf(ahi.y, bhi.y) - fminf(alo.y, blo.y);
    const float dz = fmaxf(ahi.z, bhi.z) - fminf(alo.z, blo.z);
    const float a = dx * dy + dy * dz + dz * dx;
    return a == a ? a : INFINITY;
}

__global__ void __launch_bounds__(PLOC_BLOCK) k_ploc_nn(const float4* __restrict__ clo, const float4* __restrict__ chi,
                                                        int64_t n, int* __restrict__ nn) {
    __shared__ float4 slo[PLOC_BLOCK + 2 * PLOC_R], shi[PLOC_BLOCK + 2 * PLOC_R];
    const int64_t first = (int64_t)blockIdx.x * PLOC_BLOCK;
    for (int t = threadIdx.x; t < PLOC_BLOCK + 2 * PLOC_R; t += PLOC_BLOCK) {
        const int64_t g = first - PLOC_R + t;
        if (g >= 0 && g < n) {
            slo[t] = clo[g];
            shi[t] = chi[g];
        }
    }
    __syncthreads();
    const int64_t i = first + threadIdx.x;
    if (i >= n) return;
    const int li = threadIdx.x + PLOC_R;
    const float4 alo = slo[li], ahi = shi[li];
    float ba = 0.f;
    int64_t bj = -1, bgap = 0, blo = 0;
    for (int o = -PLOC_R; o <= PLOC_R; ++o) {
        const int64_t j = i + o;
        if (o == 0 || j < 0 || j >= n) continue;
        const float a = union_area(alo, ahi, slo[li + o], shi[li + o]);
        const int64_t gap = o < 0 ? -o : o, lo = o < 0 ? j : i;
        bool better = bj < 0 || a < ba;
        if (!better && a == ba) {
            if (gap != bgap) better = gap < bgap;
            else if ((lo & 1) != (blo & 1)) better = (lo & 1) < (blo & 1);
            else better = lo < blo;
        }
        if (better) {
            ba = a;
            bj = j;
            bgap = gap;
            blo = lo;
        }
    }
    nn[i] = (int)bj;
}

// flag word per cluster: merges here (lower end of a mutual pair) << 32 | stays
__global__ void k_ploc_flags(const int* __restrict__ nn, int64_t n, unsigned long long* __restrict__ flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = nn[i];
        const bool mutual = j >= 0 && nn[j] == (int)i;
        const unsigned long long merge = (mutual && i < j) ? 1ull : 0ull;
        const unsigned long long keep = (mutual && i > j) ? 0ull : 1ull;
        flags[i] = (merge << 32) | keep;
    }
}

__device__ __forceinline__ int leaf_count(const int* cnt, int ref) { return ref >= 0 ? cnt[ref] : 1; }

// Merge mutual pairs into new nodes and compact the cluster array;
// scan[i] = exclusive prefix of the flag words.
__global__ void k_ploc_merge(const int* __restrict__ nn, int64_t n, const unsigned long long* __restrict__ scan,
                             const int* __restrict__ ref, const float4* __restrict__ clo,
                             const float4* __restrict__ chi, int node_base, int* __restrict__ ref_out,
                             float4* __restrict__ lo_out, float4* __restrict__ hi_out, int2* __restrict__ child,
                             float4* __restrict__ blo, float4* __restrict__ bhi, int* __restrict__ cnt,
                             int* __restrict__ parent_int, int* __restrict__ parent_leaf) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = nn[i];
        const bool mutual = j >= 0 && nn[j] == (int)i;
        if (mutual && i > j) continue;
        const unsigned long long s = scan[i];
        const int64_t pos = (int64_t)(s & 0xffffffffull);
        if (mutual) {
            const int node = node_base + (int)(s >> 32);
            const int ra = ref[i], rb = ref[j];
            const float4 la = clo[i], ha = chi[i], lb = clo[j], hb = chi[j];
            const float4 l = make_float4(fminf(la.x, lb.x), fminf(la.y, lb.y), fminf(la.z, lb.z), 0.f);
            const float4 h = make_float4(fmaxf(ha.x, hb.x), fmaxf(ha.y, hb.y), fmaxf(ha.z, hb.z), 0.f);
            child[node] = make_int2(ra, rb);
            blo[node] = l;
            bhi[node] = h;
            cnt[node] = leaf_count(cnt, ra) + leaf_count(cnt, rb);
            if (ra >= 0) parent_int[ra] = node;
            else parent_leaf[-ra - 1] = node;
            if (rb >= 0) parent_int[rb] = node;
            else parent_leaf[-rb - 1] = node;
            ref_out[pos] = node;
            lo_out[pos] = l;
            hi_out[pos] = h;
        } else {
            ref_out[pos] = ref[i];
            lo_out[pos] = clo[i];
            hi_out[pos] = chi[i];
        }
    }
}

__global__ void k_ploc_init(const uint32_t* __restrict__ sorted_ids, int64_t n, const float4* __restrict__ plo,
                            const float4* __restrict__ phi, int* __restrict__ ref, float4* __restrict__ clo,
                            float4* __restrict__ chi) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t id = sorted_ids[j];
        ref[j] = -(int)(j + 1);
        clo[j] = plo[id];
        chi[j] = phi[id];
    }
}

// Depth-first leaf order: a node's first leaf is the number of leaves left of
// it, i.e. the sum of the left siblings' leaf counts on its path to the root.
// Internal node i gets range (first, first + count - 1); leaf j gets pos[j].
__global__ void k_dfs_offsets(const int2* __restrict__ child, const int* __restrict__ parent_int,
                              const int* __restrict__ parent_leaf, const int* __restrict__ cnt, int64_t N,
                              int2* __restrict__ range, int* __restrict__ pos, int* err) {
    const int64_t total = 2 * N - 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const bool internal = k < N - 1;
        int cur = internal ? (int)k : -(int)(k - (N - 1)) - 1;
        int p = internal ? parent_int[k] : parent_leaf[k - (N - 1)];
        int off = 0;
        for (int guard = 0; p >= 0; ++guard) {
            if (guard >= (1 << 22)) {
                atomicAdd(err, 1);
                break;
            }
            const int2 c = child[p];
            if (c.y == cur) off += leaf_count(cnt, c.x);
            cur = p;
            p = parent_int[p];
        }
        if (internal) range[k] = make_int2(off, off + cnt[k] - 1);
        else pos[k - (N - 1)] = off;
    }
}

// Leaves renumbered into depth-first order: sorted ids permuted, and leaf
// references in the children rewritten.
__global__ void k_dfs_apply(const int* __restrict__ pos, const uint32_t* __restrict__ ids_in, int64_t N,
                            uint32_t* __restrict__ ids_out, int2* __restrict__ child, int* err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int pk = pos[k];
        if (pk < 0 || pk >= N) {
            atomicAdd(err, 1);
            continue;
        }
        ids_out[pk] = ids_in[k];
        if (k < N - 1) {
            int2 c = child[k];
            if (c.x < 0) c.x = -pos[-c.x - 1] - 1;
            if (c.y < 0) c.y = -pos[-c.y - 1] - 1;
            child[k] = c;
        }
    }
}

// ---- slot assignment of the 8-wide collapse by surface-area cost ----
// Cost model (SAH, up to the common factor 1 / area(root)): visiting a wide
// node costs SAH_NODE primitive tests, in proportion to the node's area; a
// leaf costs one test per primitive, in proportion to its area. For binary
// node n and k = 1..8, dp[n][k-1] is the least cost of the subtree of n when
// it may take up to k slots of its parent's wide node: one slot (a leaf if it
// holds <= LEAF_MAX primitives, else a wide node of its own), or its two
// children sharing the k slots (a subtree of <= LEAF_MAX primitives always
// takes one slot, a leaf). split[n] byte k-1 (k >= 2) is the left
// child's share of the best split, 0 when one slot is best; byte 0 is the
// left share of the best split of all 8 slots, used when n is a wide node.
// A node visit in the trace kernel is about 3.8 times a triangle test.
constexpr float SAH_NODE = 3.8f;

__device__ __forceinline__ float box_area(float4 lo, float4 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ void slot_costs(int ref, const float4* dp, const float4* plo, const float4* phi,
                                           const uint32_t* ids, float d[8]) {
    if (ref < 0) {  // one primitive: a leaf of one, whatever the slots
        const uint32_t id = ids[-ref - 1];
        const float a = box_area(plo[id], phi[id]);
        for (int k = 0; k < 8; ++k) d[k] = a;
    } else {
        const float4 u = __ldcg(&dp[2 * ref]), v = __ldcg(&dp[2 * ref + 1]);
        d[0] = u.x, d[1] = u.y, d[2] = u.z, d[3] = u.w, d[4] = v.x, d[5] = v.y, d[6] = v.z, d[7] = v.w;
    }
}

// Bottom up, one thread per leaf: at each node the second arriving thread
// computes it from both children (the first stops).
__global__ void k_sah_dp(const int2* __restrict__ child, const int2* __restrict__ range,
                         const int* __restrict__ parent_int, const int* __restrict__ parent_leaf,
                         const float4* __restrict__ blo, const float4* __restrict__ bhi,
                         const float4* __restrict__ plo, const float4* __restrict__ phi,
                         const uint32_t* __restrict__ ids, int64_t N, float4* dp, uint2* split, int* arrivals,
                         int* err) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        int node = parent_leaf[j];
        for (int guard = 0; node >= 0; ++guard) {
            if (guard >= (1 << 22)) {
                atomicAdd(err, 1);
                break;
            }
            __threadfence();
            if (atomicAdd(&arrivals[node], 1) == 0) break;
            __threadfence();
            const int2 c = child[node];
            float dl[8], dr[8];
            slot_costs(c.x, dp, plo, phi, ids, dl);
            slot_costs(c.y, dp, plo, phi, ids, dr);
            float dsplit[9];
            int arg[9];
            for (int k = 2; k <= 8; ++k) {
                float best = INFINITY;
                int ba = 1;
                for (int a = 1; a < k; ++a) {
                    const float v = dl[a - 1] + dr[k - a - 1];
                    if (v < best) {
                        best = v;
                        ba = a;
                    }
                }
                dsplit[k] = best;
                arg[k] = ba;
            }
            const float area = box_area(blo[node], bhi[node]);
            const int2 r = range[node];
            const int cnt = r.y - r.x + 1;
            const float c_node = area * SAH_NODE + dsplit[8];
            const float c_one = cnt <= LEAF_MAX ? fminf(area * (float)cnt, c_node) : c_node;
            float d[8];
            uint32_t bytes[8];
            d[0] = c_one;
            bytes[0] = (uint32_t)arg[8];
            for (int k = 2; k <= 8; ++k) {
                const bool sp = cnt > LEAF_MAX && dsplit[k] < c_one;  // small subtrees stay one leaf
                d[k - 1] = sp ? dsplit[k] : c_one;
                bytes[k - 1] = sp ? (uint32_t)arg[k] : 0u;
            }
            __stcg(&dp[2 * node], make_float4(d[0], d[1], d[2], d[3]));
            __stcg(&dp[2 * node + 1], make_float4(d[4], d[5], d[6], d[7]));
            split[node] = make_uint2(bytes[0] | bytes[1] << 8 | bytes[2] << 16 | bytes[3] << 24,
                                     bytes[4] | bytes[5] << 8 | bytes[6] << 16 | bytes[7] << 24);
            node = parent_int[node];
        }
    }
}

// Every binary node's box again, bottom up from the padded leaf boxes (the
// clustering decided on exact boxes): one thread per leaf, the second thread
// to arrive at a node computes it and goes on. Leaf j (clustering order)
// starts at parent_leaf[j]; the children's leaf references are in depth-first
// order, whose reference indices are ids_dfs.
__global__ void k_refit_padded(const int2* __restrict__ child, const int* __restrict__ parent_int,
                               const int* __restrict__ parent_leaf, const uint32_t* __restrict__ ids_dfs,
                               const float4* __restrict__ plo, const float4* __restrict__ phi,
                               const uint32_t* __restrict__ ref_prim, const float* __restrict__ tri,
                               const float* __restrict__ sph, int64_t T, int64_t R, float4* blo, float4* bhi,
                               int* arrivals, int* err) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < R; j += (int64_t)gridDim.x * blockDim.x) {
        int node = parent_leaf[j];
        for (int guard = 0; node >= 0; ++guard) {
            if (guard >= (1 << 22)) {
                atomicAdd(err, 1);
                break;
            }
            __threadfence();
            if (atomicAdd(&arrivals[node], 1) == 0) break;
            __threadfence();
            const int2 c = child[node];
            float3 l[2], h[2];
            const int cs[2] = {c.x, c.y};
            for (int q = 0; q < 2; ++q) {
                if (cs[q] >= 0) {
                    const float4 a = __ldcg(&blo[cs[q]]), b = __ldcg(&bhi[cs[q]]);
                    l[q] = make_float3(a.x, a.y, a.z);
                    h[q] = make_float3(b.x, b.y, b.z);
                } else {
                    padded_ref_box(plo, phi, ref_prim, tri, sph, T, ids_dfs[-cs[q] - 1], l[q], h[q]);
                }
            }
            __stcg(&blo[node], make_float4(fminf(l[0].x, l[1].x), fminf(l[0].y, l[1].y), fminf(l[0].z, l[1].z), 0.f));
            __stcg(&bhi[node], make_float4(fmaxf(h[0].x, h[1].x), fmaxf(h[0].y, h[1].y), fmaxf(h[0].z, h[1].z), 0.f));
            node = parent_int[node];
        }
    }
}

// ---- exclusive scan of 64-bit words: tiles of 1024, tile sums scanned recursively ----
constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_TILE = 4 * SCAN_BLOCK;

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_tiles(unsigned long long* data, int64_t n,
                                                           unsigned long long* sums) {
    __shared__ unsigned long long warp_tot[SCAN_BLOCK / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
    unsigned long long v[4];
    for (int q = 0; q < 4; ++q) v[q] = base + q < n ? data[base + q] : 0ull;
    const unsigned long long tsum = v[0] + v[1] + v[2] + v[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = tsum;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = lane < SCAN_BLOCK / 32 ? warp_tot[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_BLOCK / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    unsigned long long run = (warp > 0 ? warp_tot[warp - 1] : 0ull) + x - tsum;
    for (int q = 0; q < 4; ++q) {
        if (base + q < n) data[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == SCAN_BLOCK - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(unsigned long long* data, int64_t n, const unsigned long long* offs) {
    const int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    const unsigned long long o = offs[blockIdx.x];
    for (int q = 0; q < 4; ++q)
        if (i + q * SCAN_BLOCK < n) data[i + q * SCAN_BLOCK] += o;
}

struct BinTree {
    const int2* child;
    const int2* range;
    const float4* blo;
    const float4* bhi;
    const float4* plo;
    const float4* phi;
    const uint32_t* sorted_ids;
    const uint2* split;  // slot splits of the surface-area policy (k_sah_dp); nullptr: area policy
    const uint32_t* ref_prim;  // reference -> primitive (nullptr: references are the primitives)
    const float* tri;
    const float* sph;
    int64_t T;
};

__device__ __forceinline__ int split_share(const uint2 s, int k) {  // k = 1..8 slots; byte 0: wide-node split
    const uint32_t w = k <= 4 ? s.x : s.y;
    return (int)((w >> (8 * ((k - 1) & 3))) & 0xffu);
}

__device__ __forceinline__ void ref_box(const BinTree& bt, int ref, float3& lo, float3& hi, int& first, int& last) {
    float4 l, h;
    if (ref >= 0) {
        l = bt.blo[ref];
        h = bt.bhi[ref];
        const int2 r = bt.range[ref];
        first = r.x;
        last = r.y;
        lo = make_float3(l.x, l.y, l.z);
        hi = make_float3(h.x, h.y, h.z);
    } else {
        const int j = -ref - 1;
        padded_ref_box(bt.plo, bt.phi, bt.ref_prim, bt.tri, bt.sph, bt.T, bt.sorted_ids[j], lo, hi);
        first = last = j;
    }
}

}  // namespace

// Child boxes of up to 8 children into their slots, exactly as computed
// (empty slots get lo = +inf, hi = -inf, which no ray enters); returns the
// union of the children.
__device__ void write_child_boxes(WNode& nd, const float3* clo, const float3* chi, const int* slot_of, int m,
                                  float3& ulo, float3& uhi) {
    for (int s = 0; s < 8; ++s) {
        nd.lo_x[s] = nd.lo_y[s] = nd.lo_z[s] = INFINITY;
        nd.hi_x[s] = nd.hi_y[s] = nd.hi_z[s] = -INFINITY;
    }
    ulo = make_float3(INFINITY, INFINITY, INFINITY);
    uhi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    for (int c = 0; c < m; ++c) {
        const int sl = slot_of[c];
        nd.lo_x[sl] = clo[c].x;
        nd.lo_y[sl] = clo[c].y;
        nd.lo_z[sl] = clo[c].z;
        nd.hi_x[sl] = chi[c].x;
        nd.hi_y[sl] = chi[c].y;
        nd.hi_z[sl] = chi[c].z;
        ulo = make_float3(fminf(ulo.x, clo[c].x), fminf(ulo.y, clo[c].y), fminf(ulo.z, clo[c].z));
        uhi = make_float3(fmaxf(uhi.x, chi[c].x), fmaxf(uhi.y, chi[c].y), fmaxf(uhi.z, chi[c].z));
    }
}

__device__ __forceinline__ void write_prim_record(float4* __restrict__ rec, const float* __restrict__ tri,
                                                  const float* __restrict__ sph, int64_t T, uint32_t id) {
    if (id < T) {
        const float* v = tri + 9 * (int64_t)id;
        float e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        float e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        // Degenerate (collinear) triangles are never hit (det == 0). The float
        // cross product of the rounded edges is within 8 * 2^-24 * M1 * M2 (+
        // 2^-24 of itself) of the exact one (M: largest edge component), so a
        // component above 2^-19 M1 M2 proves the triangle has area; only the
        // rest take the exact test, the double cross product of the exact
        // edge differences.
        const float m1 = fmaxf(fmaxf(fabsf(e1[0]), fabsf(e1[1])), fabsf(e1[2]));
        const float m2 = fmaxf(fmaxf(fabsf(e2[0]), fabsf(e2[1])), fabsf(e2[2]));
        const float fx = e1[1] * e2[2] - e1[2] * e2[1], fy = e1[2] * e2[0] - e1[0] * e2[2],
                    fz = e1[0] * e2[1] - e1[1] * e2[0];
        const float thr = 0x1p-19f * m1 * m2;
        if (!(fmaxf(fmaxf(fabsf(fx), fabsf(fy)), fabsf(fz)) > thr && thr > 0.f)) {
            const double d1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
            const double d2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
            const double nx = d1[1] * d2[2] - d1[2] * d2[1], ny = d1[2] * d2[0] - d1[0] * d2[2],
                         nz = d1[0] * d2[1] - d1[1] * d2[0];
            if (nx == 0.0 && ny == 0.0 && nz == 0.0)
                for (int a = 0; a < 3; ++a) e1[a] = e2[a] = 0.f;
        }
        rec[0] = make_float4(v[0], v[1], v[2], e1[0]);
        rec[1] = make_float4(e1[1], e1[2], e2[0], e2[1]);
        rec[2] = make_float4(e2[2], __uint_as_float(id), 0.f, 0.f);
    } else {
        const float* s = sph + 4 * ((int64_t)id - T);
        rec[0] = make_float4(s[0], s[1], s[2], fabsf(s[3]));
        rec[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[2] = make_float4(0.f, __uint_as_float(id | SPHERE_BIT), 0.f, 0.f);
    }
}

namespace {

// One level of the collapse. frontier[i] = (binary ref, wide node index).
// rec_box (nullable) receives each record's exact reference box.
__global__ void k_collapse(BinTree bt, const int2* __restrict__ frontier, int n_front, int2* __restrict__ next_front,
                           uint32_t* counters, WNode* __restrict__ nodes, float4* __restrict__ nbox,
                           float4* __restrict__ prims, const float* __restrict__ tri, const float* __restrict__ sph,
                           int64_t T, int* max_leaf, float4* __restrict__ rec_box) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_front) return;
    const int ref = frontier[i].x;
    const int w = frontier[i].y;
    int cref[8];
    float3 clo[8], chi[8];
    int cfirst[8], clast[8];
    int m;
    if (ref < 0) {
        m = 1;
        cref[0] = ref;
        ref_box(bt, ref, clo[0], chi[0], cfirst[0], clast[0]);
    } else if (bt.split) {
        // surface-area policy: the 8 slots of this wide node are shared out by
        // the stored splits; a subtree given k slots is one slot (k == 1, a
        // primitive, or share 0) or passes shares a and k - a to its children
        int sref[8], sk[8];
        int sp = 0;
        m = 0;
        const int2 c = bt.child[ref];
        const int a = split_share(bt.split[ref], 1);
        sref[sp] = c.y, sk[sp++] = 8 - a;
        sref[sp] = c.x, sk[sp++] = a;
        while (sp > 0) {
            --sp;
            const int x = sref[sp], k = sk[sp];
            const int share = (x < 0 || k == 1) ? 0 : split_share(bt.split[x], k);
            if (share <= 0 || share >= k) {
                cref[m++] = x;
                continue;
            }
            const int2 cc = bt.child[x];
            sref[sp] = cc.y, sk[sp++] = k - share;
            sref[sp] = cc.x, sk[sp++] = share;
        }
        for (int q = 0; q < m; ++q) ref_box(bt, cref[q], clo[q], chi[q], cfirst[q], clast[q]);
    } else {
        // area policy: start from the two children and repeatedly open the
        // child of largest surface area that holds more than LEAF_MAX primitives
        const int2 c = bt.child[ref];
        cref[0] = c.x;
        cref[1] = c.y;
        m = 2;
        for (int q = 0; q < m; ++q) ref_box(bt, cref[q], clo[q], chi[q], cfirst[q], clast[q]);
        while (m < 8) {
            int best = -1;
            float best_area = -1.f;
            for (int q = 0; q < m; ++q) {
                if (cref[q] < 0 || clast[q] - cfirst[q] + 1 <= LEAF_MAX) continue;
                const float dx = chi[q].x - clo[q].x, dy = chi[q].y - clo[q].y, dz = chi[q].z - clo[q].z;
                const float area = dx * dy + dy * dz + dz * dx;
                if (area > best_area) {
                    best_area = area;
                    best = q;
                }
            }
            if (best < 0) break;
            const int2 ch = bt.child[cref[best]];
            cref[best] = ch.x;
            ref_box(bt, ch.x, clo[best], chi[best], cfirst[best], clast[best]);
            cref[m] = ch.y;
            ref_box(bt, ch.y, clo[m], chi[m], cfirst[m], clast[m]);
            ++m;
        }
    }
    // slots: greedy assignment of children to octant directions
    float3 cen;
    {
        float3 lo = clo[0], hi = chi[0];
        for (int c = 1; c < m; ++c) {
            lo = make_float3(fminf(lo.x, clo[c].x), fminf(lo.y, clo[c].y), fminf(lo.z, clo[c].z));
            hi = make_float3(fmaxf(hi.x, chi[c].x), fmaxf(hi.y, chi[c].y), fmaxf(hi.z, chi[c].z));
        }
        cen = make_float3(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z));
    }
    int slot_of[8];
    unsigned used = 0, done = 0;
    for (int it = 0; it < m; ++it) {
        float best = -INFINITY;
        int bc = -1, bs = -1;
        for (int c = 0; c < m; ++c) {
            if (done & (1u << c)) continue;
            const float ox = 0.5f * (clo[c].x + chi[c].x) - cen.x;
            const float oy = 0.5f * (clo[c].y + chi[c].y) - cen.y;
            const float oz = 0.5f * (clo[c].z + chi[c].z) - cen.z;
            for (int s = 0; s < 8; ++s) {
                if (used & (1u << s)) continue;
                const float cost = ((s & 1) ? ox : -ox) + ((s & 2) ? oy : -oy) + ((s & 4) ? oz : -oz);
                if (cost > best) {
                    best = cost;
                    bc = c;
                    bs = s;
                }
            }
        }
        slot_of[bc] = bs;
        used |= 1u << bs;
        done |= 1u << bc;
    }
    // classify, allocate and write
    int is_int[8];
    int n_int = 0, n_prim = 0;
    for (int c = 0; c < m; ++c) {
        is_int[c] = cref[c] >= 0 && clast[c] - cfirst[c] + 1 > LEAF_MAX;
        if (is_int[c]) ++n_int;
        else n_prim += clast[c] - cfirst[c] + 1;
    }
    const uint32_t child_base = n_int ? atomicAdd(&counters[0], (uint32_t)n_int) : 0u;
    const uint32_t prim_base = n_prim ? atomicAdd(&counters[1], (uint32_t)n_prim) : 0u;
    WNode nd;
    nd.child_base = child_base;
    nd.prim_base = prim_base;
    uint32_t meta[2] = {0, 0};
    uint32_t imask = 0;
    for (int c = 0; c < m; ++c)
        if (is_int[c]) imask |= 1u << slot_of[c];
    int poff = 0;
    int leaf_max = 0;
    for (int s = 0; s < 8; ++s) {
        int c = -1;
        for (int q = 0; q < m; ++q)
            if (slot_of[q] == s) c = q;
        if (c < 0) continue;
        uint32_t mb;
        if (is_int[c]) {
            const uint32_t rank = __popc(imask & ((1u << s) - 1u));
            mb = 0x80u | rank;
            const uint32_t slot_idx = atomicAdd(&counters[2], 1u);
            next_front[slot_idx] = make_int2(cref[c], (int)(child_base + rank));
        } else {
            const int cnt = clast[c] - cfirst[c] + 1;
            mb = ((uint32_t)cnt << 5) | (uint32_t)poff;
            for (int q = 0; q < cnt; ++q) {
                const uint32_t ref = bt.sorted_ids[cfirst[c] + q];
                const int64_t rec = (int64_t)(prim_base + poff + q);
                write_prim_record(prims + 3 * rec, tri, sph, T, bt.ref_prim ? bt.ref_prim[ref] : ref);
                if (rec_box) {
                    rec_box[2 * rec] = bt.plo[ref];
                    rec_box[2 * rec + 1] = bt.phi[ref];
                }
            }
            poff += cnt;
            leaf_max = max(leaf_max, cnt);
        }
        meta[s >> 2] |= mb << (8 * (s & 3));
    }
    nd.meta_lo = meta[0];
    nd.meta_hi = meta[1];
    float3 ulo, uhi;
    write_child_boxes(nd, clo, chi, slot_of, m, ulo, uhi);
    nodes[w] = nd;
    nbox[2 * w] = make_float4(ulo.x, ulo.y, ulo.z, 0.f);
    nbox[2 * w + 1] = make_float4(uhi.x, uhi.y, uhi.z, 0.f);
    if (leaf_max) atomicMax(max_leaf, leaf_max);
}

// ---------------------------------------------------------------- refit after a vertex update

// Leaf records' parts and primitive ids in a split build (both null otherwise).
struct Parts {
    const uint32_t* uv;
    const uint32_t* id;
};

// Box of record r (primitive id with its sphere flag: idb) from the current
// vertices: its part of the moved triangle when it has one (clamped to the
// whole triangle's box, which holds the part), else its whole primitive's
// box. Padded with the triangle's pad when `pad`.
__device__ __forceinline__ void record_box(uint32_t idb, int64_t r, Parts parts, const float* __restrict__ tri,
                                           const float* __restrict__ sph, int64_t T, bool pad, float3& lo,
                                           float3& hi) {
    const int64_t id = (int64_t)(idb & ~SPHERE_BIT);
    float3 tl, th;
    prim_box(tri, sph, T, id, tl, th);
    lo = tl;
    hi = th;
    if (parts.uv && id < T && parts.uv[PART_MAX * r] != PART_END) {
        const float* f = tri + 9 * id;
        const float3 a = make_float3(f[0], f[1], f[2]);
        const float3 e1 = make_float3(f[3] - f[0], f[4] - f[1], f[5] - f[2]);
        const float3 e2 = make_float3(f[6] - f[0], f[7] - f[1], f[8] - f[2]);
        float3 l = make_float3(INFINITY, INFINITY, INFINITY), h = make_float3(-INFINITY, -INFINITY, -INFINITY);
        const uint32_t* q = parts.uv + PART_MAX * r;
        for (int k = 0; k < PART_MAX; ++k) {
            const uint32_t w = q[k];
            if (w == PART_END) break;
            const float u = (float)(w & 0xffffu) * (1.f / 65535.f), v = (float)(w >> 16) * (1.f / 65535.f);
            const float3 p = make_float3(fmaf(v, e2.x, fmaf(u, e1.x, a.x)), fmaf(v, e2.y, fmaf(u, e1.y, a.y)),
                                         fmaf(v, e2.z, fmaf(u, e1.z, a.z)));
            l = make_float3(fminf(l.x, p.x), fminf(l.y, p.y), fminf(l.z, p.z));
            h = make_float3(fmaxf(h.x, p.x), fmaxf(h.y, p.y), fmaxf(h.z, p.z));
        }
        lo = make_float3(fmaxf(lo.x, l.x), fmaxf(lo.y, l.y), fmaxf(lo.z, l.z));
        hi = make_float3(fminf(hi.x, h.x), fminf(hi.y, h.y), fminf(hi.z, h.z));
    }
    // the 16-bit (u, v) and the float mapping move a vertex by ~2^-16 of the
    // triangle's extent, inside the pad of the whole triangle
    if (pad && id < T) pad_box(tri_pad(tl, th), lo, hi);
}

// First step of a refit, one thread per record: the record rewritten from the
// moved vertices (spheres do not move) and its padded box (rbox, 6 floats per
// record: lo, hi), which k_refit_wide gathers into the leaf slots. A split
// build reads the records' ids from parts.id (4 bytes, not a record's sector).
__global__ void k_refit_records(float4* __restrict__ prims, int64_t n, Parts parts, const float* __restrict__ tri,
                                const float* __restrict__ sph, int64_t T, float2* __restrict__ rbox) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t idb = parts.id ? parts.id[r] : __float_as_uint(prims[3 * r + 2].y);
        if (!(idb & SPHERE_BIT)) write_prim_record(prims + 3 * r, tri, sph, T, idb);
        float3 lo, hi;
        record_box(idb, r, parts, tri, sph, T, true, lo, hi);
        rbox[3 * r] = make_float2(lo.x, lo.y);
        rbox[3 * r + 1] = make_float2(lo.z, hi.x);
        rbox[3 * r + 2] = make_float2(hi.y, hi.z);
    }
}

// Recompute the child boxes of the nodes in [begin, end) (one level, deepest
// first). Eight lanes per node, lane s for slot s: the slot's box is the union
// of its leaf records' boxes (rbox) or its internal child's box, and each of
// the node's six box rows (8 floats, one 32-byte sector) is written by its
// eight lanes together. Empty slots get the empty box (+inf, -inf) that the
// collapse gave them. Only the node's header is read. The node's union box
// (nbox) is reduced over its eight lanes, which share a warp.
constexpr int REFIT_BLOCK = 128;
static_assert(REFIT_BLOCK % 32 == 0, "a node's eight lanes must share a warp");

__global__ void __launch_bounds__(REFIT_BLOCK) k_refit_wide(WNode* __restrict__ nodes, float4* __restrict__ nbox,
                                                            int64_t begin, int64_t end,
                                                            const float2* __restrict__ rbox) {
    const int64_t t = blockIdx.x * (int64_t)REFIT_BLOCK + threadIdx.x;
    const int64_t w = begin + (t >> 3);
    const int s = (int)(t & 7);
    const bool live = w < end;
    float3 lo = make_float3(INFINITY, INFINITY, INFINITY), hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    if (live) {
        float* nf = reinterpret_cast<float*>(nodes + w);
        const uint4 hd = *reinterpret_cast<const uint4*>(nf + 48);
        const uint32_t mb = ((s < 4 ? hd.z : hd.w) >> (8 * (s & 3))) & 0xffu;
        if (mb & 0x80u) {
            const int64_t c = hd.x + __popc(internal_mask(hd.z, hd.w) & ((1u << s) - 1u));
            const float4 l = nbox[2 * c], h = nbox[2 * c + 1];
            lo = make_float3(l.x, l.y, l.z);
            hi = make_float3(h.x, h.y, h.z);
        } else if (mb) {
            const int cnt = mb >> 5, off = mb & 31;
            const float2* b = rbox + 3 * ((int64_t)hd.y + off);
            for (int q = 0; q < cnt; ++q) {
                const float2 a = b[3 * q], m = b[3 * q + 1], z = b[3 * q + 2];
                lo = make_float3(fminf(lo.x, a.x), fminf(lo.y, a.y), fminf(lo.z, m.x));
                hi = make_float3(fmaxf(hi.x, m.y), fmaxf(hi.y, z.x), fmaxf(hi.z, z.y));
            }
        }
        nf[s] = lo.x;
        nf[8 + s] = hi.x;
        nf[16 + s] = lo.y;
        nf[24 + s] = hi.y;
        nf[32 + s] = lo.z;
        nf[40 + s] = hi.z;
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
    if (live && s == 0) {
        nbox[2 * w] = make_float4(lo.x, lo.y, lo.z, 0.f);
        nbox[2 * w + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
    }
}

// ---------------------------------------------------------------- validation

__device__ __forceinline__ void slot_box(const WNode& nd, int s, double lo[3], double hi[3]) {
    lo[0] = nd.lo_x[s];
    lo[1] = nd.lo_y[s];
    lo[2] = nd.lo_z[s];
    hi[0] = nd.hi_x[s];
    hi[1] = nd.hi_y[s];
    hi[2] = nd.hi_z[s];
}

// n_records leaf records over n_prims primitives; rec_box (nullable): each
// record's exact reference box, which must lie in its leaf slot (else the
// record's unpadded box from the current vertices must: its part of the
// triangle after a refit of a split build, or the whole primitive's box).
__global__ void k_validate(const WNode* __restrict__ nodes, int64_t n_nodes, const float4* __restrict__ nbox,
                           const float4* __restrict__ prims, int64_t n_records, int64_t n_prims,
                           const float4* __restrict__ rec_box, Parts parts, const float* __restrict__ tri,
                           const float* __restrict__ sph, int64_t T, unsigned* __restrict__ seen_rec,
                           unsigned* __restrict__ seen_id, unsigned* __restrict__ node_refs, int* errors) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= n_nodes) return;
    const WNode nd = nodes[w];
    const uint32_t imask = internal_mask(nd.meta_lo, nd.meta_hi);
    for (int s = 0; s < 8; ++s) {
        const uint32_t mb = ((s < 4 ? nd.meta_lo : nd.meta_hi) >> (8 * (s & 3))) & 0xffu;
        if (!mb) {
            if (imask & (1u << s)) atomicAdd(&errors[0], 1);
            continue;
        }
        double lo[3], hi[3];
        slot_box(nd, s, lo, hi);
        if (mb & 0x80u) {
            if (!(imask & (1u << s)) || (mb & 0x7fu) != (uint32_t)__popc(imask & ((1u << s) - 1u))) atomicAdd(&errors[0], 1);
            const int64_t c = nd.child_base + (mb & 7u);
            if (c <= w || c >= n_nodes) {
                atomicAdd(&errors[1], 1);
                continue;
            }
            atomicAdd(&node_refs[c], 1u);
            const float4 l = nbox[2 * c], h = nbox[2 * c + 1];
            if (l.x < lo[0] || l.y < lo[1] || l.z < lo[2] || h.x > hi[0] || h.y > hi[1] || h.z > hi[2])
                atomicAdd(&errors[2], 1);
        } else {
            if (imask & (1u << s)) atomicAdd(&errors[0], 1);
            const int cnt = mb >> 5, off = mb & 31;
            for (int q = 0; q < cnt; ++q) {
                const int64_t r = (int64_t)nd.prim_base + off + q;
                if (r >= n_records) {
                    atomicAdd(&errors[3], 1);
                    continue;
                }
                atomicAdd(&seen_rec[r], 1u);
                const uint32_t id = __float_as_uint(prims[3 * r + 2].y) & ~SPHERE_BIT;
                if (id < (uint32_t)n_prims) atomicAdd(&seen_id[id], 1u);
                else atomicAdd(&errors[6], 1);
                float3 pl, ph;
                if (rec_box) {
                    const float4 l = rec_box[2 * r], h = rec_box[2 * r + 1];
                    pl = make_float3(l.x, l.y, l.z);
                    ph = make_float3(h.x, h.y, h.z);
                } else {
                    record_box(__float_as_uint(prims[3 * r + 2].y), r, parts, tri, sph, T, false, pl, ph);
                }
                if (pl.x < lo[0] || pl.y < lo[1] || pl.z < lo[2] || ph.x > hi[0] || ph.y > hi[1] || ph.z > hi[2])
                    atomicAdd(&errors[4], 1);
            }
        }
    }
}

// every record referenced once; every primitive in exactly one record, or in
// at least one when triangles are split into several references
__global__ void k_check_counts(const unsigned* a, int64_t n_records, const unsigned* b, int64_t n_prims,
                               bool split, const unsigned* node_refs, int64_t n_nodes, int* errors) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_records;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a[i] != 1u) atomicAdd(&errors[5], 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_prims; i += (int64_t)gridDim.x * blockDim.x)
        if (split ? b[i] < 1u : b[i] != 1u) atomicAdd(&errors[6], 1);
    for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_nodes;
         i += (int64_t)gridDim.x * blockDim.x)
        if (node_refs[i] != 1u) atomicAdd(&errors[7], 1);
}

int grid_for(int64_t n, int block, int cap) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}



// Tile counts of each level of the recursive scan of up to n words.
std::vector<int64_t> scan_levels(int64_t n) {
    std::vector<int64_t> lv;
    do {
        n = (n + SCAN_TILE - 1) / SCAN_TILE;
        lv.push_back(n);
    } while (n > 1);
    return lv;
}

// Exclusive scan of d[0..n) in place; the sum of all n words lands in *total.
// aux holds the tile sums of this level followed by those of deeper levels.
void scan_u64(unsigned long long* d, int64_t n, unsigned long long* aux, const std::vector<int64_t>& lv, size_t l,
              unsigned long long* total, cudaStream_t st) {
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tiles<<<(unsigned)tiles, SCAN_BLOCK, 0, st>>>(d, n, aux);
    if (tiles > 1) {
        scan_u64(aux, tiles, aux + lv[l], lv, l + 1, total, st);
        k_scan_add<<<(unsigned)tiles, SCAN_BLOCK, 0, st>>>(d, n, aux);
    } else {
        cudaMemcpyAsync(total, aux, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    }
}

// Binary tree over the N >= 2 primitives in Morton order (ids_in) by PLOC.
// Fills child, blo/bhi and range of internal nodes 0..N-2 (root 0), with the
// leaves renumbered depth-first: ids_out[j] is the primitive of leaf j.
rcp_status build_ploc(int64_t N, const uint32_t* ids_in, uint32_t* ids_out, const float4* plo, const float4* phi,
                      int2* child, int2* range, float4* blo, float4* bhi, int* parent_int, int* parent_leaf,
                      int* d_err, int cap, cudaStream_t st) {
    DevBuf<int> ref_a, ref_b, nn, cnt, pos;
    DevBuf<float4> lo_a, hi_a, lo_b, hi_b;
    DevBuf<unsigned long long> flags, aux, total;
    const std::vector<int64_t> lv = scan_levels(N);
    int64_t aux_n = 0;
    for (int64_t t : lv) aux_n += t;
    RCP_CUDA(ref_a.alloc(N));
    RCP_CUDA(ref_b.alloc(N));
    RCP_CUDA(nn.alloc(N));
    RCP_CUDA(cnt.alloc(N));
    RCP_CUDA(pos.alloc(N));
    RCP_CUDA(lo_a.alloc(N));
    RCP_CUDA(hi_a.alloc(N));
    RCP_CUDA(lo_b.alloc(N));
    RCP_CUDA(hi_b.alloc(N));
    RCP_CUDA(flags.alloc(N));
    RCP_CUDA(aux.alloc(aux_n));
    RCP_CUDA(total.alloc(1));
    RCP_CUDA(cudaMemsetAsync(parent_int, 0xff, sizeof(int) * N, st));
    RCP_CUDA(cudaMemsetAsync(parent_leaf, 0xff, sizeof(int) * N, st));
    int *rin = ref_a.p, *rout = ref_b.p;
    float4 *lin = lo_a.p, *hin = hi_a.p, *lout = lo_b.p, *hout = hi_b.p;
    k_ploc_init<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(ids_in, N, plo, phi, rin, lin, hin);
    int64_t n = N, created = 0;
    while (n > 1) {
        k_ploc_nn<<<(unsigned)((n + PLOC_BLOCK - 1) / PLOC_BLOCK), PLOC_BLOCK, 0, st>>>(lin, hin, n, nn.p);
        k_ploc_flags<<<grid_for(n, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(nn.p, n, flags.p);
        scan_u64(flags.p, n, aux.p, lv, 0, total.p, st);
        unsigned long long ht = 0;
        RCP_CUDA(cudaMemcpyAsync(&ht, total.p, sizeof(ht), cudaMemcpyDeviceToHost, st));
        RCP_CUDA(cudaStreamSynchronize(st));
        const int64_t merges = (int64_t)(ht >> 32), keeps = (int64_t)(ht & 0xffffffffull);
        // the smallest pair is always mutual, so an iteration without a merge
        // means the device state is corrupt
        if (merges < 1 || keeps != n - merges || created + merges > N - 1) {
            set_error("BVH build: clustering made no progress");
            return RCP_ERR_STATE;
        }
        const int node_base = (int)(N - 1 - created - merges);
        k_ploc_merge<<<grid_for(n, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(nn.p, n, flags.p, rin, lin, hin,
                                                                             node_base, rout, lout, hout, child,
                                                                             blo, bhi, cnt.p, parent_int,
                                                                             parent_leaf);
        created += merges;
        n = keeps;
        std::swap(rin, rout);
        std::swap(lin, lout);
        std::swap(hin, hout);
    }
    k_dfs_offsets<<<grid_for(2 * N - 1, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(child, parent_int, parent_leaf,
                                                                                 cnt.p, N, range, pos.p, d_err);
    k_dfs_apply<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(pos.p, ids_in, N, ids_out, child, d_err);
    RCP_CUDA(cudaGetLastError());
    // the scratch above is freed on return: finish using it first
    RCP_CUDA(cudaStreamSynchronize(st));
    return RCP_OK;
}

}  // namespace

rcp_status build_bvh(Scene& sc, cudaStream_t st) {
    const int64_t T = sc.T, N = sc.T + sc.S;
    EventPair ev;
    RCP_CUDA(ev.create());
    RCP_CUDA(cudaEventRecord(ev.a, st));
    int sms = 148;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int cap = sms * 16;
    DevBuf<float4> plo, phi;
    DevBuf<uint32_t> bounds;
    RCP_CUDA(plo.alloc(N));
    RCP_CUDA(phi.alloc(N));
    RCP_CUDA(bounds.alloc(12));
    k_init_bounds<<<1, 32, 0, st>>>(bounds.p);
    k_prim_bounds<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(sc.d_tri, sc.d_sph, T, N, plo.p, phi.p,
                                                                          bounds.p);
    // references: the primitives themselves, or split triangles (R >= N)
    int64_t R = N;
    DevBuf<float4> rlo, rhi;
    DevBuf<uint32_t> rprim;
    const float4* ref_lo = plo.p;
    const float4* ref_hi = phi.p;
    const bool split = sc.split_max > 1 && T > 0;
    if (split) {
        DevBuf<unsigned long long> counts, aux, total;
        const std::vector<int64_t> lv = scan_levels(N);
        int64_t aux_n = 0;
        for (int64_t t : lv) aux_n += t;
        RCP_CUDA(counts.alloc(N));
        RCP_CUDA(aux.alloc(aux_n));
        RCP_CUDA(total.alloc(1));
        k_split_count<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(sc.d_tri, T, N, sc.split_max,
                                                                              counts.p);
        scan_u64(counts.p, N, aux.p, lv, 0, total.p, st);
        unsigned long long hr = 0;
        RCP_CUDA(cudaMemcpyAsync(&hr, total.p, sizeof(hr), cudaMemcpyDeviceToHost, st));
        RCP_CUDA(cudaStreamSynchronize(st));
        R = (int64_t)hr;
        if (R < N || R > N * (int64_t)SPLIT_MAX || R >= ((int64_t)1 << 30)) {
            set_error("BVH build: split references out of range (at most 2^30 - 1)");
            return RCP_ERR_ARG;
        }
        RCP_CUDA(rlo.alloc(R));
        RCP_CUDA(rhi.alloc(R));
        RCP_CUDA(rprim.alloc(R));
        DevBuf<int> split_err;
        RCP_CUDA(split_err.alloc(1));
        RCP_CUDA(cudaMemsetAsync(split_err.p, 0, sizeof(int), st));
        k_split_write<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(
            sc.d_tri, T, N, sc.split_max, counts.p, R, plo.p, phi.p, rlo.p, rhi.p, rprim.p, split_err.p);
        int h_err = 0;
        RCP_CUDA(cudaMemcpyAsync(&h_err, split_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        RCP_CUDA(cudaStreamSynchronize(st));  // counts and aux are freed on leaving this block
        if (h_err) {
            set_error("BVH build: split references counted and written differently");
            return RCP_ERR_STATE;
        }
        ref_lo = rlo.p;
        ref_hi = rhi.p;
    }
    const int64_t n_nodes_cap = R > 1 ? R : 1;
    DevBuf<float4> blo, bhi;
    DevBuf<uint32_t> keys, vals, akeys, avals, counters;
    DevBuf<int2> child, range, fa, fb;
    DevBuf<int> parent_int, parent_leaf, err;
    DevBuf<char> scratch;
    RCP_CUDA(keys.alloc(R));
    RCP_CUDA(vals.alloc(R));
    RCP_CUDA(akeys.alloc(R));
    RCP_CUDA(avals.alloc(R));
    RCP_CUDA(counters.alloc(4));
    RCP_CUDA(err.alloc(2));
    RCP_CUDA(child.alloc(R));
    RCP_CUDA(range.alloc(R));
    RCP_CUDA(blo.alloc(R));
    RCP_CUDA(bhi.alloc(R));
    RCP_CUDA(parent_int.alloc(R));
    RCP_CUDA(parent_leaf.alloc(R));
    RCP_CUDA(fa.alloc(n_nodes_cap));
    RCP_CUDA(fb.alloc(n_nodes_cap));
    RCP_CUDA(scratch.alloc(radix_sort_scratch_bytes(R)));
    // outputs sized for the worst case, trimmed at the end
    DevBuf<WNode> nodes_full;
    DevBuf<float4> nbox_full, prims, rec_box;
    RCP_CUDA(nodes_full.alloc(n_nodes_cap));
    RCP_CUDA(nbox_full.alloc(2 * n_nodes_cap));
    RCP_CUDA(prims.alloc(3 * R));
    if (split) RCP_CUDA(rec_box.alloc(2 * R));
    RCP_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(int), st));
    RCP_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(uint32_t) * 4, st));
    k_morton<<<grid_for(R, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(ref_lo, ref_hi, R, bounds.p, keys.p, vals.p);
    rcp_status rs = radix_sort_pairs(keys.p, vals.p, akeys.p, avals.p, R, 30, scratch.p, err.p, st);
    if (rs != RCP_OK) return rs;
    uint32_t* ids = vals.p;  // reference indices in leaf order (Morton order, then depth-first)
    DevBuf<float4> dp;
    DevBuf<uint2> slot_split;
    DevBuf<int> arrivals;
    if (R >= 2) {
        // a sort whose look-back wait ran out leaves no valid permutation to cluster
        int sort_flag = 0;
        RCP_CUDA(cudaMemcpyAsync(&sort_flag, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        RCP_CUDA(cudaStreamSynchronize(st));
        if (sort_flag) {
            set_error("radix sort: look-back wait ran out");
            return RCP_ERR_TIMEOUT;
        }
        rcp_status pr = build_ploc(R, vals.p, avals.p, ref_lo, ref_hi, child.p, range.p, blo.p, bhi.p, parent_int.p,
                                   parent_leaf.p, err.p + 1, cap, st);
        if (pr != RCP_OK) {
            return pr;
        }
        ids = avals.p;
    }
    if (R >= 2) {
        // node boxes from the padded leaves (the clustering used exact boxes)
        RCP_CUDA(arrivals.alloc(R - 1));
        RCP_CUDA(cudaMemsetAsync(arrivals.p, 0, sizeof(int) * (R - 1), st));
        k_refit_padded<<<grid_for(R, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(
            child.p, parent_int.p, parent_leaf.p, ids, ref_lo, ref_hi, split ? rprim.p : nullptr, sc.d_tri,
            sc.d_sph, T, R, blo.p, bhi.p, arrivals.p, err.p + 1);
    }
    if (R >= 2 && sc.collapse == RCP_COLLAPSE_SAH) {
        RCP_CUDA(dp.alloc(2 * (R - 1)));
        RCP_CUDA(slot_split.alloc(R - 1));
        RCP_CUDA(cudaMemsetAsync(arrivals.p, 0, sizeof(int) * (R - 1), st));
        k_sah_dp<<<grid_for(R, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(child.p, range.p, parent_int.p,
                                                                         parent_leaf.p, blo.p, bhi.p, ref_lo, ref_hi,
                                                                         ids, R, dp.p, slot_split.p, arrivals.p,
                                                                         err.p + 1);
    }
    // scene bounds -> diameter
    uint32_t hb[12];
    RCP_CUDA(cudaMemcpyAsync(hb, bounds.p, sizeof(hb), cudaMemcpyDeviceToHost, st));
    RCP_CUDA(cudaStreamSynchronize(st));
    auto ord2f_h = [](uint32_t u) {
        uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
        float f;
        memcpy(&f, &v, 4);
        return f;
    };
    if (N > 0) {
        float d2 = 0.f;
        for (int a = 0; a < 3; ++a) {
            const float ext = ord2f_h(hb[9 + a]) - ord2f_h(hb[6 + a]);
            d2 += ext * ext;
        }
        sc.diam = sqrtf(d2);
    } else {
        sc.diam = 0.f;
    }

    // collapse, level by level
    std::vector<int64_t> level_begin;
    int depth = 0;
    int64_t n_nodes = 0;
    if (N > 0) {
        int2 root = make_int2(R >= 2 ? 0 : -1, 0);
        RCP_CUDA(cudaMemcpyAsync(fa.p, &root, sizeof(int2), cudaMemcpyHostToDevice, st));
        uint32_t one = 1;
        RCP_CUDA(cudaMemcpyAsync(counters.p, &one, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        int* d_max_leaf = err.p;  // reuse: err[0] is the sort's flag, checked below before reuse
        int herr[2] = {0, 0};
        RCP_CUDA(cudaMemcpyAsync(herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, st));
        RCP_CUDA(cudaStreamSynchronize(st));
        if (herr[1]) {
            set_error("BVH build: the clustered tree is malformed (a path to the root too long or a leaf out of range)");
            return RCP_ERR_STATE;
        }
        if (herr[0]) {
            set_error("radix sort: look-back wait ran out");
            return RCP_ERR_TIMEOUT;
        }
        RCP_CUDA(cudaMemsetAsync(d_max_leaf, 0, sizeof(int), st));
        BinTree bt{child.p, range.p, blo.p, bhi.p, ref_lo, ref_hi, ids,
                   sc.collapse == RCP_COLLAPSE_SAH ? slot_split.p : nullptr, split ? rprim.p : nullptr, sc.d_tri,
                   sc.d_sph, T};
        int n_front = 1;
        int64_t begin = 0;
        int2* cur = fa.p;
        int2* nxt = fb.p;
        while (n_front > 0) {
            if (depth >= 512) {
                set_error("BVH collapse did not terminate (corrupted binary tree)");
                return RCP_ERR_STATE;
            }
            level_begin.push_back(begin);
            ++depth;
            RCP_CUDA(cudaMemsetAsync(counters.p + 2, 0, sizeof(uint32_t), st));
            k_collapse<<<(n_front + 127) / 128, 128, 0, st>>>(bt, cur, n_front, nxt, counters.p, nodes_full.p,
                                                               nbox_full.p, prims.p, sc.d_tri, sc.d_sph, T, d_max_leaf,
                                                               rec_box.p);
            uint32_t hc[3];
            RCP_CUDA(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
            RCP_CUDA(cudaStreamSynchronize(st));
            begin += n_front;
            n_front = (int)hc[2];
            n_nodes = hc[0];
            std::swap(cur, nxt);
        }
        level_begin.push_back(begin);
        RCP_CUDA(cudaMemcpyAsync(&sc.max_leaf, d_max_leaf, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    // the parts of split references, for refits
    DevBuf<uint32_t> part_uv, rec_id;
    if (split) {
        RCP_CUDA(part_uv.alloc(PART_MAX * R));
        RCP_CUDA(rec_id.alloc(R));
        k_record_parts<<<grid_for(R, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(prims.p, R, rec_box.p, sc.d_tri, T,
                                                                               part_uv.p, rec_id.p);
    }
    // trim the node arrays to size
    if (sc.d_nodes) cudaFree(sc.d_nodes);
    if (sc.d_nbox) cudaFree(sc.d_nbox);
    if (sc.d_prims) cudaFree(sc.d_prims);
    if (sc.d_refbox) cudaFree(sc.d_refbox);
    if (sc.d_part_uv) cudaFree(sc.d_part_uv);
    if (sc.d_rec_id) cudaFree(sc.d_rec_id);
    if (sc.d_rbox) cudaFree(sc.d_rbox);
    sc.d_rbox = nullptr;
    sc.d_part_uv = nullptr;
    sc.d_rec_id = nullptr;
    sc.d_nodes = nullptr;
    sc.d_nbox = nullptr;
    sc.d_prims = nullptr;
    sc.d_refbox = nullptr;
    RCP_CUDA(cudaMalloc((void**)&sc.d_nodes, sizeof(WNode) * (n_nodes ? n_nodes : 1)));
    RCP_CUDA(cudaMalloc((void**)&sc.d_nbox, sizeof(float4) * 2 * (n_nodes ? n_nodes : 1)));
    if (n_nodes) {
        RCP_CUDA(cudaMemcpyAsync(sc.d_nodes, nodes_full.p, sizeof(WNode) * n_nodes, cudaMemcpyDeviceToDevice, st));
        RCP_CUDA(cudaMemcpyAsync(sc.d_nbox, nbox_full.p, sizeof(float4) * 2 * n_nodes, cudaMemcpyDeviceToDevice,
                                 st));
    }
    RCP_CUDA(cudaEventRecord(ev.b, st));
    RCP_CUDA(cudaStreamSynchronize(st));
    sc.d_prims = prims.release();
    sc.d_refbox = rec_box.release();
    sc.d_part_uv = part_uv.release();
    sc.d_rec_id = rec_id.release();
    sc.n_records = R;
    sc.n_nodes = n_nodes;
    sc.depth = depth;
    sc.level_begin = level_begin;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    sc.build_ms = ms;
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

rcp_status refit_bvh(Scene& sc, cudaStream_t st) {
    const int64_t N = sc.T + sc.S;
    if (N == 0 || sc.n_nodes == 0) return RCP_OK;
    // a split build's references are bounded by their parts of the moved
    // triangles; the build-time reference boxes no longer apply
    if (sc.d_refbox) {
        RCP_CUDA(cudaStreamSynchronize(st));
        cudaFree(sc.d_refbox);
        sc.d_refbox = nullptr;
    }
    if (!sc.d_rbox) RCP_CUDA(cudaMalloc((void**)&sc.d_rbox, sizeof(float2) * 3 * sc.n_records));
    EventPair ev;
    RCP_CUDA(ev.create());
    RCP_CUDA(cudaEventRecord(ev.a, st));
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_refit_records<<<grid_for(sc.n_records, BUILD_BLOCK, sms * 16), BUILD_BLOCK, 0, st>>>(
        sc.d_prims, sc.n_records, Parts{sc.d_part_uv, sc.d_rec_id}, sc.d_tri, sc.d_sph, sc.T, sc.d_rbox);
    for (int l = (int)sc.level_begin.size() - 2; l >= 0; --l) {
        const int64_t b = sc.level_begin[l], e = sc.level_begin[l + 1];
        if (e <= b) continue;
        k_refit_wide<<<(int)((8 * (e - b) + REFIT_BLOCK - 1) / REFIT_BLOCK), REFIT_BLOCK, 0, st>>>(
            (WNode*)sc.d_nodes, sc.d_nbox, b, e, sc.d_rbox);
    }
    RCP_CUDA(cudaEventRecord(ev.b, st));
    RCP_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    sc.build_ms = ms;
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

rcp_status validate_bvh(const Scene& sc, cudaStream_t st) {
    const int64_t N = sc.T + sc.S, R = sc.n_records;
    if (N == 0) return RCP_OK;
    DevBuf<unsigned> seen_rec, seen_id, node_refs;
    DevBuf<int> errors;
    RCP_CUDA(seen_rec.alloc(R));
    RCP_CUDA(seen_id.alloc(N));
    RCP_CUDA(node_refs.alloc(sc.n_nodes));
    RCP_CUDA(errors.alloc(8));
    RCP_CUDA(cudaMemsetAsync(seen_rec.p, 0, sizeof(unsigned) * R, st));
    RCP_CUDA(cudaMemsetAsync(seen_id.p, 0, sizeof(unsigned) * N, st));
    RCP_CUDA(cudaMemsetAsync(node_refs.p, 0, sizeof(unsigned) * sc.n_nodes, st));
    RCP_CUDA(cudaMemsetAsync(errors.p, 0, sizeof(int) * 8, st));
    k_validate<<<(int)((sc.n_nodes + 127) / 128), 128, 0, st>>>((const WNode*)sc.d_nodes, sc.n_nodes, sc.d_nbox,
                                                                 sc.d_prims, R, N, sc.d_refbox,
                                                                 Parts{sc.d_part_uv, sc.d_rec_id}, sc.d_tri, sc.d_sph,
                                                                 sc.T, seen_rec.p, seen_id.p, node_refs.p, errors.p);
    k_check_counts<<<grid_for(std::max<int64_t>(std::max(R, N), sc.n_nodes), 256, 4096), 256, 0, st>>>(
        seen_rec.p, R, seen_id.p, N, sc.split_max > 1, node_refs.p, sc.n_nodes, errors.p);
    int h[8];
    RCP_CUDA(cudaMemcpyAsync(h, errors.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RCP_CUDA(cudaStreamSynchronize(st));
    static const char* what[8] = {"slot masks",       "child index order", "child box outside slot",
                                  "leaf record range", "primitive outside leaf slot",
                                  "record not referenced exactly once", "primitive id missing or repeated",
                                  "node not referenced exactly once"};
    for (int i = 0; i < 8; ++i)
        if (h[i]) {
            set_error(std::string("BVH validation failed: ") + what[i] + " (" + std::to_string(h[i]) + ")");
            return RCP_ERR_STATE;
        }
    return RCP_OK;
}

rcp_status debug_morton(const float* xyz, int64_t n, const float* lo, const float* hi, uint32_t* codes,
                        cudaStream_t st) {
    if (n <= 0) return RCP_OK;
    k_morton_points<<<grid_for(n, 256, 4096), 256, 0, st>>>(xyz, n, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2],
                                                             codes);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

}  // namespace rcp
