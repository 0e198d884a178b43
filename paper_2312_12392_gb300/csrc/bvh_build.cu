// bvh_build.cu -- GPU LBVH builder collapsed to a compressed 8-wide BVH.
//
// The paper (§6) traced its scenes with OptiX and says nothing about the
// acceleration structure; this builder serves the scene S(n) of §2, Eq. 1.
// Steps, all on the device:
//  1. primitive boxes and centroids; scene and centroid bounds (atomic min/max
//     on order-preserving integer images of the floats);
//  2. 30-bit Morton codes of the centroids (10 bits per axis);
//  3. radix sort of (code, primitive) pairs (radix_sort.cu);
//  4. binary radix tree over the sorted codes: Karras's construction, one
//     thread per internal node, equal codes ordered by index;
//  5. bottom-up box refit, one thread per leaf, the second arrival at each
//     node continuing upwards (atomic arrival counters);
//  6. collapse to 8-wide nodes, one launch per level: each wide node takes a
//     binary node's two children and repeatedly opens the child with the
//     largest surface area that holds more than 3 primitives, until 8 children
//     or none left to open. Subtrees of <= 3 primitives become leaves. Children
//     are placed in slots so that slot order approximates front-to-back order
//     per ray octant; boxes are quantised to 8 bits against a per-node origin
//     and power-of-two scale, rounded outwards with a small pad. Leaf
//     primitives are copied into 48-byte records, contiguous per node.
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
__device__ __forceinline__ uint32_t morton30(float x, float y, float z, const float* lo, const float* hi) {
    const float c[3] = {x, y, z};
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        const float ext = hi[a] - lo[a];
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

// Length of the common prefix of sorted keys i and j; equal keys extend the
// comparison with the indices themselves (so every key is distinct). -1 when j
// is out of range.
__device__ __forceinline__ int delta(const uint32_t* __restrict__ k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = k[i], b = k[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((uint32_t)i ^ (uint32_t)j);
}

// Binary radix tree (Karras 2012): internal node i covers a key range that
// starts or ends at i. Children refs: >= 0 internal node, < 0 leaf -(j+1).
__global__ void k_karras(const uint32_t* __restrict__ k, int64_t n, int2* __restrict__ child,
                         int2* __restrict__ range, int* __restrict__ parent_int, int* __restrict__ parent_leaf) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 1; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
        const int dmin = delta(k, n, i, i - d);
        int64_t lmax = 2;
        while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
        int64_t l = 0;
        for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
            if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
        const int64_t j = i + l * d;
        const int dnode = delta(k, n, i, j);
        int64_t s = 0;
        int64_t t = l;
        do {
            t = (t + 1) >> 1;
            if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        } while (t > 1);
        const int64_t gamma = i + s * d + min(d, 0);
        const int64_t lo = min(i, j), hi = max(i, j);
        const int left = (lo == gamma) ? -(int)(gamma + 1) : (int)gamma;
        const int right = (hi == gamma + 1) ? -(int)(gamma + 2) : (int)(gamma + 1);
        child[i] = make_int2(left, right);
        range[i] = make_int2((int)lo, (int)hi);
        if (left >= 0) parent_int[left] = (int)i;
        else parent_leaf[-left - 1] = (int)i;
        if (right >= 0) parent_int[right] = (int)i;
        else parent_leaf[-right - 1] = (int)i;
    }
}

// Bottom-up refit: one thread per leaf; at each internal node the second
// arriving thread merges both children and goes on (the first stops).
__global__ void k_refit_binary(const uint32_t* __restrict__ sorted_ids, int64_t n, const float4* __restrict__ plo,
                               const float4* __restrict__ phi, const int2* __restrict__ child,
                               const int* __restrict__ parent_int, const int* __restrict__ parent_leaf,
                               float4* blo, float4* bhi, int* arrivals) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        int node = parent_leaf[j];
        int guard = 0;
        while (node >= 0 && ++guard < 4096) {
            __threadfence();
            if (atomicAdd(&arrivals[node], 1) == 0) break;
            __threadfence();
            const int2 c = child[node];
            float4 l[2], h[2];
            const int cs[2] = {c.x, c.y};
            for (int q = 0; q < 2; ++q) {
                if (cs[q] >= 0) {
                    l[q] = __ldcg(&blo[cs[q]]);
                    h[q] = __ldcg(&bhi[cs[q]]);
                } else {
                    const uint32_t id = sorted_ids[-cs[q] - 1];
                    l[q] = plo[id];
                    h[q] = phi[id];
                }
            }
            __stcg(&blo[node], make_float4(fminf(l[0].x, l[1].x), fminf(l[0].y, l[1].y), fminf(l[0].z, l[1].z), 0.f));
            __stcg(&bhi[node], make_float4(fmaxf(h[0].x, h[1].x), fmaxf(h[0].y, h[1].y), fmaxf(h[0].z, h[1].z), 0.f));
            node = parent_int[node];
        }
    }
}

struct BinTree {
    const int2* child;
    const int2* range;
    const float4* blo;
    const float4* bhi;
    const float4* plo;
    const float4* phi;
    const uint32_t* sorted_ids;
};

__device__ __forceinline__ void ref_box(const BinTree& bt, int ref, float3& lo, float3& hi, int& first, int& last) {
    float4 l, h;
    if (ref >= 0) {
        l = bt.blo[ref];
        h = bt.bhi[ref];
        const int2 r = bt.range[ref];
        first = r.x;
        last = r.y;
    } else {
        const int j = -ref - 1;
        const uint32_t id = bt.sorted_ids[j];
        l = bt.plo[id];
        h = bt.phi[id];
        first = last = j;
    }
    lo = make_float3(l.x, l.y, l.z);
    hi = make_float3(h.x, h.y, h.z);
}

}  // namespace

// Quantise up to 8 child boxes against their union. Writes the node's origin,
// exponents and q bytes (empty slots get an inverted box); returns the union.
__device__ void quantise_node(WNode& nd, const float3* clo, const float3* chi, const int* slot_of, int m,
                              float3& ulo, float3& uhi) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int c = 0; c < m; ++c) {
        const double l[3] = {clo[c].x, clo[c].y, clo[c].z}, h[3] = {chi[c].x, chi[c].y, chi[c].z};
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], l[a]);
            hi[a] = fmax(hi[a], h[a]);
        }
    }
    ulo = make_float3((float)lo[0], (float)lo[1], (float)lo[2]);
    uhi = make_float3((float)hi[0], (float)hi[1], (float)hi[2]);
    double ext = fmax(fmax(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    double mag = fmax(fmax(fabs(lo[0]), fabs(hi[0])), fmax(fmax(fabs(lo[1]), fabs(hi[1])), fmax(fabs(lo[2]), fabs(hi[2]))));
    double pad = ext > 0.0 ? ldexp(ext, -18) : ldexp(mag, -18) + 1e-30;
    float p[3];
    int e[3];
    double s[3];
    for (int a = 0; a < 3; ++a) {
        p[a] = __double2float_rd(lo[a] - pad);
        const double span = (hi[a] + pad) - (double)p[a];
        int x = 0;
        frexp(span / 255.0, &x);  // span/255 = m 2^x, m in [0.5, 1) -> 255 * 2^x >= span
        x = max(x, -120);
        x = min(x, 40);  // keeps 256 * 2^x / |d| finite for |d| >= 1e-20
        e[a] = x;
        s[a] = ldexp(1.0, x);
    }
    nd.px = p[0];
    nd.py = p[1];
    nd.pz = p[2];
    uint32_t qlo[3][2] = {{0xffffffffu, 0xffffffffu}, {0xffffffffu, 0xffffffffu}, {0xffffffffu, 0xffffffffu}};
    uint32_t qhi[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int c = 0; c < m; ++c) {
        const int sl = slot_of[c];
        const double l[3] = {clo[c].x, clo[c].y, clo[c].z}, h[3] = {chi[c].x, chi[c].y, chi[c].z};
        for (int a = 0; a < 3; ++a) {
            double ql = floor((l[a] - pad - (double)p[a]) / s[a]);
            double qh = ceil((h[a] + pad - (double)p[a]) / s[a]);
            ql = fmin(fmax(ql, 0.0), 255.0);
            qh = fmin(fmax(qh, 0.0), 255.0);
            const int sh = 8 * (sl & 3);
            qlo[a][sl >> 2] = (qlo[a][sl >> 2] & ~(0xffu << sh)) | ((uint32_t)ql << sh);
            qhi[a][sl >> 2] = (qhi[a][sl >> 2] & ~(0xffu << sh)) | ((uint32_t)qh << sh);
        }
    }
    for (int w = 0; w < 2; ++w) {
        nd.qlo_x[w] = qlo[0][w];
        nd.qlo_y[w] = qlo[1][w];
        nd.qlo_z[w] = qlo[2][w];
        nd.qhi_x[w] = qhi[0][w];
        nd.qhi_y[w] = qhi[1][w];
        nd.qhi_z[w] = qhi[2][w];
    }
    nd.e_imask = (nd.e_imask & 0xff000000u) | (uint32_t)(e[0] + 127) | ((uint32_t)(e[1] + 127) << 8) |
                 ((uint32_t)(e[2] + 127) << 16);
}

__device__ __forceinline__ void write_prim_record(float4* __restrict__ rec, const float* __restrict__ tri,
                                                  const float* __restrict__ sph, int64_t T, uint32_t id) {
    if (id < T) {
        const float* v = tri + 9 * (int64_t)id;
        float e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        float e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        // exact double cross product of the float edges: zero only for degenerate triangles
        const double d1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
        const double d2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
        const double nx = d1[1] * d2[2] - d1[2] * d2[1], ny = d1[2] * d2[0] - d1[0] * d2[2],
                     nz = d1[0] * d2[1] - d1[1] * d2[0];
        if (nx == 0.0 && ny == 0.0 && nz == 0.0)
            for (int a = 0; a < 3; ++a) e1[a] = e2[a] = 0.f;  // never hit (det == 0)
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
__global__ void k_collapse(BinTree bt, const int2* __restrict__ frontier, int n_front, int2* __restrict__ next_front,
                           uint32_t* counters, WNode* __restrict__ nodes, float4* __restrict__ nbox,
                           float4* __restrict__ prims, const float* __restrict__ tri, const float* __restrict__ sph,
                           int64_t T, int* max_leaf) {
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
    } else {
        const int2 c = bt.child[ref];
        cref[0] = c.x;
        cref[1] = c.y;
        m = 2;
    }
    for (int c = 0; c < m; ++c) ref_box(bt, cref[c], clo[c], chi[c], cfirst[c], clast[c]);
    while (m < 8) {
        int best = -1;
        float best_area = -1.f;
        for (int c = 0; c < m; ++c) {
            if (cref[c] < 0 || clast[c] - cfirst[c] + 1 <= 3) continue;
            const float dx = chi[c].x - clo[c].x, dy = chi[c].y - clo[c].y, dz = chi[c].z - clo[c].z;
            const float area = dx * dy + dy * dz + dz * dx;
            if (area > best_area) {
                best_area = area;
                best = c;
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
        is_int[c] = cref[c] >= 0 && clast[c] - cfirst[c] + 1 > 3;
        if (is_int[c]) ++n_int;
        else n_prim += clast[c] - cfirst[c] + 1;
    }
    const uint32_t child_base = n_int ? atomicAdd(&counters[0], (uint32_t)n_int) : 0u;
    const uint32_t prim_base = n_prim ? atomicAdd(&counters[1], (uint32_t)n_prim) : 0u;
    WNode nd;
    nd.e_imask = 0;
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
            for (int q = 0; q < cnt; ++q)
                write_prim_record(prims + 3 * (int64_t)(prim_base + poff + q), tri, sph, T,
                                  bt.sorted_ids[cfirst[c] + q]);
            poff += cnt;
            leaf_max = max(leaf_max, cnt);
        }
        meta[s >> 2] |= mb << (8 * (s & 3));
    }
    nd.meta_lo = meta[0];
    nd.meta_hi = meta[1];
    nd.e_imask = imask << 24;
    float3 ulo, uhi;
    quantise_node(nd, clo, chi, slot_of, m, ulo, uhi);
    nodes[w] = nd;
    nbox[2 * w] = make_float4(ulo.x, ulo.y, ulo.z, 0.f);
    nbox[2 * w + 1] = make_float4(uhi.x, uhi.y, uhi.z, 0.f);
    if (leaf_max) atomicMax(max_leaf, leaf_max);
}

// ---------------------------------------------------------------- refit after a vertex update

__global__ void k_update_records(float4* __restrict__ prims, int64_t n, const float* __restrict__ tri,
                                 const float* __restrict__ sph, int64_t T) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t idb = __float_as_uint(prims[3 * r + 2].y);
        if (idb & SPHERE_BIT) continue;
        write_prim_record(prims + 3 * r, tri, sph, T, idb);
    }
}

__device__ __forceinline__ void record_box(const float4* __restrict__ prims, int64_t r, const float* __restrict__ tri,
                                           const float* __restrict__ sph, int64_t T, float3& lo, float3& hi) {
    const uint32_t idb = __float_as_uint(prims[3 * r + 2].y);
    prim_box(tri, sph, T, (int64_t)(idb & ~SPHERE_BIT), lo, hi);
}

// Recompute the child boxes of the nodes in [begin, end) (one level, deepest
// first) from their leaves' primitives and their internal children's boxes.
__global__ void k_refit_wide(WNode* __restrict__ nodes, float4* __restrict__ nbox, int64_t begin, int64_t end,
                             const float4* __restrict__ prims, const float* __restrict__ tri,
                             const float* __restrict__ sph, int64_t T) {
    const int64_t w = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= end) return;
    WNode nd = nodes[w];
    float3 clo[8], chi[8];
    int slot_of[8];
    int m = 0;
    const uint32_t imask = nd.e_imask >> 24;
    for (int s = 0; s < 8; ++s) {
        const uint32_t mb = ((s < 4 ? nd.meta_lo : nd.meta_hi) >> (8 * (s & 3))) & 0xffu;
        if (!mb) continue;
        float3 lo, hi;
        if (mb & 0x80u) {
            const int64_t c = nd.child_base + __popc(imask & ((1u << s) - 1u));
            const float4 l = nbox[2 * c], h = nbox[2 * c + 1];
            lo = make_float3(l.x, l.y, l.z);
            hi = make_float3(h.x, h.y, h.z);
        } else {
            const int cnt = mb >> 5, off = mb & 31;
            record_box(prims, nd.prim_base + off, tri, sph, T, lo, hi);
            for (int q = 1; q < cnt; ++q) {
                float3 l2, h2;
                record_box(prims, nd.prim_base + off + q, tri, sph, T, l2, h2);
                lo = make_float3(fminf(lo.x, l2.x), fminf(lo.y, l2.y), fminf(lo.z, l2.z));
                hi = make_float3(fmaxf(hi.x, h2.x), fmaxf(hi.y, h2.y), fmaxf(hi.z, h2.z));
            }
        }
        clo[m] = lo;
        chi[m] = hi;
        slot_of[m] = s;
        ++m;
    }
    float3 ulo, uhi;
    quantise_node(nd, clo, chi, slot_of, m, ulo, uhi);
    nodes[w] = nd;
    nbox[2 * w] = make_float4(ulo.x, ulo.y, ulo.z, 0.f);
    nbox[2 * w + 1] = make_float4(uhi.x, uhi.y, uhi.z, 0.f);
}

// ---------------------------------------------------------------- validation

__device__ __forceinline__ void slot_box(const WNode& nd, int s, double lo[3], double hi[3]) {
    const float p[3] = {nd.px, nd.py, nd.pz};
    const uint32_t* ql[3] = {nd.qlo_x, nd.qlo_y, nd.qlo_z};
    const uint32_t* qh[3] = {nd.qhi_x, nd.qhi_y, nd.qhi_z};
    for (int a = 0; a < 3; ++a) {
        const double sc = ldexp(1.0, (int)((nd.e_imask >> (8 * a)) & 0xffu) - 127);
        lo[a] = (double)p[a] + sc * (double)((ql[a][s >> 2] >> (8 * (s & 3))) & 0xffu);
        hi[a] = (double)p[a] + sc * (double)((qh[a][s >> 2] >> (8 * (s & 3))) & 0xffu);
    }
}

__global__ void k_validate(const WNode* __restrict__ nodes, int64_t n_nodes, const float4* __restrict__ nbox,
                           const float4* __restrict__ prims, int64_t n_prims, const float* __restrict__ tri,
                           const float* __restrict__ sph, int64_t T, unsigned* __restrict__ seen_rec,
                           unsigned* __restrict__ seen_id, unsigned* __restrict__ node_refs, int* errors) {
    const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w >= n_nodes) return;
    const WNode nd = nodes[w];
    const uint32_t imask = nd.e_imask >> 24;
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
                if (r >= n_prims) {
                    atomicAdd(&errors[3], 1);
                    continue;
                }
                atomicAdd(&seen_rec[r], 1u);
                const uint32_t id = __float_as_uint(prims[3 * r + 2].y) & ~SPHERE_BIT;
                if (id < (uint32_t)n_prims) atomicAdd(&seen_id[id], 1u);
                float3 pl, ph;
                prim_box(tri, sph, T, id, pl, ph);
                if (pl.x < lo[0] || pl.y < lo[1] || pl.z < lo[2] || ph.x > hi[0] || ph.y > hi[1] || ph.z > hi[2])
                    atomicAdd(&errors[4], 1);
            }
        }
    }
}

__global__ void k_check_counts(const unsigned* a, const unsigned* b, int64_t n, const unsigned* node_refs,
                               int64_t n_nodes, int* errors) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (a[i] != 1u) atomicAdd(&errors[5], 1);
        if (b[i] != 1u) atomicAdd(&errors[6], 1);
    }
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

template <class T>
struct DevBuf {
    T* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc((void**)&p, sizeof(T) * (n ? n : 1)); }
};

}  // namespace

rcp_status build_bvh(Scene& sc, cudaStream_t st) {
    const int64_t T = sc.T, N = sc.T + sc.S;
    const int64_t n_nodes_cap = N > 1 ? N : 1;
    cudaEvent_t e0, e1;
    RCP_CUDA(cudaEventCreate(&e0));
    RCP_CUDA(cudaEventCreate(&e1));
    RCP_CUDA(cudaEventRecord(e0, st));
    DevBuf<float4> plo, phi, blo, bhi;
    DevBuf<uint32_t> keys, vals, akeys, avals, bounds, counters;
    DevBuf<int2> child, range, fa, fb;
    DevBuf<int> parent_int, parent_leaf, arrivals, err;
    DevBuf<char> scratch;
    RCP_CUDA(plo.alloc(N));
    RCP_CUDA(phi.alloc(N));
    RCP_CUDA(keys.alloc(N));
    RCP_CUDA(vals.alloc(N));
    RCP_CUDA(akeys.alloc(N));
    RCP_CUDA(avals.alloc(N));
    RCP_CUDA(bounds.alloc(12));
    RCP_CUDA(counters.alloc(4));
    RCP_CUDA(err.alloc(1));
    RCP_CUDA(child.alloc(N));
    RCP_CUDA(range.alloc(N));
    RCP_CUDA(blo.alloc(N));
    RCP_CUDA(bhi.alloc(N));
    RCP_CUDA(parent_int.alloc(N));
    RCP_CUDA(parent_leaf.alloc(N));
    RCP_CUDA(arrivals.alloc(N));
    RCP_CUDA(fa.alloc(n_nodes_cap));
    RCP_CUDA(fb.alloc(n_nodes_cap));
    RCP_CUDA(scratch.alloc(radix_sort_scratch_bytes(N)));
    // outputs sized for the worst case, trimmed at the end
    WNode* nodes_full = nullptr;
    float4* nbox_full = nullptr;
    RCP_CUDA(cudaMalloc((void**)&nodes_full, sizeof(WNode) * n_nodes_cap));
    RCP_CUDA(cudaMalloc((void**)&nbox_full, sizeof(float4) * 2 * n_nodes_cap));
    float4* prims = nullptr;
    RCP_CUDA(cudaMalloc((void**)&prims, sizeof(float4) * 3 * (N ? N : 1)));

    int sms = 148;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int cap = sms * 16;
    RCP_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    RCP_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(uint32_t) * 4, st));
    k_init_bounds<<<1, 32, 0, st>>>(bounds.p);
    k_prim_bounds<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(sc.d_tri, sc.d_sph, T, N, plo.p, phi.p,
                                                                          bounds.p);
    k_morton<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(plo.p, phi.p, N, bounds.p, keys.p, vals.p);
    rcp_status rs = radix_sort_pairs(keys.p, vals.p, akeys.p, avals.p, N, 30, scratch.p, err.p, st);
    if (rs != RCP_OK) return rs;
    if (N >= 2) {
        RCP_CUDA(cudaMemsetAsync(arrivals.p, 0, sizeof(int) * N, st));
        k_karras<<<grid_for(N - 1, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(keys.p, N, child.p, range.p,
                                                                             parent_int.p, parent_leaf.p);
        // the root has no parent
        int minus1 = -1;
        RCP_CUDA(cudaMemcpyAsync(parent_int.p, &minus1, sizeof(int), cudaMemcpyHostToDevice, st));
        k_refit_binary<<<grid_for(N, BUILD_BLOCK, cap), BUILD_BLOCK, 0, st>>>(
            vals.p, N, plo.p, phi.p, child.p, parent_int.p, parent_leaf.p, blo.p, bhi.p, arrivals.p);
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
        int2 root = make_int2(N >= 2 ? 0 : -1, 0);
        RCP_CUDA(cudaMemcpyAsync(fa.p, &root, sizeof(int2), cudaMemcpyHostToDevice, st));
        uint32_t one = 1;
        RCP_CUDA(cudaMemcpyAsync(counters.p, &one, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
        int* d_max_leaf = err.p;  // reuse: err[0] is the sort's flag, checked below before reuse
        int sort_err = 0;
        RCP_CUDA(cudaMemcpyAsync(&sort_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        RCP_CUDA(cudaStreamSynchronize(st));
        if (sort_err) {
            set_error("radix sort: look-back wait ran out");
            cudaFree(nodes_full);
            cudaFree(nbox_full);
            cudaFree(prims);
            return RCP_ERR_TIMEOUT;
        }
        RCP_CUDA(cudaMemsetAsync(d_max_leaf, 0, sizeof(int), st));
        BinTree bt{child.p, range.p, blo.p, bhi.p, plo.p, phi.p, vals.p};
        int n_front = 1;
        int64_t begin = 0;
        int2* cur = fa.p;
        int2* nxt = fb.p;
        while (n_front > 0) {
            if (depth >= 512) {
                set_error("BVH collapse did not terminate (corrupted binary tree)");
                cudaFree(nodes_full);
                cudaFree(nbox_full);
                cudaFree(prims);
                return RCP_ERR_STATE;
            }
            level_begin.push_back(begin);
            ++depth;
            RCP_CUDA(cudaMemsetAsync(counters.p + 2, 0, sizeof(uint32_t), st));
            k_collapse<<<(n_front + 127) / 128, 128, 0, st>>>(bt, cur, n_front, nxt, counters.p, nodes_full,
                                                               nbox_full, prims, sc.d_tri, sc.d_sph, T, d_max_leaf);
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
    // trim the node arrays to size
    if (sc.d_nodes) cudaFree(sc.d_nodes);
    if (sc.d_nbox) cudaFree(sc.d_nbox);
    if (sc.d_prims) cudaFree(sc.d_prims);
    sc.d_nodes = nullptr;
    sc.d_nbox = nullptr;
    RCP_CUDA(cudaMalloc((void**)&sc.d_nodes, sizeof(WNode) * (n_nodes ? n_nodes : 1)));
    RCP_CUDA(cudaMalloc((void**)&sc.d_nbox, sizeof(float4) * 2 * (n_nodes ? n_nodes : 1)));
    if (n_nodes) {
        RCP_CUDA(cudaMemcpyAsync(sc.d_nodes, nodes_full, sizeof(WNode) * n_nodes, cudaMemcpyDeviceToDevice, st));
        RCP_CUDA(cudaMemcpyAsync(sc.d_nbox, nbox_full, sizeof(float4) * 2 * n_nodes, cudaMemcpyDeviceToDevice, st));
    }
    RCP_CUDA(cudaEventRecord(e1, st));
    RCP_CUDA(cudaStreamSynchronize(st));
    cudaFree(nodes_full);
    cudaFree(nbox_full);
    sc.d_prims = prims;
    sc.n_nodes = n_nodes;
    sc.depth = depth;
    sc.level_begin = level_begin;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    sc.build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

rcp_status refit_bvh(Scene& sc, cudaStream_t st) {
    const int64_t N = sc.T + sc.S;
    if (N == 0 || sc.n_nodes == 0) return RCP_OK;
    cudaEvent_t e0, e1;
    RCP_CUDA(cudaEventCreate(&e0));
    RCP_CUDA(cudaEventCreate(&e1));
    RCP_CUDA(cudaEventRecord(e0, st));
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_update_records<<<grid_for(N, BUILD_BLOCK, sms * 16), BUILD_BLOCK, 0, st>>>(sc.d_prims, N, sc.d_tri, sc.d_sph,
                                                                                 sc.T);
    for (int l = (int)sc.level_begin.size() - 2; l >= 0; --l) {
        const int64_t b = sc.level_begin[l], e = sc.level_begin[l + 1];
        if (e <= b) continue;
        k_refit_wide<<<(int)((e - b + 127) / 128), 128, 0, st>>>((WNode*)sc.d_nodes, sc.d_nbox, b, e, sc.d_prims,
                                                                  sc.d_tri, sc.d_sph, sc.T);
    }
    RCP_CUDA(cudaEventRecord(e1, st));
    RCP_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    sc.build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

rcp_status validate_bvh(const Scene& sc, cudaStream_t st) {
    const int64_t N = sc.T + sc.S;
    if (N == 0) return RCP_OK;
    DevBuf<unsigned> seen_rec, seen_id, node_refs;
    DevBuf<int> errors;
    RCP_CUDA(seen_rec.alloc(N));
    RCP_CUDA(seen_id.alloc(N));
    RCP_CUDA(node_refs.alloc(sc.n_nodes));
    RCP_CUDA(errors.alloc(8));
    RCP_CUDA(cudaMemsetAsync(seen_rec.p, 0, sizeof(unsigned) * N, st));
    RCP_CUDA(cudaMemsetAsync(seen_id.p, 0, sizeof(unsigned) * N, st));
    RCP_CUDA(cudaMemsetAsync(node_refs.p, 0, sizeof(unsigned) * sc.n_nodes, st));
    RCP_CUDA(cudaMemsetAsync(errors.p, 0, sizeof(int) * 8, st));
    k_validate<<<(int)((sc.n_nodes + 127) / 128), 128, 0, st>>>((const WNode*)sc.d_nodes, sc.n_nodes, sc.d_nbox,
                                                                 sc.d_prims, N, sc.d_tri, sc.d_sph, sc.T,
                                                                 seen_rec.p, seen_id.p, node_refs.p, errors.p);
    k_check_counts<<<grid_for(std::max<int64_t>(N, sc.n_nodes), 256, 4096), 256, 0, st>>>(
        seen_rec.p, seen_id.p, N, node_refs.p, sc.n_nodes, errors.p);
    int h[8];
    RCP_CUDA(cudaMemcpyAsync(h, errors.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RCP_CUDA(cudaStreamSynchronize(st));
    static const char* what[8] = {"slot masks",       "child index order", "child box outside slot",
                                  "leaf record range", "primitive outside leaf slot",
                                  "record not referenced exactly once", "primitive id not exactly once",
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
