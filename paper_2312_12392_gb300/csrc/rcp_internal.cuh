// rcp_internal.cuh -- shared device types of the renderer (not part of the ABI).
//
// Layout in device memory (all 16-byte aligned):
//  * WNode: one 8-wide BVH node with float child boxes, 208 bytes = 13 x float4.
//  * Prim records: 3 x float4 = 48 bytes per primitive, in leaf order:
//      triangle  w0 = (v0.xyz, e1.x)  w1 = (e1.yz, e2.xy)  w2 = (e2.z, id, 0, 0)
//      sphere    w0 = (centre, r)     w1 = 0               w2 = (0, id | SPHERE_BIT, 0, 0)
//    with e1 = v1 - v0, e2 = v2 - v0 (float32), id = the caller's primitive id.
//  * Albedo: float4 per primitive, indexed by id.
//  * Images: float4 per pixel (RGB, hit distance), row-major.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rcp.h"

namespace rcp {

constexpr uint32_t SPHERE_BIT = 0x80000000u;
constexpr int MAX_STACK = 64;  // traversal stack entries (>= BVH depth)

// One 8-wide node, 13 rows of 16 bytes. Child slot s (0..7) has the float
// box lo_a[s]..hi_a[s] per axis a (an empty slot: lo = +inf, hi = -inf), and
// meta[s]: 0 = empty, 0x80 | rank = internal child (node child_base + rank,
// ranks counted in slot order), (count << 5) | offset = leaf of `count` (1..3)
// primitive records at prim_base + offset. Rows 0-1 lo_x, 2-3 hi_x, 4-5 lo_y,
// 6-7 hi_y, 8-9 lo_z, 10-11 hi_z, 12 the header.
struct __align__(16) WNode {
    float lo_x[8], hi_x[8], lo_y[8], hi_y[8], lo_z[8], hi_z[8];
    uint32_t child_base;
    uint32_t prim_base;
    uint32_t meta_lo, meta_hi;  // meta[0..3], meta[4..7]
};
constexpr int NODE_ROWS = 13;
static_assert(sizeof(WNode) == 16 * NODE_ROWS, "WNode must be 13 rows of 16 bytes");

// Slots holding internal children: bit s set when meta byte s has its top bit.
// Each half gathers bits 7, 15, 23, 31 into bits 28..31 with one multiply
// (the partial products below bit 28 never carry into it).
__host__ __device__ __forceinline__ uint32_t internal_mask(uint32_t meta_lo, uint32_t meta_hi) {
    const uint32_t a = ((meta_lo & 0x80808080u) * 0x00204081u) >> 28;
    const uint32_t b = ((meta_hi & 0x80808080u) * 0x00204081u) >> 28;
    return a | (b << 4);
}

struct LightDev {
    int type;
    float x, y, z;
    float ambient;
};

// Device-resident scene: BVH, primitive records and shading data.
struct SceneDev {
    const float4* nodes;   // n_nodes * NODE_ROWS
    const float4* prims;   // n_records * 3
    const float4* albedo;  // n_prims
    int64_t n_prims;
    int64_t n_records;     // leaf records (more than n_prims when triangles are split)
    int64_t n_nodes;
    LightDev light;
    float tmin;  // 1e-6 * diameter
    float eps;   // 1e-4 * diameter (shadow-ray offset)
};

// One view (camera + image) of a batched pass. The camera terms are
// precomputed on the host in double and rounded once:
//   g(x, y) = fF + (2x + 1 - W) fR + (H - 2y - 1) fU  (eye -> focal-plane point)
//   V(c)    = (2c.r - 1) kR + (2c.g - 1) kU + (2c.b - 1) kF
struct ViewDev {
    const struct SceneDev* scene;  // the view's scene (launches over views of several scenes)
    int* status;                   // set to 1 when a walk of this view overflowed its stack (device or host memory)
    float E[3];
    float fF[3], fR[3], fU[3];
    float kR[3], kU[3], kF[3];
    float Fw[3];  // unit view axis F: the z-depth of a hit is t (d . F)
    int W, H;
    int mapping;
    float z0;
    float kpx;  // IMAGE: displacement in pixels; NORMAL: k in world units
    int passes;  // passes a chained launch runs for this view (in: its first input, out: its last output)
    const float4* in;    // previous image, nullptr = I_0
    const float4* base;  // image-space passes: the frame's traced image
    float4* out;         // this pass's image
    int32_t* prim;     // nullable hit ids
    float* rgb;        // nullable: this pass also writes R, G, B (3 floats per pixel, row-major) here,
                       // host memory that the device reads and writes coherently
    int2* hint;        // nullable: per pixel, the record of its latest primary hit and of its latest
                       // shadow occluder (-1 none); tested first, rewritten by every traced pass
    int64_t pix_begin;  // first global pixel index of this view
    int64_t chunk_begin;  // first work chunk (8x4 tile) of this view
    int tiles_x;
    int spp;              // samples per pixel, 0 = one at the centre
    float jit[2 * RCP_MAX_SPP];
    int* done_count;  // nullable: tiles of this view still to finish in the launch (device)
    int* done_flag;   // set to 1 (host-visible) once they have all finished
};

// Host-side owner of a built scene.
struct Scene;

struct Counters {
    unsigned long long rays, primary, shadow, nodes, boxes, tris, spheres;
};

// thread-local error message
void set_error(const std::string& msg);
rcp_status cuda_fail(cudaError_t e, const char* what);

// Owner of one device array, freed on every return path.
template <class T>
struct DevBuf {
    T* p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc((void**)&p, sizeof(T) * (n ? n : 1)); }
    T* release() {
        T* q = p;
        p = nullptr;
        return q;
    }
};

// Two timing events, destroyed on every return path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() = default;
    EventPair(const EventPair&) = delete;
    EventPair& operator=(const EventPair&) = delete;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    cudaError_t create() {
        cudaError_t e = cudaEventCreate(&a);
        return e == cudaSuccess ? cudaEventCreate(&b) : e;
    }
};

#define RCP_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return rcp::cuda_fail(e_, #call); \
    } while (0)

}  // namespace rcp
