// rcp_internal.cuh -- shared device types of the renderer (not part of the ABI).
//
// Layout in device memory (all 16-byte aligned):
//  * WNode: one compressed 8-wide BVH node, 80 bytes = 5 x uint4.
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

// One 8-wide node. Child slot s (0..7) has a quantised box
//   lo = p + q_lo[s] * 2^e,  hi = p + q_hi[s] * 2^e   (per axis)
// and meta[s]: 0 = empty, 0x80 | rank = internal child (node child_base +
// rank, ranks counted in slot order), (count << 5) | offset = leaf of `count`
// (1..3) primitive records at prim_base + offset.
struct __align__(16) WNode {
    float px, py, pz;
    uint32_t e_imask;  // ex | ey << 8 | ez << 16 | imask << 24 (exponents biased by 127)
    uint32_t child_base;
    uint32_t prim_base;
    uint32_t meta_lo, meta_hi;  // meta[0..3], meta[4..7]
    uint32_t qlo_x[2], qlo_y[2], qlo_z[2];
    uint32_t qhi_x[2], qhi_y[2], qhi_z[2];
};
static_assert(sizeof(WNode) == 80, "WNode must be 80 bytes");

struct LightDev {
    int type;
    float x, y, z;
    float ambient;
};

// Device-resident scene: BVH, primitive records and shading data.
struct SceneDev {
    const uint4* nodes;    // n_nodes * 5
    const float4* prims;   // n_prims * 3
    const float4* albedo;  // n_prims
    int64_t n_prims;
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
    float E[3];
    float fF[3], fR[3], fU[3];
    float kR[3], kU[3], kF[3];
    int W, H;
    int mapping;
    float z0;
    float kpx;  // IMAGE: displacement in pixels; NORMAL: k in world units
    int pad0_;
    const float4* in;    // previous image, nullptr = I_0
    const float4* base;  // image-space passes: the frame's traced image
    float4* out;         // this pass's image
    int32_t* prim;     // nullable hit ids
    int64_t pix_begin;  // first global pixel index of this view
    int64_t chunk_begin;  // first work chunk (8x4 tile) of this view
    int tiles_x;
    int spp;              // samples per pixel, 0 = one at the centre
    float jit[2 * RCP_MAX_SPP];
};

// Host-side owner of a built scene.
struct Scene;

struct Counters {
    unsigned long long rays, primary, shadow, nodes, boxes, tris, spheres;
};

// thread-local error message
void set_error(const std::string& msg);
rcp_status cuda_fail(cudaError_t e, const char* what);

#define RCP_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return rcp::cuda_fail(e_, #call); \
    } while (0)

}  // namespace rcp
