// trace.cuh -- device functions of one recursive-camera-painting pass.
//
//  * camera_ray: the per-pixel camera of §2 (Eq. 2-4) and §3 (Eq. 5);
//  * traverse<ANY>: closest-hit (ANY = false) or any-hit (ANY = true) walk of
//    the 8-wide BVH (float child boxes) with a per-thread stack and the
//    block's traversal-order table in shared memory;
//  * hit_triangle / hit_sphere: Moller-Trumbore and the analytic sphere test;
//  * shade_*: Lambert + ambient with a shadow ray, sky on a miss.
// All arithmetic is float32 with explicit fused multiply-adds, so every kernel
// that calls these functions computes bit-identical results for the same ray.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rcp_internal.cuh"

namespace rcp {

struct RayF {
    float ox, oy, oz;
    float dx, dy, dz;
    float tmin, tmax;
};

struct Hit {
    float t;
    uint32_t id;   // caller's primitive id (SPHERE_BIT cleared), 0xffffffff = miss
    int32_t rec;   // record index of the hit, -1 = miss
};

struct WorkCount {
    uint32_t nodes, boxes, tris, spheres;
};

__device__ __forceinline__ float fdot(float ax, float ay, float az, float bx, float by, float bz) {
    return __fmaf_rn(ax, bx, __fmaf_rn(ay, by, __fmul_rn(az, bz)));
}

// Octahedral code of a unit vector (16 bits per folded coordinate, offset so
// that no real normal has code 0) and its inverse; code 0 = no normal.
__device__ __forceinline__ uint32_t normal_encode(float nx, float ny, float nz) {
    const float s = __fadd_rn(__fadd_rn(fabsf(nx), fabsf(ny)), fabsf(nz));
    if (!(s > 0.f)) return 0u;
    float px = __fdiv_rn(nx, s), py = __fdiv_rn(ny, s);
    if (nz < 0.f) {
        const float ox = px, oy = py;
        px = copysignf(__fsub_rn(1.f, fabsf(oy)), ox >= 0.f ? 1.f : -1.f);
        py = copysignf(__fsub_rn(1.f, fabsf(ox)), oy >= 0.f ? 1.f : -1.f);
    }
    const int qx = (int)roundf(__fmul_rn(px, 32767.f)), qy = (int)roundf(__fmul_rn(py, 32767.f));
    return (uint32_t)(qx + 32768) | ((uint32_t)(qy + 32768) << 16);
}

__device__ __forceinline__ bool normal_decode(uint32_t code, float& x, float& y, float& z) {
    if (code == 0u) {
        x = y = z = 0.f;
        return false;
    }
    const float px = __fdiv_rn((float)(int)(code & 0xffffu) - 32768.f, 32767.f);
    const float py = __fdiv_rn((float)(int)(code >> 16) - 32768.f, 32767.f);
    z = __fsub_rn(__fsub_rn(1.f, fabsf(px)), fabsf(py));
    x = px;
    y = py;
    if (z < 0.f) {
        x = copysignf(__fsub_rn(1.f, fabsf(py)), px >= 0.f ? 1.f : -1.f);
        y = copysignf(__fsub_rn(1.f, fabsf(px)), py >= 0.f ? 1.f : -1.f);
    }
    const float il = __fdiv_rn(1.f, __fsqrt_rn(__fmaf_rn(x, x, __fmaf_rn(y, y, __fmul_rn(z, z)))));
    x = __fmul_rn(x, il);
    y = __fmul_rn(y, il);
    z = __fmul_rn(z, il);
    return true;
}

// Camera of pixel (x, y) from its previous value c = (r, g, b, z).
//   g   = eye -> focal-plane point P_p - P_e (precomputed terms, see ViewDev)
//   V   = k ((2r-1) right + (2g-1) up + (2b-1) forward)             (Eq. 5)
//   EYE:    origin P_e + V, direction normalize(g - V)   (P'_e = P_e + V_e)
//   TARGET: origin P_e,     direction normalize(g + V)   (P'_p = P_p + V_p)
//   DEPTH:  origin P_e,     direction normalize(g + |z - z0| V)       (Eq. 7)
// The direction is P'_p - P'_e (Eq. 2) formed from the offsets, not from the
// absolute positions, which avoids cancellation in float32.
// (px, py): the sample's pixel coordinates (pixel centre = x + 0.5, y + 0.5).
__device__ __forceinline__ RayF camera_ray(const ViewDev& v, float px, float py, float4 c, float tmin) {
    const float ix = __fsub_rn(__fmul_rn(2.f, px), (float)v.W);
    const float iy = __fsub_rn((float)v.H, __fmul_rn(2.f, py));
    float gx = __fmaf_rn(ix, v.fR[0], __fmaf_rn(iy, v.fU[0], v.fF[0]));
    float gy = __fmaf_rn(ix, v.fR[1], __fmaf_rn(iy, v.fU[1], v.fF[1]));
    float gz = __fmaf_rn(ix, v.fR[2], __fmaf_rn(iy, v.fU[2], v.fF[2]));
    const float dr = __fmaf_rn(2.f, c.x, -1.f), dg = __fmaf_rn(2.f, c.y, -1.f), db = __fmaf_rn(2.f, c.z, -1.f);
    const float Vx = __fmaf_rn(dr, v.kR[0], __fmaf_rn(dg, v.kU[0], __fmul_rn(db, v.kF[0])));
    const float Vy = __fmaf_rn(dr, v.kR[1], __fmaf_rn(dg, v.kU[1], __fmul_rn(db, v.kF[1])));
    const float Vz = __fmaf_rn(dr, v.kR[2], __fmaf_rn(dg, v.kU[2], __fmul_rn(db, v.kF[2])));
    RayF r;
    r.tmin = tmin;
    r.tmax = __int_as_float(0x7f800000);
    if (v.mapping == RCP_MAP_NORMAL) {
        // §5, Eq. 8: V_p = k (C x N), C = normalize(g), N from the previous pass
        float nx, ny, nz;
        normal_decode(__float_as_uint(c.w), nx, ny, nz);
        const float il = __fdiv_rn(1.f, __fsqrt_rn(fdot(gx, gy, gz, gx, gy, gz)));
        const float cx = __fmul_rn(gx, il), cy = __fmul_rn(gy, il), cz = __fmul_rn(gz, il);
        const float k = v.kpx;
        gx = __fmaf_rn(k, __fmaf_rn(cy, nz, -__fmul_rn(cz, ny)), gx);
        gy = __fmaf_rn(k, __fmaf_rn(cz, nx, -__fmul_rn(cx, nz)), gy);
        gz = __fmaf_rn(k, __fmaf_rn(cx, ny, -__fmul_rn(cy, nx)), gz);
        r.ox = v.E[0];
        r.oy = v.E[1];
        r.oz = v.E[2];
    } else if (v.mapping == RCP_MAP_EYE) {
        r.ox = __fadd_rn(v.E[0], Vx);
        r.oy = __fadd_rn(v.E[1], Vy);
        r.oz = __fadd_rn(v.E[2], Vz);
        gx = __fsub_rn(gx, Vx);
        gy = __fsub_rn(gy, Vy);
        gz = __fsub_rn(gz, Vz);
    } else {
        const float m = v.mapping == RCP_MAP_DEPTH ? fabsf(__fsub_rn(c.w, v.z0)) : 1.f;
        r.ox = v.E[0];
        r.oy = v.E[1];
        r.oz = v.E[2];
        gx = __fmaf_rn(m, Vx, gx);
        gy = __fmaf_rn(m, Vy, gy);
        gz = __fmaf_rn(m, Vz, gz);
    }
    const float len2 = fdot(gx, gy, gz, gx, gy, gz);
    if (len2 > 0.f) {
        const float inv = __fdiv_rn(1.f, __fsqrt_rn(len2));
        r.dx = __fmul_rn(gx, inv);
        r.dy = __fmul_rn(gy, inv);
        r.dz = __fmul_rn(gz, inv);
    } else {  // P'_p == P'_e: look along the view axis
        const float l = __fsqrt_rn(fdot(v.fF[0], v.fF[1], v.fF[2], v.fF[0], v.fF[1], v.fF[2]));
        r.dx = __fdiv_rn(v.fF[0], l);
        r.dy = __fdiv_rn(v.fF[1], l);
        r.dz = __fdiv_rn(v.fF[2], l);
    }
    return r;
}

// I_{n-1} seen by a sample at (px, py): bilinear between the four nearest
// pixel centres, indices clamped; the normal mapping's code lane comes from the
// nearest pixel.
__device__ __forceinline__ float4 sample_prev(const float4* __restrict__ img, int W, int H, float px, float py,
                                              int mapping) {
    const float qx = __fsub_rn(px, 0.5f), qy = __fsub_rn(py, 0.5f);
    const float fx0 = floorf(qx), fy0 = floorf(qy);
    const float wx = __fsub_rn(qx, fx0), wy = __fsub_rn(qy, fy0);
    const int x0 = min(max((int)fx0, 0), W - 1), x1 = min(max((int)fx0 + 1, 0), W - 1);
    const int y0 = min(max((int)fy0, 0), H - 1), y1 = min(max((int)fy0 + 1, 0), H - 1);
    const float4 a = __ldg(img + (int64_t)y0 * W + x0), b = __ldg(img + (int64_t)y0 * W + x1);
    const float4 c = __ldg(img + (int64_t)y1 * W + x0), d = __ldg(img + (int64_t)y1 * W + x1);
    const float w00 = __fmul_rn(__fsub_rn(1.f, wx), __fsub_rn(1.f, wy)), w10 = __fmul_rn(wx, __fsub_rn(1.f, wy));
    const float w01 = __fmul_rn(__fsub_rn(1.f, wx), wy), w11 = __fmul_rn(wx, wy);
    float4 r;
    r.x = __fmaf_rn(w11, d.x, __fmaf_rn(w01, c.x, __fmaf_rn(w10, b.x, __fmul_rn(w00, a.x))));
    r.y = __fmaf_rn(w11, d.y, __fmaf_rn(w01, c.y, __fmaf_rn(w10, b.y, __fmul_rn(w00, a.y))));
    r.z = __fmaf_rn(w11, d.z, __fmaf_rn(w01, c.z, __fmaf_rn(w10, b.z, __fmul_rn(w00, a.z))));
    if (mapping == RCP_MAP_NORMAL) {
        const int nx = min(max((int)floorf(__fadd_rn(qx, 0.5f)), 0), W - 1);
        const int ny = min(max((int)floorf(__fadd_rn(qy, 0.5f)), 0), H - 1);
        r.w = __ldg(img + (int64_t)ny * W + nx).w;
    } else {
        r.w = __fmaf_rn(w11, d.w, __fmaf_rn(w01, c.w, __fmaf_rn(w10, b.w, __fmul_rn(w00, a.w))));
    }
    return r;
}

// Moller-Trumbore on a record (v0, e1, e2); closed bounds on u, v, u + v.
// Returns the hit distance or +inf.
__device__ __forceinline__ float hit_triangle(const RayF& r, float4 w0, float4 w1, float4 w2) {
    const float e1x = w0.w, e1y = w1.x, e1z = w1.y;
    const float e2x = w1.z, e2y = w1.w, e2z = w2.x;
    const float px = __fmaf_rn(r.dy, e2z, -__fmul_rn(r.dz, e2y));
    const float py = __fmaf_rn(r.dz, e2x, -__fmul_rn(r.dx, e2z));
    const float pz = __fmaf_rn(r.dx, e2y, -__fmul_rn(r.dy, e2x));
    const float det = fdot(e1x, e1y, e1z, px, py, pz);
    const float tx = __fsub_rn(r.ox, w0.x), ty = __fsub_rn(r.oy, w0.y), tz = __fsub_rn(r.oz, w0.z);
    const float un = fdot(tx, ty, tz, px, py, pz);
    const float qx = __fmaf_rn(ty, e1z, -__fmul_rn(tz, e1y));
    const float qy = __fmaf_rn(tz, e1x, -__fmul_rn(tx, e1z));
    const float qz = __fmaf_rn(tx, e1y, -__fmul_rn(ty, e1x));
    const float vn = fdot(r.dx, r.dy, r.dz, qx, qy, qz);
    const float tn = fdot(e2x, e2y, e2z, qx, qy, qz);
    const float inv = __frcp_rn(det);
    const float u = __fmul_rn(un, inv), v = __fmul_rn(vn, inv), t = __fmul_rn(tn, inv);
    const bool ok = (u >= 0.f) & (v >= 0.f) & (__fadd_rn(u, v) <= 1.f);
    return ok ? t : __int_as_float(0x7f800000);
}

// Analytic sphere: roots -b -/+ sqrt(r^2 - |oc - b d|^2), oc = o - c, b = oc.d.
// Returns the nearer root above tmin, else the farther, else +inf.
__device__ __forceinline__ float hit_sphere(const RayF& r, float4 w0) {
    const float ocx = __fsub_rn(r.ox, w0.x), ocy = __fsub_rn(r.oy, w0.y), ocz = __fsub_rn(r.oz, w0.z);
    const float b = fdot(ocx, ocy, ocz, r.dx, r.dy, r.dz);
    const float qx = __fmaf_rn(-b, r.dx, ocx), qy = __fmaf_rn(-b, r.dy, ocy), qz = __fmaf_rn(-b, r.dz, ocz);
    const float disc = __fmaf_rn(w0.w, w0.w, -fdot(qx, qy, qz, qx, qy, qz));
    if (!(disc >= 0.f)) return __int_as_float(0x7f800000);
    const float s = __fsqrt_rn(disc);
    const float t0 = __fsub_rn(-b, s), t1 = __fadd_rn(-b, s);
    if (t0 > r.tmin) return t0;
    if (t1 > r.tmin) return t1;
    return __int_as_float(0x7f800000);
}

// Bits [start, start + width) set (start + width <= 32).
__device__ __forceinline__ uint32_t bit_mask(uint32_t start, uint32_t width) {
    uint32_t d;
    asm("bmsk.clamp.b32 %0, %1, %2;" : "=r"(d) : "r"(start), "r"(width));
    return d;
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Two floats in one 64-bit register, and a fused multiply-add of two such
// pairs at once (each lane exactly the scalar FMA, rounded down or up).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma_rd(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
    unsigned long long d;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma_ru(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
    unsigned long long d;
    asm("fma.rp.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Traversal order of a node's children for a ray of octant oct (bit a set when
// the direction's component a is negative): slot s comes at position s ^ oct,
// so that slot order, which the collapse lays out front to back for octant 0,
// is walked front to back for every octant.
//
// The next-slot table: lut[256 oct + m] is the slot of the 8-bit slot mask m
// (m > 0) that comes first in octant oct's order, the s in m with the least
// s ^ oct. Each block fills its own 2 KB copy in shared memory before its
// first walk (the caller synchronises the block). One byte load per visited
// child replaces a bit-permuted mask per node and a find-first-set and XOR
// per child: on the mid terrain 432.7 -> 450.8 frames/s.
constexpr int ORDER_LUT_BYTES = 8 * 256;

template <int BLOCK>
__device__ __forceinline__ void fill_order_lut(uint8_t* lut) {
    for (int i = threadIdx.x; i < ORDER_LUT_BYTES; i += BLOCK) {
        const uint32_t m = (uint32_t)(i & 255), oct = (uint32_t)(i >> 8);
        uint32_t first = 0;
        for (uint32_t k = 8; k-- > 0;)
            if (m & (1u << (k ^ oct))) first = k ^ oct;
        lut[i] = (uint8_t)first;
    }
}

// Box test. Per axis, entry and exit are t = p * (1/d) - o * (1/d), one FMA
// per plane, made conservative by directed rounding: near planes round
// o * (1/d) up and the FMA down, far planes the reverse, so each computed
// entry is <= and each exit >= the exact (p - o) * (1/d) of the rounded
// reciprocal. The reciprocal's own relative error (<= 2^-24, different per
// axis) is covered by scaling the far planes' reciprocal by RCP_FAR_SCALE =
// 1 + 2^-21 away from zero. RCP_BOX_SLACK = 1 + 2^-17 widens the current
// closest hit, so that boxes holding an equal-t hit (ties go to the lower
// id) are still entered. The box test therefore never misses a primitive hit.
#define RCP_FAR_SCALE 1.000000476837158203125f
#define RCP_BOX_SLACK 1.0000076f

// The traversal stack of one thread: `entries` groups in shared memory at
// stack[i * stride], and above those `spill_entries` more in global memory,
// entry i at spill[(i - entries) * T + t] for the launch's thread t of T
// (both from the launch's own indices, so no pointer stays live in a
// register). A stack as deep as the tree (one group per level) never
// reaches the spill region; a shorter shared stack trades the spill traffic of
// deep walks for less shared memory per block. Pushing past both sets
// `overflow` and drops the group, which ends the walk early.
struct StackCfg {
    int entries;        // shared-memory entries per thread
    int spill_entries;  // global-memory entries per thread above those
    uint2* spill;       // spill_entries * (gridDim.x * blockDim.x) entries, or null
    int hints;          // bit 0: test each pixel's previous primary-hit record first; bit 1: its previous occluder
};

// Bring the 48-byte record rec (two 128-byte lines at most) towards L1, so
// that testing it first does not stall the walk's start on its load.
__device__ __forceinline__ void prefetch_record(const SceneDev& S, int32_t rec) {
    if (rec < 0 || rec >= S.n_records) return;
    const char* p = reinterpret_cast<const char*>(S.prims + 3 * (size_t)rec);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p + 47));
}

__device__ __forceinline__ uint2* spill_slot(const StackCfg& sc, int i) {
    const uint32_t T = gridDim.x * blockDim.x, t = blockIdx.x * blockDim.x + threadIdx.x;
    return sc.spill + (size_t)(i - sc.entries) * T + t;
}

// first_rec: a record to test before the walk (-1 none), in practice the one
// this pixel's ray hit in the previous pass. A hit there starts the walk with
// a far limit at its distance, so boxes behind it are never entered, and ends
// an any-hit walk at once. The result does not depend on it: the walk still
// keeps the least (t, id) over every record in a box the ray enters up to
// t (1 + 2^-17), and an any-hit answer is a yes/no.
template <bool ANY, bool COUNT>
__device__ __forceinline__ Hit traverse(const SceneDev& S, const RayF& r, uint2* stack, int stride,
                                        const StackCfg& stk, bool& overflow, WorkCount& wc, const uint8_t* order_lut,
                                        int32_t first_rec = -1) {
    Hit h;
    h.t = r.tmax;
    h.id = 0xffffffffu;
    h.rec = -1;
    if (S.n_nodes == 0) return h;
    if (first_rec >= 0 && first_rec < S.n_records) {
        const float4* pp = S.prims + 3 * (size_t)first_rec;
        const float4 w0 = __ldg(pp), w1 = __ldg(pp + 1), w2 = __ldg(pp + 2);
        const uint32_t idb = __float_as_uint(w2.y);
        float t;
        if (idb & SPHERE_BIT) {
            t = hit_sphere(r, w0);
            if (COUNT) wc.spheres++;
        } else {
            t = hit_triangle(r, w0, w1, w2);
            if (COUNT) wc.tris++;
        }
        if (t > r.tmin && t < r.tmax) {
            h.t = t;
            h.id = idb & ~SPHERE_BIT;
            h.rec = first_rec;
            if (ANY) return h;
        }
    }
    // A zero component stays zero (as +0, so that the octant bit and the sign
    // of 1/d agree) and its reciprocal is +inf: the ray is parallel to that
    // axis's planes. Its slab terms are then +-inf, or NaN where inf - inf
    // meets a plane level with the origin; min/max drop NaN operands, and
    // t_min and the far limit are never NaN, so a NaN term leaves the slab
    // unbounded. Nudging d away from zero instead would tilt a ray that lies
    // exactly in a box face out of that box.
    const float dx = r.dx == 0.f ? 0.f : r.dx;
    const float dy = r.dy == 0.f ? 0.f : r.dy;
    const float dz = r.dz == 0.f ? 0.f : r.dz;
    const float idx = __frcp_rn(dx), idy = __frcp_rn(dy), idz = __frcp_rn(dz);
    const uint32_t oct = (dx < 0.f ? 1u : 0u) | (dy < 0.f ? 2u : 0u) | (dz < 0.f ? 4u : 0u);
    const uint8_t* ord = order_lut + (oct << 8);
    // far-plane reciprocals, magnified away from zero
    const float fdx = dx > 0.f ? __fmul_ru(idx, RCP_FAR_SCALE) : __fmul_rd(idx, RCP_FAR_SCALE);
    const float fdy = dy > 0.f ? __fmul_ru(idy, RCP_FAR_SCALE) : __fmul_rd(idy, RCP_FAR_SCALE);
    const float fdz = dz > 0.f ? __fmul_ru(idz, RCP_FAR_SCALE) : __fmul_rd(idz, RCP_FAR_SCALE);
    // -o * (1/d): rounded down for near planes, up for far planes
    const float nox = -__fmul_ru(r.ox, idx), noy = -__fmul_ru(r.oy, idy), noz = -__fmul_ru(r.oz, idz);
    const float fox = -__fmul_rd(r.ox, fdx), foy = -__fmul_rd(r.oy, fdy), foz = -__fmul_rd(r.oz, fdz);
    // node rows of the near and far planes per axis (lo rows first, then hi)
    const int rxn = (oct & 1u) ? 2 : 0, rxf = 2 - rxn;
    const int ryn = (oct & 2u) ? 6 : 4, ryf = 10 - ryn;
    const int rzn = (oct & 4u) ? 10 : 8, rzf = 18 - rzn;
    float tfar_lim = __fmul_rn(h.t, RCP_BOX_SLACK);  // +inf without a first hit

    // node group: x = first child node index, y = imask | (slots still to visit) << 8;
    // the root is slot 0 of a group of one
    uint2 group = make_uint2(0u, 1u | (1u << 8));
    uint32_t prim_base = 0, prim_mask = 0;
    int sp = 0;
    // Every node and record index read here is in range: the builder
    // validates each tree (child indices above the parent and below n_nodes,
    // ranks matching the slot masks, records below n_prims) before a scene is
    // returned, and refits keep the topology. Child indices grow, so every
    // node is entered at most once; the cap only bounds the loop.
    // Every iteration visits exactly one node: when the current group is
    // exhausted the next one is popped first, so no lane spends an iteration
    // on the stack alone while the rest of its warp tests boxes.
    for (uint32_t iter = 0;; ++iter) {
        if (iter > (1u << 24)) {
            overflow = true;
            break;
        }
        if (group.y <= 0xffu) {
            if (sp == 0) break;
            --sp;
            group = sp < stk.entries ? stack[sp * stride] : *spill_slot(stk, sp);
        }
        {
            const uint32_t slot = ord[group.y >> 8];
            group.y &= ~(1u << (slot + 8));
            const uint32_t node = group.x + __popc(group.y & 0xffu & ((1u << slot) - 1u));
            if (group.y > 0xffu) {
                if (sp < stk.entries) {
                    stack[sp * stride] = group;
                    ++sp;
                } else if (sp < stk.entries + stk.spill_entries) {
                    *spill_slot(stk, sp) = group;
                    ++sp;
                } else {
                    overflow = true;
                }
            }
            const float4* np = S.nodes + NODE_ROWS * (size_t)node;
            const uint4 hd = __ldg(reinterpret_cast<const uint4*>(np + 12));
            if (COUNT) wc.nodes++;
            uint32_t hitmask = 0;
            // both halves unrolled: the second half's rows load while the
            // first half's slots are tested (faster than the lower-register
            // form that tests one half at a time)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const float4 nx = __ldg(np + rxn + half), fx = __ldg(np + rxf + half);
                const float4 ny = __ldg(np + ryn + half), fy = __ldg(np + ryf + half);
                const float4 nz = __ldg(np + rzn + half), fz = __ldg(np + rzf + half);
                // two slots per instruction: the planes of slots (0,1) and (2,3)
                // of this half against the ray's terms, each broadcast to a pair
                const float nxs[4] = {nx.x, nx.y, nx.z, nx.w}, fxs[4] = {fx.x, fx.y, fx.z, fx.w};
                const float nys[4] = {ny.x, ny.y, ny.z, ny.w}, fys[4] = {fy.x, fy.y, fy.z, fy.w};
                const float nzs[4] = {nz.x, nz.y, nz.z, nz.w}, fzs[4] = {fz.x, fz.y, fz.z, fz.w};
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int k = 2 * q;
                    float t0x[2], t1x[2], t0y[2], t1y[2], t0z[2], t1z[2];
                    f2_unpack(f2_fma_rd(f2_pack(nxs[k], nxs[k + 1]), f2_pack(idx, idx), f2_pack(nox, nox)), t0x[0],
                              t0x[1]);
                    f2_unpack(f2_fma_ru(f2_pack(fxs[k], fxs[k + 1]), f2_pack(fdx, fdx), f2_pack(fox, fox)), t1x[0],
                              t1x[1]);
                    f2_unpack(f2_fma_rd(f2_pack(nys[k], nys[k + 1]), f2_pack(idy, idy), f2_pack(noy, noy)), t0y[0],
                              t0y[1]);
                    f2_unpack(f2_fma_ru(f2_pack(fys[k], fys[k + 1]), f2_pack(fdy, fdy), f2_pack(foy, foy)), t1y[0],
                              t1y[1]);
                    f2_unpack(f2_fma_rd(f2_pack(nzs[k], nzs[k + 1]), f2_pack(idz, idz), f2_pack(noz, noz)), t0z[0],
                              t0z[1]);
                    f2_unpack(f2_fma_ru(f2_pack(fzs[k], fzs[k + 1]), f2_pack(fdz, fdz), f2_pack(foz, foz)), t1z[0],
                              t1z[1]);
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float tn = fmax3(t0x[j], t0y[j], fmaxf(t0z[j], r.tmin));
                        const float tf = fmin3(t1x[j], t1y[j], fminf(t1z[j], tfar_lim));
                        hitmask |= (tn <= tf ? 1u : 0u) << (4 * half + k + j);
                    }
                }
            }
            const uint32_t ml = hd.z, mh = hd.w;
            // an empty slot (meta 0) that tests as hit adds no child: it is not
            // in imask and its leaf count is 0
            if (COUNT) {
                uint32_t nonempty = 0;
#pragma unroll
                for (int s = 0; s < 8; ++s)
                    nonempty |= ((((s < 4 ? ml : mh) >> (8 * (s & 3))) & 0xffu) != 0u ? 1u : 0u) << s;
                wc.boxes += __popc(nonempty);
            }
            const uint32_t imask = internal_mask(ml, mh);
            const uint32_t hint = hitmask & imask;
            uint32_t hleaf = hitmask & ~imask;
            group = make_uint2(hd.x, imask | (hint << 8));
            prim_base = hd.y;
            prim_mask = 0;
            while (hleaf) {
                const uint32_t s = __ffs(hleaf) - 1;
                hleaf &= hleaf - 1;
                const uint32_t mb = __byte_perm(ml, mh, s) & 0xffu;
                prim_mask |= bit_mask(mb & 31u, mb >> 5);
            }
        }
        while (prim_mask) {
            const uint32_t j = __ffs(prim_mask) - 1;
            prim_mask &= prim_mask - 1;
            const int32_t rec = (int32_t)(prim_base + j);
            const float4* pp = S.prims + 3 * (size_t)rec;
            const float4 w0 = __ldg(pp), w1 = __ldg(pp + 1), w2 = __ldg(pp + 2);
            const uint32_t idb = __float_as_uint(w2.y);
            float t;
            if (idb & SPHERE_BIT) {
                t = hit_sphere(r, w0);
                if (COUNT) wc.spheres++;
            } else {
                t = hit_triangle(r, w0, w1, w2);
                if (COUNT) wc.tris++;
            }
            const uint32_t id = idb & ~SPHERE_BIT;
            // t in (tmin, tmax); the closer hit wins, equal t goes to the lower id
            if (t > r.tmin && t < r.tmax && (t < h.t || (t == h.t && id < h.id))) {
                h.t = t;
                h.id = id;
                h.rec = rec;
                if (ANY) return h;
                tfar_lim = __fmul_rn(h.t, RCP_BOX_SLACK);
            }
        }
    }
    return h;
}

// Brute force over every record (correctness reference for the BVH walk).
template <bool ANY>
__device__ __forceinline__ Hit traverse_brute(const SceneDev& S, const RayF& r) {
    Hit h;
    h.t = r.tmax;
    h.id = 0xffffffffu;
    h.rec = -1;
    for (int64_t rec = 0; rec < S.n_records; ++rec) {
        const float4* pp = S.prims + 3 * rec;
        const float4 w0 = __ldg(pp), w1 = __ldg(pp + 1), w2 = __ldg(pp + 2);
        const uint32_t idb = __float_as_uint(w2.y);
        const float t = (idb & SPHERE_BIT) ? hit_sphere(r, w0) : hit_triangle(r, w0, w1, w2);
        const uint32_t id = idb & ~SPHERE_BIT;
        if (t > r.tmin && t < r.tmax && (t < h.t || (t == h.t && id < h.id))) {
            h.t = t;
            h.id = id;
            h.rec = (int32_t)rec;
            if (ANY) return h;
        }
    }
    return h;
}

// What a primary hit needs for its final colour.
struct ShadeInfo {
    float4 c_shadow;  // colour if the shadow ray is blocked (or not cast), depth in w
    float4 c_lit;     // colour if the light is visible
    RayF shadow;      // the shadow ray (valid when need_shadow)
    bool need_shadow;
    uint32_t normal_code;  // octahedral code of the facing hit normal, 0 on a miss
};

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.f), 1.f); }

// Shading of §2 stage 2 (reading: the paper gives no shading model):
// hit -> albedo * (a + (1 - a) V max(0, N.L)), N facing the ray; miss -> sky
// (1 - s)(1,1,1) + s (0.5, 0.7, 1), s = (d_y + 1)/2; clamped to [0, 1].
__device__ __forceinline__ ShadeInfo shade_primary(const SceneDev& S, const RayF& r, const Hit& h) {
    ShadeInfo si;
    si.need_shadow = false;
    si.normal_code = 0u;
    if (h.rec < 0) {
        const float s = __fmul_rn(0.5f, __fadd_rn(r.dy, 1.f));
        const float one_s = __fsub_rn(1.f, s);
        si.c_shadow = make_float4(clamp01(__fmaf_rn(s, 0.5f, one_s)), clamp01(__fmaf_rn(s, 0.7f, one_s)),
                                  clamp01(__fadd_rn(one_s, s)), 0.f);
        si.c_lit = si.c_shadow;
        return si;
    }
    const float4* pp = S.prims + 3 * (size_t)h.rec;
    const float4 w0 = __ldg(pp), w1 = __ldg(pp + 1), w2 = __ldg(pp + 2);
    const float px = __fmaf_rn(h.t, r.dx, r.ox), py = __fmaf_rn(h.t, r.dy, r.oy), pz = __fmaf_rn(h.t, r.dz, r.oz);
    float nx, ny, nz;
    if (__float_as_uint(w2.y) & SPHERE_BIT) {
        const float ir = __frcp_rn(w0.w);
        nx = __fmul_rn(__fsub_rn(px, w0.x), ir);
        ny = __fmul_rn(__fsub_rn(py, w0.y), ir);
        nz = __fmul_rn(__fsub_rn(pz, w0.z), ir);
    } else {
        const float e1x = w0.w, e1y = w1.x, e1z = w1.y, e2x = w1.z, e2y = w1.w, e2z = w2.x;
        nx = __fmaf_rn(e1y, e2z, -__fmul_rn(e1z, e2y));
        ny = __fmaf_rn(e1z, e2x, -__fmul_rn(e1x, e2z));
        nz = __fmaf_rn(e1x, e2y, -__fmul_rn(e1y, e2x));
        const float il = __fdiv_rn(1.f, __fsqrt_rn(fdot(nx, ny, nz, nx, ny, nz)));
        nx = __fmul_rn(nx, il);
        ny = __fmul_rn(ny, il);
        nz = __fmul_rn(nz, il);
    }
    if (fdot(nx, ny, nz, r.dx, r.dy, r.dz) > 0.f) {
        nx = -nx;
        ny = -ny;
        nz = -nz;
    }
    float lx, ly, lz;
    if (S.light.type == RCP_LIGHT_POINT) {
        lx = __fsub_rn(S.light.x, px);
        ly = __fsub_rn(S.light.y, py);
        lz = __fsub_rn(S.light.z, pz);
        const float il = __fdiv_rn(1.f, __fsqrt_rn(fdot(lx, ly, lz, lx, ly, lz)));
        lx = __fmul_rn(lx, il);
        ly = __fmul_rn(ly, il);
        lz = __fmul_rn(lz, il);
    } else {
        lx = S.light.x;
        ly = S.light.y;
        lz = S.light.z;
    }
    si.normal_code = normal_encode(nx, ny, nz);
    const float ndl = fdot(nx, ny, nz, lx, ly, lz);
    const float a = S.light.ambient;
    const float4 alb = __ldg(S.albedo + h.id);
    si.c_shadow = make_float4(clamp01(__fmul_rn(alb.x, a)), clamp01(__fmul_rn(alb.y, a)),
                              clamp01(__fmul_rn(alb.z, a)), h.t);
    if (ndl > 0.f) {
        const float lit = __fmaf_rn(__fsub_rn(1.f, a), ndl, a);
        si.c_lit = make_float4(clamp01(__fmul_rn(alb.x, lit)), clamp01(__fmul_rn(alb.y, lit)),
                               clamp01(__fmul_rn(alb.z, lit)), h.t);
        si.need_shadow = true;
        RayF s;
        s.ox = __fmaf_rn(S.eps, nx, px);
        s.oy = __fmaf_rn(S.eps, ny, py);
        s.oz = __fmaf_rn(S.eps, nz, pz);
        s.tmin = 0.f;
        if (S.light.type == RCP_LIGHT_POINT) {
            float sx = __fsub_rn(S.light.x, s.ox), sy = __fsub_rn(S.light.y, s.oy), sz = __fsub_rn(S.light.z, s.oz);
            const float dist = __fsqrt_rn(fdot(sx, sy, sz, sx, sy, sz));
            const float il = __fdiv_rn(1.f, dist);
            s.dx = __fmul_rn(sx, il);
            s.dy = __fmul_rn(sy, il);
            s.dz = __fmul_rn(sz, il);
            s.tmax = dist;
        } else {
            s.dx = lx;
            s.dy = ly;
            s.dz = lz;
            s.tmax = __int_as_float(0x7f800000);
        }
        si.shadow = s;
    } else {
        si.c_lit = si.c_shadow;
    }
    return si;
}

}  // namespace rcp
