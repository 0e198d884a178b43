// trace.cu -- the pass kernels: per-pixel camera, primary + shadow trace, shade.
//
// Work is split into 8x4-pixel tiles (one warp each, 32 rays). A persistent
// grid of blocks claims tiles from a global counter, a warp at a time, across
// every view of the pass, so views of uneven size share one launch (§2: every
// (u,v) of every image gets its own camera in the same pass).
#include <cuda_runtime.h>
#include <stdint.h>

#include "scene.h"
#include "trace.cuh"

namespace rcp {

namespace {

__device__ __forceinline__ int find_view_by_chunk(const ViewDev* __restrict__ views, int n, int64_t chunk) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].chunk_begin <= chunk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_view_by_pix(const ViewDev* __restrict__ views, int n, int64_t pix) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].pix_begin <= pix) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Camera kernel: one thread per pixel, coalesced float4 reads of I_{n-1} and
// float4 writes of the ray (origin, t_min) + (direction, t_max).
__global__ void __launch_bounds__(256) k_camera(const ViewDev* __restrict__ views, int n_views, int64_t total_pix,
                                                float tmin, float4* __restrict__ rays) {
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_pix;
         gp += (int64_t)gridDim.x * blockDim.x) {
        const ViewDev& v = views[find_view_by_pix(views, n_views, gp)];
        const int64_t p = gp - v.pix_begin;
        const int x = (int)(p % v.W), y = (int)(p / v.W);
        const float4 c = v.in ? __ldg(v.in + p) : make_float4(0.5f, 0.5f, 0.5f, 0.f);
        const RayF r = camera_ray(v, (float)x + 0.5f, (float)y + 0.5f, c, tmin);
        rays[2 * gp] = make_float4(r.ox, r.oy, r.oz, r.tmin);
        rays[2 * gp + 1] = make_float4(r.dx, r.dy, r.dz, r.tmax);
    }
}

// Trace, shadow and shade one camera ray; returns the pixel value: RGB and
// the hit's z-depth t (d . F) along the view axis F (0 on a miss).
// hint: the records of this pixel's previous primary hit and shadow occluder
// (-1 none), tested first; updated to this ray's.
template <bool COUNT>
__device__ __forceinline__ float4 trace_shade(const SceneDev& S, const RayF& r, const float* Fw, uint2* stack,
                                              int stride, const StackCfg& stk, bool& overflow, WorkCount& wc,
                                              uint32_t& n_shadow, uint32_t& code, int32_t& prim,
                                              const uint8_t* order_lut, int2& hint) {
    const Hit h = traverse<false, COUNT>(S, r, stack, stride, stk, overflow, wc, order_lut, hint.x);
    prefetch_record(S, hint.y);  // the previous occluder, ahead of the shadow walk
    const ShadeInfo si = shade_primary(S, r, h);
    float4 out = si.c_shadow;
    hint.x = h.rec;
    if (si.need_shadow) {
        ++n_shadow;
        const Hit hs =
            traverse<true, COUNT>(S, si.shadow, stack, stride, stk, overflow, wc, order_lut, hint.y);
        if (hs.rec < 0) out = si.c_lit;
        hint.y = hs.rec;
    }
    out.w = h.rec < 0 ? 0.f : __fmul_rn(h.t, fdot(r.dx, r.dy, r.dz, Fw[0], Fw[1], Fw[2]));
    code = si.normal_code;
    prim = h.rec < 0 ? -1 : (int32_t)h.id;
    return out;
}

// A warp counts n finished tiles of view v (with a done counter) at once:
// every lane's writes for them made visible first, at system scope (the RGB
// may go straight to host memory, which the host reads once the flag is set),
// then one atomic; the warp that counts the view's last tiles sets its
// host-visible done flag. Counting when the warp moves to another view (or
// ends) keeps the fences, which wait for the writes in flight, to one per run
// of tiles.
__device__ __forceinline__ void tiles_done(const ViewDev* v, int n, int lane) {
    if (!v || n == 0) return;
    __threadfence_system();
    __syncwarp();
    if (lane == 0 && atomicSub(v->done_count, n) == n) {
        __threadfence_system();
        *(volatile int*)v->done_flag = 1;
    }
}

// MULTI: every view names its own scene (views of several scenes in one
// launch); otherwise all views render the launch's scene S0.
// CHAIN: one launch runs v.passes passes of each view v (v.in its first
// input, v.out its last output); a warp carries each pixel of its tile from
// pass to pass, its colour and hints in registers, and writes only the last
// pass's outputs. At one sample per pixel with a camera that reads only the
// pixel's own previous value (every mapping but the image-space one), this
// computes exactly what one launch per pass computes.
template <int BLOCK, bool FUSED, bool COUNT, bool MS, bool MULTI, bool CHAIN>
__global__ void __launch_bounds__(BLOCK, CHAIN ? 640 / BLOCK : 0)  // CHAIN: 20 warps per SM, as the one-pass kernel
    k_trace(SceneDev S0, const ViewDev* __restrict__ views, int n_views,
                                                 int64_t total_chunks, int chunk_tiles,
                                                 const float4* __restrict__ rays, unsigned* work, StackCfg stk,
                                                 unsigned long long* ray_counts, unsigned long long* counters) {
    static_assert(!CHAIN || (FUSED && !MS), "a chained launch makes its rays itself, one per pixel");
    extern __shared__ uint2 s_stack[];
    __shared__ uint8_t s_order[ORDER_LUT_BYTES];
    __shared__ SceneDev s_scene[MULTI ? BLOCK / 32 : 1];  // MULTI: the scene of each warp's current tile
    // per warp: the view (with a done counter) whose tiles it finished last,
    // and how many of them it has not yet counted. Done counters come with
    // the server's launches, which name each view's scene (MULTI).
    constexpr bool SIGNAL = MULTI;
    __shared__ const ViewDev* s_done_v[BLOCK / 32];
    __shared__ int s_done_n[BLOCK / 32];
    fill_order_lut<BLOCK>(s_order);
    if ((threadIdx.x & 31) == 0) {
        s_done_v[threadIdx.x >> 5] = nullptr;
        s_done_n[threadIdx.x >> 5] = 0;
    }
    __syncthreads();
    uint2* stack = s_stack + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool overflow = false;
    WorkCount wc{0, 0, 0, 0};
    uint32_t n_primary = 0, n_shadow = 0;
    static_assert(sizeof(SceneDev) % 4 == 0 && sizeof(SceneDev) <= 128, "SceneDev is copied by one warp");
    for (;;) {
        unsigned c0 = 0;
        if (lane == 0) c0 = atomicAdd(work, (unsigned)chunk_tiles);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if ((int64_t)c0 >= total_chunks) break;
        for (int sub = 0; sub < chunk_tiles; ++sub) {
            const int64_t chunk = (int64_t)c0 + sub;
            if (chunk >= total_chunks) break;
            const ViewDev& v = views[find_view_by_chunk(views, n_views, chunk)];
            if (MULTI) {  // the warp's tile is one view: copy its scene to the warp's slot
                __syncwarp();
                const uint32_t* src = reinterpret_cast<const uint32_t*>(v.scene);
                uint32_t* dst = reinterpret_cast<uint32_t*>(&s_scene[threadIdx.x >> 5]);
                for (int i = lane; i < (int)(sizeof(SceneDev) / 4); i += 32) dst[i] = __ldg(src + i);
                __syncwarp();
            }
            const SceneDev& S = MULTI ? s_scene[threadIdx.x >> 5] : S0;
            do {  // the tile's pixel of this lane ("continue" leaves the block)
                const int64_t tile = chunk - v.chunk_begin;
                const int tx = (int)(tile % v.tiles_x), ty = (int)(tile / v.tiles_x);
                const int x = tx * 8 + (lane & 7), y = ty * 4 + (lane >> 3);
                if (x >= v.W || y >= v.H) continue;
                const int64_t p = (int64_t)y * v.W + x;
                if (MS) {
                    // jittered samples (§2): each reads I_{n-1} at its own position
                    const int ns = v.spp > 0 ? v.spp : 1;
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                    uint32_t code0 = 0;
                    int32_t prim0 = -1;
                    int2 hint = v.hint && stk.hints ? v.hint[p] : make_int2(-1, -1);
                    if (!(stk.hints & 1)) hint.x = -1;
                    if (!(stk.hints & 2)) hint.y = -1;
                    prefetch_record(S, hint.x);
                    for (int s = 0; s < ns; ++s) {
                        const float jx = v.spp > 0 ? v.jit[2 * s] : 0.5f, jy = v.spp > 0 ? v.jit[2 * s + 1] : 0.5f;
                        const float px = __fadd_rn((float)x, jx), py = __fadd_rn((float)y, jy);
                        const float4 c = v.in ? sample_prev(v.in, v.W, v.H, px, py, v.mapping)
                                              : make_float4(0.5f, 0.5f, 0.5f, 0.f);
                        const RayF r = camera_ray(v, px, py, c, S.tmin);
                        uint32_t code;
                        int32_t prim;
                        const float4 o = trace_shade<COUNT>(S, r, v.Fw, stack, BLOCK, stk, overflow, wc,
                                                            n_shadow, code, prim, s_order, hint);
                        ++n_primary;
                        acc.x = __fadd_rn(acc.x, o.x);
                        acc.y = __fadd_rn(acc.y, o.y);
                        acc.z = __fadd_rn(acc.z, o.z);
                        acc.w = __fadd_rn(acc.w, o.w);
                        if (s == 0) {
                            code0 = code;
                            prim0 = prim;
                        }
                    }
                    const float fn = (float)ns;
                    float4 out = make_float4(__fdiv_rn(acc.x, fn), __fdiv_rn(acc.y, fn), __fdiv_rn(acc.z, fn),
                                             __fdiv_rn(acc.w, fn));
                    if (v.mapping == RCP_MAP_NORMAL) out.w = __uint_as_float(code0);
                    v.out[p] = out;
                    if (v.hint) v.hint[p] = hint;
                    if (v.prim) v.prim[p] = prim0;
                    if (v.rgb) {
                        v.rgb[3 * p] = out.x;
                        v.rgb[3 * p + 1] = out.y;
                        v.rgb[3 * p + 2] = out.z;
                    }
                    if (overflow) {  // this view's image is incomplete
                        *(volatile int*)v.status = 1;
                        overflow = false;
                    }
                    continue;
                }
                int2 hint = v.hint && stk.hints ? v.hint[p] : make_int2(-1, -1);
                if (!(stk.hints & 1)) hint.x = -1;
                if (!(stk.hints & 2)) hint.y = -1;
                // CHAIN: passes 1..K, the camera reading this pixel's own previous value
                float4 out = FUSED && v.in ? __ldg(v.in + p) : make_float4(0.5f, 0.5f, 0.5f, 0.f);
                uint32_t code;
                int32_t prim;
                for (int n = 0; n < (CHAIN ? v.passes : 1); ++n) {
                    prefetch_record(S, hint.x);  // its lines arrive while the camera ray is made
                    RayF r;
                    if (FUSED) {
                        r = camera_ray(v, (float)x + 0.5f, (float)y + 0.5f, out, S.tmin);
                    } else {
                        const float4 a = __ldg(rays + 2 * (v.pix_begin + p));
                        const float4 b = __ldg(rays + 2 * (v.pix_begin + p) + 1);
                        r.ox = a.x;
                        r.oy = a.y;
                        r.oz = a.z;
                        r.tmin = a.w;
                        r.dx = b.x;
                        r.dy = b.y;
                        r.dz = b.z;
                        r.tmax = b.w;
                    }
                    out = trace_shade<COUNT>(S, r, v.Fw, stack, BLOCK, stk, overflow, wc, n_shadow, code, prim,
                                             s_order, hint);
                    ++n_primary;
                    if (v.mapping == RCP_MAP_NORMAL) out.w = __uint_as_float(code);
                }
                v.out[p] = out;
                if (v.hint) v.hint[p] = hint;
                if (v.prim) v.prim[p] = prim;
                if (v.rgb) {
                    v.rgb[3 * p] = out.x;
                    v.rgb[3 * p + 1] = out.y;
                    v.rgb[3 * p + 2] = out.z;
                }
                if (overflow) {  // this view's image is incomplete
                    *(volatile int*)v.status = 1;
                    overflow = false;
                }
            } while (0);
            if (SIGNAL && v.done_count) {  // counted when the warp leaves the view
                const int w = threadIdx.x >> 5;
                __syncwarp();
                if (s_done_v[w] != &v) {
                    tiles_done(s_done_v[w], s_done_n[w], lane);
                    __syncwarp();
                    if (lane == 0) {
                        s_done_v[w] = &v;
                        s_done_n[w] = 0;
                    }
                }
                __syncwarp();
                if (lane == 0) ++s_done_n[w];
            }
        }
    }
    if (SIGNAL) {
        __syncwarp();
        tiles_done(s_done_v[threadIdx.x >> 5], s_done_n[threadIdx.x >> 5], lane);
    }
    {
        const unsigned np = __reduce_add_sync(0xffffffffu, n_primary);
        const unsigned ns = __reduce_add_sync(0xffffffffu, n_shadow);
        if (lane == 0 && ray_counts) {
            atomicAdd(&ray_counts[0], (unsigned long long)np);
            atomicAdd(&ray_counts[1], (unsigned long long)ns);
        }
    }
    if (COUNT) {
        atomicAdd(&counters[0], (unsigned long long)(n_primary + n_shadow));
        atomicAdd(&counters[1], (unsigned long long)n_primary);
        atomicAdd(&counters[2], (unsigned long long)n_shadow);
        atomicAdd(&counters[3], (unsigned long long)wc.nodes);
        atomicAdd(&counters[4], (unsigned long long)wc.boxes);
        atomicAdd(&counters[5], (unsigned long long)wc.tris);
        atomicAdd(&counters[6], (unsigned long long)wc.spheres);
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_debug_trace(SceneDev S, int64_t n, const float4* __restrict__ ot,
                                                       const float4* __restrict__ dt, int any, int brute,
                                                       float* __restrict__ t_out, int32_t* __restrict__ prim_out,
                                                       int stack_entries, int* status) {
    extern __shared__ uint2 s_stack[];
    __shared__ uint8_t s_order[ORDER_LUT_BYTES];
    fill_order_lut<BLOCK>(s_order);
    __syncthreads();
    uint2* stack = s_stack + threadIdx.x;
    const StackCfg stk{stack_entries, 0, nullptr, 0};
    bool overflow = false;
    WorkCount wc{0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = ot[i], b = dt[i];
        RayF r{a.x, a.y, a.z, b.x, b.y, b.z, a.w, b.w};
        Hit h;
        if (brute) h = any ? traverse_brute<true>(S, r) : traverse_brute<false>(S, r);
        else h = any ? traverse<true, false>(S, r, stack, BLOCK, stk, overflow, wc, s_order)
                     : traverse<false, false>(S, r, stack, BLOCK, stk, overflow, wc, s_order);
        if (any) {
            prim_out[i] = h.rec >= 0 ? 1 : 0;
            t_out[i] = 0.f;
        } else {
            prim_out[i] = h.rec < 0 ? -1 : (int32_t)h.id;
            t_out[i] = h.rec < 0 ? __int_as_float(0x7f800000) : h.t;
        }
    }
    if (overflow) atomicExch(&status[0], 1);
}

__global__ void k_pack_rgb(const float4* __restrict__ img, float* __restrict__ rgb, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 c = img[i];
        rgb[3 * i] = c.x;
        rgb[3 * i + 1] = c.y;
        rgb[3 * i + 2] = c.z;
    }
}

// ---------------------------------------------------------------- image space (§6, §6.1)

// Reflect a pixel index into [0, n) about the image edges, the edge pixel not
// repeated (-1 -> 0, n -> n-1), as often as needed.
__device__ __forceinline__ int64_t mirror_px(int64_t i, int64_t n) {
    if (i >= 0 && i < n) return i;
    if (n <= 1) return 0;
    const int64_t period = 2 * n;
    int64_t m = i % period;
    if (m < 0) m += period;
    return m < n ? m : period - 1 - m;
}

// I_n(x, y) = base at the nearest pixel to (x + kpx (2r - 1), y - kpx (2g - 1)),
// (r, g) = I_{n-1}(x, y); float32 without fused multiply-add decides the pixel.
// Returns the index of that pixel of `base`.
__device__ __forceinline__ int64_t gather_source(float4 c, int W, int H, int x, int y, float kpx) {
    const float dr = __fsub_rn(__fmul_rn(2.f, c.x), 1.f);
    const float dg = __fsub_rn(__fmul_rn(2.f, c.y), 1.f);
    const float sx = __fadd_rn((float)x, __fmul_rn(kpx, dr));
    const float sy = __fsub_rn((float)y, __fmul_rn(kpx, dg));
    const int64_t ix = mirror_px((int64_t)floorf(__fadd_rn(sx, 0.5f)), W);
    const int64_t iy = mirror_px((int64_t)floorf(__fadd_rn(sy, 0.5f)), H);
    return iy * W + ix;
}

// One view's gather over pixels [first, P) in steps of `step`, the view's
// fields in registers and 32-bit pixel indices (P <= 8192 * 8192). One pixel
// per thread per iteration measured best at 4K (64.5 us a pass, against 68, 70
// and 78 us with 2, 4 and 8 pixels per thread): the HBM traffic is fed by
// resident warps, not by more loads per thread.
__device__ __forceinline__ void gather_view(const float4* __restrict__ base, const float4* __restrict__ prev,
                                            float4* __restrict__ out, int W, int H, float kpx, int P, int first,
                                            int step) {
    for (int p = first; p < P; p += step) out[p] = __ldg(base + gather_source(__ldg(prev + p), W, H, p % W, p / W, kpx));
}

// One view: gather_view with the view's fields in registers. Several views:
// one pixel per thread per iteration over the global pixel range, each pixel
// finding its view, so that small views share the grid.
__global__ void __launch_bounds__(256) k_imagespace(const ViewDev* __restrict__ views, int n_views, int64_t total_pix) {
    if (n_views == 1) {
        const ViewDev& v = views[0];
        gather_view(v.base, v.in, v.out, v.W, v.H, v.kpx, v.W * v.H, blockIdx.x * blockDim.x + threadIdx.x,
                    gridDim.x * blockDim.x);
        return;
    }
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_pix;
         gp += (int64_t)gridDim.x * blockDim.x) {
        const ViewDev& v = views[find_view_by_pix(views, n_views, gp)];
        const int p = (int)(gp - v.pix_begin);
        const float4 c = __ldg(v.in + p);
        v.out[p] = __ldg(v.base + gather_source(c, v.W, v.H, p % v.W, p / v.W, v.kpx));
    }
}

__global__ void __launch_bounds__(256) k_imagespace_single(const float4* __restrict__ base,
                                                          const float4* __restrict__ prev, float4* __restrict__ out,
                                                          int W, int H, float kpx) {
    gather_view(base, prev, out, W, H, kpx, W * H, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Resident blocks per SM of a 256-thread gather kernel (cached per kernel).
template <class K>
int gather_blocks_per_sm(K kern) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

template <int BLOCK, bool FUSED, bool COUNT, bool MS, bool MULTI, bool CHAIN>
rcp_status launch_trace_t(const SceneDev& S, const LaunchCfg& cfg, const ViewDev* d_views, int n_views,
                          int64_t total_chunks, const float4* rays, unsigned* d_work, unsigned long long* d_rays,
                          unsigned long long* d_counters, cudaStream_t st) {
    auto kern = k_trace<BLOCK, FUSED, COUNT, MS, MULTI, CHAIN>;
    const size_t smem = sizeof(uint2) * (size_t)cfg.stack * BLOCK;
    if (smem > 48 * 1024) RCP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = cfg.blocks_per_sm;
    if (per_sm <= 0) {
        RCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem));
        if (per_sm <= 0) per_sm = 1;
    }
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t need = (total_chunks * 32 + BLOCK - 1) / BLOCK;
    if (grid > need) grid = need > 0 ? need : 1;
    StackCfg stk{cfg.stack, cfg.spill ? cfg.spill_entries : 0, cfg.spill, cfg.hints};
    if (stk.spill_entries > 0 && grid * BLOCK * (int64_t)stk.spill_entries > cfg.spill_cap) {
        set_error("traversal spill region too small for the launch");
        return RCP_ERR_STATE;
    }
    kern<<<(int)grid, BLOCK, smem, st>>>(S, d_views, n_views, total_chunks, cfg.chunk / 32, rays, d_work, stk, d_rays,
                                         d_counters);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

template <bool FUSED, bool COUNT, bool MS, bool MULTI, bool CHAIN = false>
rcp_status launch_trace_b(const SceneDev& S, const LaunchCfg& cfg, const ViewDev* d_views, int n_views,
                          int64_t total_chunks, const float4* rays, unsigned* d_work, unsigned long long* d_rays,
                          unsigned long long* d_counters, cudaStream_t st) {
    switch (cfg.block) {
        case 64:
            return launch_trace_t<64, FUSED, COUNT, MS, MULTI, CHAIN>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                      d_work, d_rays, d_counters, st);
        case 256:
            return launch_trace_t<256, FUSED, COUNT, MS, MULTI, CHAIN>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                       d_work, d_rays, d_counters, st);
        default:
            return launch_trace_t<128, FUSED, COUNT, MS, MULTI, CHAIN>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                       d_work, d_rays, d_counters, st);
    }
}

}  // namespace

rcp_status launch_pass(const SceneDev& S, const LaunchCfg& cfg, const ViewDev* d_views, int n_views,
                       int64_t total_pix, int64_t total_chunks, float4* rays, unsigned* d_work,
                       unsigned long long* d_rays, unsigned long long* d_counters, cudaStream_t st) {
    if (cfg.multi) {  // views of several scenes: fused camera, no counters
        return cfg.ms ? launch_trace_b<true, false, true, true>(S, cfg, d_views, n_views, total_chunks, rays, d_work,
                                                                d_rays, nullptr, st)
                      : launch_trace_b<true, false, false, true>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                 d_work, d_rays, nullptr, st);
    }
    if (!cfg.fused && !cfg.ms) {
        int64_t g = (total_pix + 255) / 256;
        if (g > (int64_t)sm_count() * 16) g = (int64_t)sm_count() * 16;
        if (g < 1) g = 1;
        k_camera<<<(int)g, 256, 0, st>>>(d_views, n_views, total_pix, S.tmin, rays);
        RCP_CUDA(cudaGetLastError());
    }
    if (cfg.ms) {  // jittered samples: camera inside the trace kernel
        return cfg.count ? launch_trace_b<true, true, true, false>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                   d_work, d_rays, d_counters, st)
                         : launch_trace_b<true, false, true, false>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                    d_work, d_rays, d_counters, st);
    }
    if (cfg.count)
        return cfg.fused ? launch_trace_b<true, true, false, false>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                    d_work, d_rays, d_counters, st)
                         : launch_trace_b<false, true, false, false>(S, cfg, d_views, n_views, total_chunks, rays,
                                                                     d_work, d_rays, d_counters, st);
    return cfg.fused ? launch_trace_b<true, false, false, false>(S, cfg, d_views, n_views, total_chunks, rays, d_work,
                                                                 d_rays, d_counters, st)
                     : launch_trace_b<false, false, false, false>(S, cfg, d_views, n_views, total_chunks, rays, d_work,
                                                                  d_rays, d_counters, st);
}

rcp_status launch_chain(const SceneDev& S, const LaunchCfg& cfg, const ViewDev* d_views, int n_views,
                        int64_t total_chunks, unsigned* d_work, unsigned long long* d_rays,
                        unsigned long long* d_counters, cudaStream_t st) {
    if (cfg.ms) {
        set_error("launch_chain: a chained launch is single-sample");
        return RCP_ERR_STATE;
    }
    if (cfg.multi)  // views of several scenes: no counters
        return launch_trace_b<true, false, false, true, true>(S, cfg, d_views, n_views, total_chunks, nullptr, d_work,
                                                              d_rays, nullptr, st);
    return cfg.count ? launch_trace_b<true, true, false, false, true>(S, cfg, d_views, n_views, total_chunks,
                                                                      nullptr, d_work, d_rays, d_counters, st)
                     : launch_trace_b<true, false, false, false, true>(S, cfg, d_views, n_views, total_chunks,
                                                                       nullptr, d_work, d_rays, d_counters, st);
}

rcp_status launch_debug_trace(const SceneDev& S, int64_t n, const float* orig_tmin, const float* dir_tmax, int any,
                              int brute, float* t_out, int32_t* prim_out, int stack_entries, int* d_status,
                              cudaStream_t st) {
    if (n <= 0) return RCP_OK;
    const size_t smem = sizeof(uint2) * MAX_STACK * 128;
    RCP_CUDA(cudaFuncSetAttribute(k_debug_trace<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t g = (n + 127) / 128;
    if (g > (int64_t)sm_count() * 8) g = (int64_t)sm_count() * 8;
    k_debug_trace<128><<<(int)g, 128, smem, st>>>(S, n, (const float4*)orig_tmin, (const float4*)dir_tmax, any, brute,
                                                 t_out, prim_out, stack_entries, d_status);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

rcp_status launch_imagespace(const ViewDev* d_views, int n_views, int64_t total_pix, cudaStream_t st) {
    static const int per_sm = gather_blocks_per_sm(k_imagespace);
    int64_t g = (total_pix + 255) / 256;
    if (g > (int64_t)sm_count() * per_sm) g = (int64_t)sm_count() * per_sm;
    if (g < 1) g = 1;
    k_imagespace<<<(int)g, 256, 0, st>>>(d_views, n_views, total_pix);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

rcp_status launch_imagespace_single(const float4* base, const float4* prev, float4* out, int W, int H, float kpx,
                                    cudaStream_t st) {
    static const int per_sm = gather_blocks_per_sm(k_imagespace_single);
    const int64_t P = (int64_t)W * H;
    int64_t g = (P + 255) / 256;
    if (g > (int64_t)sm_count() * per_sm) g = (int64_t)sm_count() * per_sm;
    if (g < 1) g = 1;
    k_imagespace_single<<<(int)g, 256, 0, st>>>(base, prev, out, W, H, kpx);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

rcp_status launch_pack_rgb(const float4* img, float* rgb, int64_t n, cudaStream_t st) {
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)sm_count() * 16) g = (int64_t)sm_count() * 16;
    if (g < 1) g = 1;
    k_pack_rgb<<<(int)g, 256, 0, st>>>(img, rgb, n);
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

}  // namespace rcp
