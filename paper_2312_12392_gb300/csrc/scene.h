// scene.h -- host-side scene object and the render launch interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "rcp_internal.cuh"

namespace rcp {

// Cached resources of one launch shape: ping-pong images, ray buffer, view
// descriptors (device + pinned staging), work counters and the CUDA graph of
// the K-pass sequence.
struct RenderCtx {
    int n_views = 0;
    int K = 0;
    int64_t total_pix = 0;
    int64_t total_chunks = 0;
    float4* img[2] = {nullptr, nullptr};
    float4* rays = nullptr;
    ViewDev* d_views = nullptr;  // K * n_views
    ViewDev* h_views = nullptr;  // pinned staging
    unsigned* d_work = nullptr;  // one work counter per launch
    int* d_status = nullptr;     // [0] stack overflow
    unsigned long long* d_rays = nullptr;  // rays traced by the last render: primary, shadow
    float* d_rgb = nullptr;      // packed RGB for host output
    float4* io = nullptr;        // host-API input / final image
    float4* base_img = nullptr;  // image-space mapping: the traced pass-1 image
    bool image_mode = false;     // passes 2..K are image-space gathers
    bool chained = false;        // one launch runs all K passes (one descriptor per view)
    int32_t* io_prim = nullptr;  // host-API hit ids
    int2* hints = nullptr;       // per pixel: latest primary-hit and shadow-occluder records (-1 none)
    cudaEvent_t staged = nullptr;
    cudaEvent_t pass_ev[17] = {};  // timing events around every launch (recorded inside the graph)
    int launches = 0;              // launches of the latest enqueue: K, or 1 when the passes are chained
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
    cudaEvent_t done = nullptr;  // recorded after the context's latest launch
    uint64_t last_use = 0;
    int64_t bytes = 0;
    ~RenderCtx();
};

struct Scene {
    int64_t T = 0, S = 0;
    float* d_tri = nullptr;
    float* d_sph = nullptr;
    float4* d_albedo = nullptr;
    void* d_nodes = nullptr;  // WNode[n_nodes]
    float4* d_nbox = nullptr;  // 2 per node: union box of the node's children
    float4* d_prims = nullptr;  // 3 per leaf record (n_records)
    float4* d_refbox = nullptr;  // 2 per record: its exact clipped box in a split build (else null)
    uint32_t* d_part_uv = nullptr;  // split build: 9 per record, its part of its triangle as 16-bit (u, v) pairs
    uint32_t* d_rec_id = nullptr;   // split build: each record's primitive id (with the sphere flag)
    float2* d_rbox = nullptr;       // 3 per record: padded record boxes of the latest refit (from the first refit)
    int64_t n_records = 0;       // leaf records: T + S, more when triangles are split
    int split_max = 1;           // references per triangle at most (1: no splitting)
    int64_t n_nodes = 0;
    int depth = 0;
    int max_leaf = 0;
    int collapse = RCP_COLLAPSE_AREA;  // rcp_collapse policy of the build
    std::vector<int64_t> level_begin;
    float diam = 0.f;
    float build_ms = 0.f;
    LightDev light{};
    rcp_tuning tuning{128, 0, 32, 1, 0, 3, 1};
    std::mutex mu;
    std::map<std::string, std::unique_ptr<RenderCtx>> ctx;
    RenderCtx* last = nullptr;  // context of the most recent render
    uint64_t use_clock = 0;
    SceneDev* d_dev = nullptr;  // device copy of dev(), named by views of multi-scene launches
    uint2* d_spill = nullptr;   // global-memory traversal stack entries of a short shared stack
    int64_t spill_cap = 0;
    ~Scene();
    SceneDev dev() const;
    int64_t device_bytes() const;
};

rcp_status build_bvh(Scene& sc, cudaStream_t st);
rcp_status refit_bvh(Scene& sc, cudaStream_t st);
rcp_status validate_bvh(const Scene& sc, cudaStream_t st);
rcp_status debug_morton(const float* xyz, int64_t n, const float* lo, const float* hi, uint32_t* codes,
                        cudaStream_t st);

// Fill a view descriptor (camera terms in double, rounded once).
void make_view(ViewDev& v, const rcp_camera& cam, int W, int H, const rcp_params& p);

// Launch configuration of the pass kernels.
struct LaunchCfg {
    int block = 128;
    int blocks_per_sm = 0;
    int chunk = 32;
    bool fused = true;
    int stack = 32;  // shared-memory stack entries per thread
    int spill_entries = 0;  // global-memory stack entries per thread above those
    uint2* spill = nullptr;  // their region (spill_cap entries)
    int64_t spill_cap = 0;
    bool count = false;
    bool ms = false;  // jittered multi-sample kernel
    bool multi = false;  // each view names its scene (views of several scenes; the server's launches)
    int hints = 3;    // previous-hit hints: bit 0 primary, bit 1 shadow
    bool chain = false;  // all K passes in one launch where the render allows it
};

// One pass over n_views views whose descriptors are at d_views (device). A
// walk that overflows its stack sets its view's status word.
rcp_status launch_pass(const SceneDev& S, const LaunchCfg& cfg, const ViewDev* d_views, int n_views,
                       int64_t total_pix, int64_t total_chunks, float4* rays, unsigned* d_work,
                       unsigned long long* d_rays, unsigned long long* d_counters, cudaStream_t st);
// Several passes of n_views views in one launch: view v runs v.passes passes
// from v.in to v.out, each pixel's colour and hints kept in registers from
// pass to pass, only the last pass's outputs written. Single-sample, fused
// camera (cfg.fused is not read), and a mapping that reads only the pixel's
// own previous value; cfg.multi: the views name their scenes.
rcp_status launch_chain(const SceneDev& S, const LaunchCfg& cfg, const ViewDev* d_views, int n_views,
                        int64_t total_chunks, unsigned* d_work, unsigned long long* d_rays,
                        unsigned long long* d_counters, cudaStream_t st);
rcp_status launch_debug_trace(const SceneDev& S, int64_t n, const float* orig_tmin, const float* dir_tmax, int any,
                              int brute, float* t_out, int32_t* prim_out, int stack_entries, int* d_status,
                              cudaStream_t st);
rcp_status launch_pack_rgb(const float4* img, float* rgb, int64_t n, cudaStream_t st);

// Whether kernels on the current device read and write pageable host memory
// coherently (then a render's last pass can write the caller's RGB directly).
bool host_coherent();
// Whether a frame goes straight into host buffer [p, p + bytes) (the host
// output policy of rcp_set_host_output; records the buffer as written).
bool use_direct_output(const void* p, size_t bytes);
// Read and write back one byte in every page of [p, p + bytes).
void touch_pages(void* p, size_t bytes);
// Image-space pass over every view (views' base/in/out set).
rcp_status launch_imagespace(const ViewDev* d_views, int n_views, int64_t total_pix, cudaStream_t st);
rcp_status launch_imagespace_single(const float4* base, const float4* prev, float4* out, int W, int H, float kpx,
                                    cudaStream_t st);

}  // namespace rcp

// The opaque handle of the C ABI is the scene object itself.
struct rcp_scene : public rcp::Scene {};
