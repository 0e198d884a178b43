// serve.cu -- continuous-batching render server (rcp_server_* in rcp.h).
//
// Two host threads own the device work:
//  * the scheduler admits queued requests (FIFO) while a slot is free and the
//    request's device memory -- two rgbz images, per-pixel hit hints and a
//    status word (plus an RGB staging buffer where the device cannot write
//    host memory), allocated stream-ordered from the device's memory pool --
//    fits the budget. Each step then advances admitted requests by one or
//    more passes in ONE persistent launch: a single tile queue over the
//    step's views, whatever their scene, size or K (each view names its scene;
//    views are grouped by scene for cache locality). A request that advances
//    by several passes in a step runs them chained: each warp carries its
//    tile's pixels from pass to pass in registers. A step takes requests in
//    admission order: the oldest always (one pass at least), each as many of
//    its remaining passes as the step's pixel-pass budget still holds (at
//    most max_chain), the others while one pass of theirs fits; the rest wait,
//    with their images resident, for a later step. Old requests thus run as
//    soon as they would on their own and new small ones fill the rest of a
//    step: first come first served with backfill, like a token budget in LLM
//    continuous batching, rather than every request sharing every step, which
//    stretches the largest requests. Which requests finish at a step is known
//    when it is enqueued, so the scheduler never waits for the device except
//    to bound how far it runs ahead (STEPS_AHEAD steps);
//  * the copy-out thread waits for each finished request, reads its status
//    word (a walk that overflowed its stack fails the request), copies its RGB
//    image to the caller's buffer where needed, releases its memory and
//    records its latency, while the device already runs the next steps. A
//    request is finished when the last of its tiles in its final step is: the
//    warp that completes it sets the request's done word in page-locked host
//    memory, so a request does not wait for the other views of its launch
//    (views are queued oldest first). Its last pass writes its RGB into the
//    caller's buffer where the host output policy chooses direct writes
//    (rcp_set_host_output), else into a device staging buffer that the
//    copy-out thread copies.
// New requests join at the next step while others are mid-recursion, so short
// and long requests share every launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "scene.h"

namespace rcp {
namespace {

constexpr int STEPS_AHEAD = 3;  // steps enqueued before the oldest must finish
// pixel-passes per step: a 3840x2160 K=8 request (66.4M) runs to its end in one step
constexpr int64_t DEFAULT_STEP_PIXELS = 67000000;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct Request {
    int64_t ticket = 0;
    const rcp_scene* scene = nullptr;
    rcp_camera cam{};
    int W = 0, H = 0, K = 0;
    rcp_params p{};
    float* out_rgb = nullptr;
    int passes_done = 0;  // passes enqueued so far
    int step_passes = 0;  // passes of the step being enqueued (0: not in it)
    float4* img[2] = {nullptr, nullptr};
    float* rgb = nullptr;
    bool direct = false;     // the last pass writes out_rgb itself (else pack and copy)
    int2* hint = nullptr;    // per pixel: latest primary-hit and shadow-occluder records
    int status_slot = -1;     // the request's two words in the server's page-locked status array
    int64_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    rcp_status status = RCP_OK;
    bool done = false;
    cudaEvent_t ready = nullptr;  // the RGB image (packed, or in the caller's buffer) and status word are complete
};

// Launch resources of one step: the views of every in-flight request.
struct StepSlot {
    ViewDev* d_views = nullptr;
    ViewDev* h_views = nullptr;  // pinned staging
    int cap = 0;
    unsigned* d_work = nullptr;
    int* d_counts = nullptr;  // per view: its tiles still to finish (final steps of requests)
    int* h_counts = nullptr;  // pinned staging
    cudaEvent_t start = nullptr, done = nullptr;  // around the step's device work
    bool used = false;
};

}  // namespace rcp

using namespace rcp;

struct rcp_server {
    int64_t budget = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_copy;
    std::deque<Request*> queue;
    std::vector<Request*> inflight;
    std::deque<Request*> copyq;
    std::map<int64_t, std::unique_ptr<Request>> all;
    int64_t next_ticket = 1;
    bool stop = false, copy_stop = false;
    std::thread worker, copier;
    int64_t bytes_in_use = 0, bytes_peak = 0;
    int64_t submitted = 0, completed = 0, rejected = 0, steps = 0;
    double t_first = 0, t_last = 0;
    std::vector<double> latencies_ms;
    unsigned long long* d_rays = nullptr;  // running total: primary, shadow
    cudaStream_t st_main = nullptr, st_copy = nullptr;
    StepSlot slots[STEPS_AHEAD];
    int64_t step_no = 0;
    int device = 0;
    // page-locked, mapped: per admitted, unfinished request, [2 slot] its
    // overflow word (written by the device) and [2 slot + 1] its done word
    int* h_status = nullptr;
    int* d_hstatus = nullptr;  // the same array as the device addresses it
    std::vector<int> free_status;
    int64_t step_pixels = DEFAULT_STEP_PIXELS;  // pixel-passes per step (0: every admitted request every step)
    int max_chain = 16;  // passes one request may advance by in one step
    double busy_ms = 0;  // device time of completed steps

    void run();
    void copy_out();
    rcp_status enqueue_step(std::vector<Request*>& batch, StepSlot& slot);
    void finish(Request* q, rcp_status st, double t);
};

namespace {

// Device memory of a request: two rgbz images, the per-pixel hit hints, and
// the RGB staging buffer unless its last pass writes the caller's buffer
// directly.
int64_t request_bytes(int W, int H, bool direct) {
    const int64_t P = (int64_t)W * H;
    return P * (2 * 16 + 8 + (direct ? 0 : 12)) + 3 * 256;
}

rcp_status alloc_request(Request& r, bool direct, cudaStream_t st) {
    const int64_t P = (int64_t)r.W * r.H;
    RCP_CUDA(cudaMallocAsync((void**)&r.img[0], sizeof(float4) * P, st));
    RCP_CUDA(cudaMallocAsync((void**)&r.img[1], sizeof(float4) * P, st));
    RCP_CUDA(cudaMallocAsync((void**)&r.hint, sizeof(int2) * P, st));
    RCP_CUDA(cudaMemsetAsync(r.hint, 0xff, sizeof(int2) * P, st));  // -1: no earlier hit
    if (!direct) RCP_CUDA(cudaMallocAsync((void**)&r.rgb, sizeof(float) * 3 * P, st));
    if (!r.ready) RCP_CUDA(cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming));
    return RCP_OK;
}

void free_request(Request& r, cudaStream_t st) {
    for (auto*& p : r.img)
        if (p) {
            cudaFreeAsync(p, st);
            p = nullptr;
        }
    if (r.rgb) {
        cudaFreeAsync(r.rgb, st);
        r.rgb = nullptr;
    }
    if (r.hint) {
        cudaFreeAsync(r.hint, st);
        r.hint = nullptr;
    }
}

rcp_status ensure_slot(StepSlot& s, int n) {
    if (!s.d_work) {
        RCP_CUDA(cudaMalloc((void**)&s.d_work, sizeof(unsigned)));
        RCP_CUDA(cudaEventCreate(&s.start));
        RCP_CUDA(cudaEventCreate(&s.done));
    }
    if (s.cap < n) {
        if (s.d_views) cudaFree(s.d_views);
        if (s.h_views) cudaFreeHost(s.h_views);
        if (s.d_counts) cudaFree(s.d_counts);
        if (s.h_counts) cudaFreeHost(s.h_counts);
        s.d_views = nullptr;
        s.h_views = nullptr;
        s.d_counts = nullptr;
        s.h_counts = nullptr;
        s.cap = 0;
        const int cap = std::max(n, 16);
        RCP_CUDA(cudaMalloc((void**)&s.d_views, sizeof(ViewDev) * cap));
        RCP_CUDA(cudaMallocHost((void**)&s.h_views, sizeof(ViewDev) * cap));
        RCP_CUDA(cudaMalloc((void**)&s.d_counts, sizeof(int) * cap));
        RCP_CUDA(cudaMallocHost((void**)&s.h_counts, sizeof(int) * cap));
        s.cap = cap;
    }
    return RCP_OK;
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

// Enqueue the step's passes of every request in the batch (q->step_passes
// each) as one launch (the slot's resources are free: its previous step has
// completed). Several passes of a request run chained; a step with a
// multi-sample request runs one pass of each (its jittered samples read
// neighbouring pixels of the previous image).
rcp_status rcp_server::enqueue_step(std::vector<Request*>& batch, StepSlot& slot) {
    rcp_status r = ensure_slot(slot, (int)batch.size());
    if (r != RCP_OK) return r;
    // views grouped by scene (its tree stays in L2 while its views run),
    // scenes in order of their oldest request, admission order within a
    // scene: the tile queue runs them in that order, and each request is done
    // when its own tiles are
    std::vector<const rcp_scene*> order;
    for (Request* q : batch)
        if (std::find(order.begin(), order.end(), q->scene) == order.end()) order.push_back(q->scene);
    std::stable_sort(batch.begin(), batch.end(), [&](Request* a, Request* b) {
        return std::find(order.begin(), order.end(), a->scene) < std::find(order.begin(), order.end(), b->scene);
    });
    std::set<const rcp_scene*> scenes;
    int stack = 4;
    bool ms = false;
    for (Request* q : batch) {
        scenes.insert(q->scene);
        stack = std::max(stack, q->scene->depth);
        ms = ms || q->p.spp > 0;
    }
    LaunchCfg cfg;  // 128 threads, 32-pixel chunks, fused camera: no ray buffer per request
    cfg.stack = std::min((stack + 3) & ~3, MAX_STACK);  // one entry per level of the deepest tree
    cfg.ms = ms;
    cfg.multi = true;  // each view names its scene (and the kernels count each request's tiles)
    int64_t total_pix = 0, total_chunks = 0;
    for (size_t i = 0; i < batch.size(); ++i) {
        Request* q = batch[i];
        ViewDev v;
        make_view(v, q->cam, q->W, q->H, q->p);
        v.scene = q->scene->d_dev;
        v.status = d_hstatus + 2 * q->status_slot;
        const int last = q->passes_done + q->step_passes;  // passes done after this step
        v.in = q->passes_done == 0 ? nullptr : q->img[(q->passes_done - 1) & 1];
        v.out = q->img[(last - 1) & 1];
        v.passes = q->step_passes;
        v.hint = q->hint;
        const int64_t tiles = (int64_t)v.tiles_x * ((q->H + 3) / 4);
        slot.h_counts[i] = 0;
        if (last == q->K) {  // its final step: the last pass writes the RGB, its last tile the done word
            v.rgb = q->direct ? q->out_rgb : q->rgb;
            slot.h_counts[i] = (int)tiles;
            v.done_count = slot.d_counts + i;
            v.done_flag = d_hstatus + 2 * q->status_slot + 1;
        }
        v.pix_begin = total_pix;
        v.chunk_begin = total_chunks;
        total_pix += (int64_t)q->W * q->H;
        total_chunks += tiles;
        slot.h_views[i] = v;
    }
    RCP_CUDA(cudaEventRecord(slot.start, st_main));
    RCP_CUDA(cudaMemcpyAsync(slot.d_views, slot.h_views, sizeof(ViewDev) * batch.size(), cudaMemcpyHostToDevice,
                             st_main));
    RCP_CUDA(cudaMemcpyAsync(slot.d_counts, slot.h_counts, sizeof(int) * batch.size(), cudaMemcpyHostToDevice,
                             st_main));
    RCP_CUDA(cudaMemsetAsync(slot.d_work, 0, sizeof(unsigned), st_main));
    r = ms ? launch_pass((*scenes.begin())->dev(), cfg, slot.d_views, (int)batch.size(), total_pix, total_chunks,
                         nullptr, slot.d_work, d_rays, nullptr, st_main)
           : launch_chain((*scenes.begin())->dev(), cfg, slot.d_views, (int)batch.size(), total_chunks, slot.d_work,
                          d_rays, nullptr, st_main);
    if (r != RCP_OK) return r;
    for (Request* q : batch)  // after the step, whatever the done words say
        if (q->passes_done + q->step_passes == q->K) RCP_CUDA(cudaEventRecord(q->ready, st_main));
    RCP_CUDA(cudaEventRecord(slot.done, st_main));
    slot.used = true;
    return RCP_OK;
}

void rcp_server::finish(Request* q, rcp_status st, double t) {
    // called with mu held
    bytes_in_use -= q->bytes;
    if (q->status_slot >= 0) {
        free_status.push_back(q->status_slot);
        q->status_slot = -1;
    }
    q->t_done = t;
    if (q->status == RCP_OK) q->status = st;
    q->done = true;
    if (q->status == RCP_OK) {
        ++completed;
        latencies_ms.push_back(1000.0 * (q->t_done - q->t_submit));
        t_last = t;
    }
    cv_done.notify_all();
    cv_work.notify_all();
}

void rcp_server::copy_out() {
    cudaSetDevice(device);
    for (;;) {
        Request* q = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_copy.wait(lk, [&] { return copy_stop || !copyq.empty(); });
            if (copyq.empty()) return;
            q = copyq.front();
            copyq.pop_front();
        }
        rcp_status st = RCP_OK;
        if (q->status == RCP_OK) {
            // the done word (set by the request's last tile), or the end of
            // its step, whichever is seen first
            const volatile int* done = h_status + 2 * q->status_slot + 1;
            cudaError_t e = cudaSuccess;
            for (int spin = 0; !*done; ++spin) {
                e = cudaEventQuery(q->ready);
                if (e != cudaErrorNotReady) break;
                e = cudaSuccess;
                if (spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
            std::atomic_thread_fence(std::memory_order_acquire);  // the image and overflow word written before it
            if (e == cudaSuccess && ((volatile int*)h_status)[2 * q->status_slot]) {
                set_error("server: a traversal stack overflowed; the request's image is incomplete");
                st = RCP_ERR_STACK;
            }
            if (e == cudaSuccess && st == RCP_OK && !q->direct)
                e = cudaMemcpyAsync(q->out_rgb, q->rgb, sizeof(float) * 3 * (int64_t)q->W * q->H,
                                    cudaMemcpyDeviceToHost, st_copy);
            if (e == cudaSuccess && st == RCP_OK && !q->direct) e = cudaStreamSynchronize(st_copy);
            if (e != cudaSuccess) st = cuda_fail(e, "server copy-out");
        } else {
            // A failed request may have passes still queued (a step that failed
            // part-way): let the device drain before its images are freed and
            // the caller, whose buffer a last pass may write, is told.
            cudaDeviceSynchronize();
        }
        free_request(*q, st_copy);
        const double t = now_s();
        std::lock_guard<std::mutex> lk(mu);
        finish(q, st, t);
    }
}

void rcp_server::run() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<Request*> batch;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait_for(lk, std::chrono::milliseconds(20),
                             [&] { return stop || !queue.empty() || !inflight.empty(); });
            if (stop && inflight.empty()) {
                for (Request* q : queue) {
                    q->status = RCP_ERR_STATE;
                    q->done = true;
                }
                queue.clear();
                cv_done.notify_all();
                return;
            }
            // admission: FIFO while a slot is free and the memory fits
            while (!stop && !queue.empty() && (int)inflight.size() < max_slots && !free_status.empty()) {
                Request* q = queue.front();
                if (q->bytes > budget) {  // can never fit
                    queue.pop_front();
                    q->status = RCP_ERR_OOM;
                    q->done = true;
                    ++rejected;
                    cv_done.notify_all();
                    continue;
                }
                if (q->scene->depth > MAX_STACK) {
                    queue.pop_front();
                    q->status = RCP_ERR_STACK;
                    q->done = true;
                    cv_done.notify_all();
                    continue;
                }
                if (bytes_in_use + q->bytes > budget) break;
                queue.pop_front();
                bytes_in_use += q->bytes;
                bytes_peak = std::max(bytes_peak, bytes_in_use);
                q->t_admit = now_s();
                q->status_slot = free_status.back();
                free_status.pop_back();
                h_status[2 * q->status_slot] = 0;  // overflow
                h_status[2 * q->status_slot + 1] = 0;  // done
                inflight.push_back(q);
            }
            batch = inflight;
        }
        if (batch.empty()) {  // idle: account the device time of the last steps
            for (StepSlot& sl : slots)
                if (sl.used && cudaEventQuery(sl.done) == cudaSuccess) {
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, sl.start, sl.done) == cudaSuccess) {
                        std::lock_guard<std::mutex> lk(mu);
                        busy_ms += ms;
                    }
                    sl.used = false;
                }
            continue;
        }
        for (Request* q : batch)
            if (!q->img[0] && q->status == RCP_OK) {
                rcp_status r = alloc_request(*q, q->direct, st_main);
                if (r != RCP_OK) q->status = r;
            }
        // the step: admission order, the oldest always, each request as many
        // of its remaining passes as the step's pixel-pass budget holds (one
        // where a multi-sample request is admitted)
        bool any_ms = false;
        for (Request* q : batch) any_ms = any_ms || (q->status == RCP_OK && q->p.spp > 0);
        std::vector<Request*> ok;
        int64_t px = 0;
        for (Request* q : batch) {
            q->step_passes = 0;
            if (q->status != RCP_OK) continue;
            const int64_t qp = (int64_t)q->W * q->H;
            int m = std::min(q->K - q->passes_done, any_ms ? 1 : max_chain);
            if (step_pixels > 0) m = (int)std::min<int64_t>(m, (step_pixels - px) / qp);
            if (ok.empty()) m = std::max(m, 1);
            if (m <= 0) continue;
            ok.push_back(q);
            q->step_passes = m;
            px += m * qp;
        }
        StepSlot& slot = slots[step_no % STEPS_AHEAD];
        if (slot.used) {  // bound the run-ahead; frees the slot's staging
            cudaEventSynchronize(slot.done);
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, slot.start, slot.done) == cudaSuccess) {
                std::lock_guard<std::mutex> lk(mu);
                busy_ms += ms;
            }
            slot.used = false;
        }
        rcp_status r = ok.empty() ? RCP_OK : enqueue_step(ok, slot);
        ++step_no;
        std::lock_guard<std::mutex> lk(mu);
        ++steps;
        std::vector<Request*> still;
        for (Request* q : inflight) {
            if (r != RCP_OK && q->status == RCP_OK) q->status = r;
            if (q->status == RCP_OK) q->passes_done += q->step_passes;
            if (q->status != RCP_OK || q->passes_done >= q->K) {
                copyq.push_back(q);  // the copy-out thread waits for its image
                cv_copy.notify_one();
            } else {
                still.push_back(q);
            }
        }
        inflight.swap(still);
    }
}

extern "C" {

rcp_status rcp_server_create(int64_t budget, int max_slots, rcp_server** out) {
    if (!out || budget <= 0 || max_slots < 1 || max_slots > 4096) {
        set_error("rcp_server_create: budget > 0 and 1 <= max_slots <= 4096");
        return RCP_ERR_ARG;
    }
    auto s = std::make_unique<rcp_server>();
    s->budget = budget;
    s->max_slots = max_slots;
    RCP_CUDA(cudaGetDevice(&s->device));
    RCP_CUDA(cudaStreamCreateWithFlags(&s->st_main, cudaStreamNonBlocking));
    RCP_CUDA(cudaStreamCreateWithFlags(&s->st_copy, cudaStreamNonBlocking));
    RCP_CUDA(cudaMalloc((void**)&s->d_rays, sizeof(unsigned long long) * 2));
    RCP_CUDA(cudaMemset(s->d_rays, 0, sizeof(unsigned long long) * 2));
    // admitted, unfinished requests: at most max_slots in flight and as many
    // again waiting for copy-out (admission waits for a free word)
    const int n_status = 2 * max_slots + 16;
    RCP_CUDA(cudaHostAlloc((void**)&s->h_status, sizeof(int) * 2 * n_status, cudaHostAllocMapped));
    RCP_CUDA(cudaHostGetDevicePointer((void**)&s->d_hstatus, s->h_status, 0));
    for (int i = n_status - 1; i >= 0; --i) s->free_status.push_back(i);
    cudaMemPool_t pool = nullptr;
    RCP_CUDA(cudaDeviceGetDefaultMemPool(&pool, s->device));
    uint64_t thr = (uint64_t)budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    // Back the pool with memory now (up to 8 GB of the budget, within half of
    // what is free): growing it while requests are served maps memory inside
    // the driver, which holds up CUDA calls on other threads for milliseconds.
    size_t free_b = 0, total_b = 0;
    RCP_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t reserve = std::min<size_t>({(size_t)budget, (size_t)8 << 30, free_b / 2});
    if (reserve > 0) {
        void* p = nullptr;
        RCP_CUDA(cudaMallocAsync(&p, reserve, s->st_main));
        RCP_CUDA(cudaFreeAsync(p, s->st_main));
        RCP_CUDA(cudaStreamSynchronize(s->st_main));
    }
    rcp_server* raw = s.release();
    raw->worker = std::thread([raw] { raw->run(); });
    raw->copier = std::thread([raw] { raw->copy_out(); });
    *out = raw;
    return RCP_OK;
}

rcp_status rcp_server_submit(rcp_server* srv, const rcp_scene* scene, const rcp_camera* cam, int W, int H, int K,
                             const rcp_params* p, float* out_rgb, int64_t* ticket) {
    if (!srv || !scene || !cam || !p || !out_rgb || !ticket) {
        set_error("rcp_server_submit: NULL argument");
        return RCP_ERR_ARG;
    }
    if (W < 1 || H < 1 || W > 8192 || H > 8192 || K < 1 || K > 16 || !(p->k >= 0.f) || !(p->focal_dist > 0.f) ||
        p->mapping < RCP_MAP_EYE || p->mapping > RCP_MAP_NORMAL || p->mapping == RCP_MAP_IMAGE ||
        !(cam->fov_y_deg > 0.f) || p->spp > RCP_MAX_SPP ||
        !(cam->fov_y_deg < 180.f)) {
        set_error("rcp_server_submit: argument out of range");
        return RCP_ERR_ARG;
    }
    auto q = std::make_unique<Request>();
    q->scene = scene;
    q->cam = *cam;
    q->W = W;
    q->H = H;
    q->K = K;
    q->p = *p;
    q->out_rgb = out_rgb;
    q->direct = use_direct_output(out_rgb, sizeof(float) * 3 * (size_t)W * H);
    q->bytes = request_bytes(W, H, q->direct);
    if (q->direct) touch_pages(out_rgb, sizeof(float) * 3 * (size_t)W * H);  // mapped before the device writes
    q->t_submit = now_s();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) {
        set_error("rcp_server_submit: server is stopping");
        return RCP_ERR_STATE;
    }
    q->ticket = srv->next_ticket++;
    *ticket = q->ticket;
    if (srv->submitted == 0) srv->t_first = q->t_submit;
    ++srv->submitted;
    srv->queue.push_back(q.get());
    srv->all[q->ticket] = std::move(q);
    srv->cv_work.notify_one();
    return RCP_OK;
}

rcp_status rcp_server_set_step_pixels(rcp_server* srv, int64_t pixels) {
    if (!srv || pixels < 0) {
        set_error("rcp_server_set_step_pixels: NULL server or negative budget");
        return RCP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->step_pixels = pixels;
    return RCP_OK;
}

rcp_status rcp_server_set_max_chain(rcp_server* srv, int passes) {
    if (!srv || passes < 1 || passes > 16) {
        set_error("rcp_server_set_max_chain: NULL server or passes outside [1, 16]");
        return RCP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->max_chain = passes;
    return RCP_OK;
}

rcp_status rcp_server_poll(rcp_server* srv, int64_t ticket, int* done) {
    if (!srv || !done) {
        set_error("rcp_server_poll: NULL argument");
        return RCP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) {
        set_error("rcp_server_poll: unknown ticket");
        return RCP_ERR_ARG;
    }
    *done = it->second->done ? 1 : 0;
    return it->second->done ? it->second->status : RCP_OK;
}

rcp_status rcp_server_latency(rcp_server* srv, int64_t ticket, double* ms) {
    if (!srv || !ms) {
        set_error("rcp_server_latency: NULL argument");
        return RCP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) {
        set_error("rcp_server_latency: unknown ticket");
        return RCP_ERR_ARG;
    }
    if (!it->second->done) {
        set_error("rcp_server_latency: request not finished");
        return RCP_ERR_STATE;
    }
    *ms = 1000.0 * (it->second->t_done - it->second->t_submit);
    return RCP_OK;
}

rcp_status rcp_server_wait(rcp_server* srv, int64_t ticket, double timeout_s) {
    if (!srv) {
        set_error("rcp_server_wait: NULL server");
        return RCP_ERR_ARG;
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->all.find(ticket);
    if (it == srv->all.end()) {
        set_error("rcp_server_wait: unknown ticket");
        return RCP_ERR_ARG;
    }
    Request* q = it->second.get();
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return q->done; });
    if (!ok) {
        set_error("rcp_server_wait: timed out");
        return RCP_ERR_TIMEOUT;
    }
    if (q->status != RCP_OK) set_error("rcp_server_wait: request failed");
    return q->status;
}

rcp_status rcp_server_stats_get(rcp_server* srv, rcp_server_stats* out) {
    if (!srv || !out) {
        set_error("rcp_server_stats_get: NULL argument");
        return RCP_ERR_ARG;
    }
    unsigned long long h[2] = {0, 0};
    // the counters only grow; a read that races a running pass sees a lower bound
    RCP_CUDA(cudaMemcpy(h, srv->d_rays, sizeof(h), cudaMemcpyDeviceToHost));
    std::lock_guard<std::mutex> lk(srv->mu);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->rejected = srv->rejected;
    out->in_flight = (int64_t)srv->inflight.size() + (int64_t)srv->copyq.size();
    out->queued = (int64_t)srv->queue.size();
    out->steps = srv->steps;
    out->p50_ms = percentile(srv->latencies_ms, 0.50);
    out->p99_ms = percentile(srv->latencies_ms, 0.99);
    const double span = srv->t_last - srv->t_first;
    out->frames_per_s = span > 0 ? srv->completed / span : 0.0;
    out->mrays_per_s = span > 0 ? (double)(h[0] + h[1]) / span / 1e6 : 0.0;
    out->device_bytes_in_use = srv->bytes_in_use;
    out->device_bytes_peak = srv->bytes_peak;
    out->device_busy_ms = srv->busy_ms;
    return RCP_OK;
}

void rcp_server_destroy(rcp_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->copy_stop = true;
        srv->cv_copy.notify_all();
    }
    if (srv->copier.joinable()) srv->copier.join();
    cudaStreamSynchronize(srv->st_main);
    cudaStreamSynchronize(srv->st_copy);
    for (auto& sl : srv->slots) {
        if (sl.d_views) cudaFree(sl.d_views);
        if (sl.h_views) cudaFreeHost(sl.h_views);
        if (sl.d_counts) cudaFree(sl.d_counts);
        if (sl.h_counts) cudaFreeHost(sl.h_counts);
        if (sl.d_work) cudaFree(sl.d_work);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.start) cudaEventDestroy(sl.start);
    }
    if (srv->h_status) cudaFreeHost(srv->h_status);
    for (auto& kv : srv->all)
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    if (srv->d_rays) cudaFree(srv->d_rays);
    if (srv->st_main) cudaStreamDestroy(srv->st_main);
    if (srv->st_copy) cudaStreamDestroy(srv->st_copy);
    delete srv;
}

}  // extern "C"
