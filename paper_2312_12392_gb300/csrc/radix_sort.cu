// radix_sort.cu -- onesweep LSD radix sort of (uint32 key, uint32 value) pairs.
//
// Used by the BVH builder to order primitives by 30-bit Morton code. One
// histogram kernel counts all digit passes at once; then one kernel per 8-bit
// digit ranks a tile of keys in shared memory (warp match + per-warp counters,
// stable), finds the tile's global offset per digit by decoupled look-back over
// earlier tiles (tiles are numbered in launch order by an atomic counter, so
// every earlier tile is already running), and scatters through shared memory
// so that writes of one digit run are contiguous.
//
// Every wait on another tile's status is bounded: after spin_limit polls
// (SPIN_LIMIT in a sort) the kernel records an error flag and proceeds, so a
// fault in the protocol shows up as an error status instead of a hang.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "rcp_internal.cuh"

namespace rcp {

namespace {

constexpr int RADIX = 256;
constexpr int SORT_BLOCK = 256;  // one thread per digit in the scan/look-back steps
constexpr int SORT_WARPS = SORT_BLOCK / 32;
constexpr int ITEMS = 15;
constexpr int TILE = SORT_BLOCK * ITEMS;  // 3840 keys
constexpr uint32_t FLAG_AGG = 1u << 30;
constexpr uint32_t FLAG_INC = 2u << 30;
constexpr uint32_t COUNT_MASK = (1u << 30) - 1;
constexpr long long SPIN_LIMIT = 1ll << 26;

__global__ void __launch_bounds__(SORT_BLOCK) k_histogram(const uint32_t* __restrict__ keys, int64_t n,
                                                          int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[4][RADIX];
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// Exclusive scan of each pass's 256 bins (one block of 256 threads).
__global__ void k_scan_histogram(uint32_t* hist, int passes) {
    __shared__ uint32_t s[RADIX];
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = hist[p * RADIX + threadIdx.x];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < RADIX; off <<= 1) {
            uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        hist[p * RADIX + threadIdx.x] = s[threadIdx.x] - v;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SORT_BLOCK) k_onesweep(const uint32_t* __restrict__ keys_in,
                                                         const uint32_t* __restrict__ vals_in,
                                                         uint32_t* __restrict__ keys_out,
                                                         uint32_t* __restrict__ vals_out, int64_t n, int shift,
                                                         const uint32_t* __restrict__ bucket_base,
                                                         uint32_t* status, uint32_t* tile_counter,
                                                         int* error_flag, long long spin_limit) {
    __shared__ uint32_t s_keys[TILE];
    __shared__ uint32_t s_vals[TILE];
    __shared__ uint32_t s_wcnt[SORT_WARPS][RADIX];
    __shared__ uint32_t s_tile_off[RADIX];
    __shared__ uint32_t s_global[RADIX];
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_BLOCK) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t base = (int64_t)tile * TILE;

    uint32_t k[ITEMS], v[ITEMS], rank[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t idx = base + (int64_t)warp * (32 * ITEMS) + j * 32 + lane;
        if (idx < n) {
            k[j] = keys_in[idx];
            v[j] = vals_in[idx];
        } else {
            k[j] = 0xffffffffu;  // past the end: ranks after every real key of its digit
            v[j] = 0;
        }
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t d = (k[j] >> shift) & 0xff;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = s_wcnt[warp][d];
        rank[j] = before + __popc(peers & lt);
        __syncwarp();
        if ((peers >> lane) == 1u) s_wcnt[warp][d] = before + __popc(peers);  // highest lane of the group
        __syncwarp();
    }
    __syncthreads();

    // per digit: exclusive scan over warps, then the tile's count
    {
        const int d = tid;
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = sum;
            sum += c;
        }
        const uint32_t count = sum;
        // publish this tile's aggregate (tile 0 is already inclusive)
        volatile uint32_t* st = status + (size_t)tile * RADIX;
        __threadfence();
        st[d] = (tile == 0 ? FLAG_INC : FLAG_AGG) | count;
        // look back over earlier tiles
        uint32_t prefix = 0;
        if (tile > 0) {
            int64_t t = (int64_t)tile - 1;
            long long spins = 0;
            while (t >= 0) {
                const uint32_t sv = ((volatile uint32_t*)status)[(size_t)t * RADIX + d];
                const uint32_t flag = sv & ~COUNT_MASK;
                if (flag == 0) {
                    if (++spins > spin_limit) {
                        atomicExch(error_flag, 1);
                        break;
                    }
                    continue;
                }
                prefix += sv & COUNT_MASK;
                if (flag == FLAG_INC) break;
                --t;
            }
            __threadfence();
            st[d] = FLAG_INC | (prefix + count);
        }
        s_global[d] = bucket_base[d] + prefix;
        s_tile_off[d] = count;
    }
    __syncthreads();
    // exclusive scan of the tile's digit counts -> tile offsets (Hillis-Steele)
    {
        const uint32_t c = s_tile_off[tid];
        uint32_t x = c;
        for (int off = 1; off < RADIX; off <<= 1) {
            __syncthreads();
            const uint32_t y = tid >= off ? s_tile_off[tid - off] : 0;
            __syncthreads();
            x += y;
            s_tile_off[tid] = x;
        }
        __syncthreads();
        s_tile_off[tid] = x - c;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t d = (k[j] >> shift) & 0xff;
        const uint32_t r = s_tile_off[d] + s_wcnt[warp][d] + rank[j];
        s_keys[r] = k[j];
        s_vals[r] = v[j];
    }
    __syncthreads();
    const int64_t valid = n - base < TILE ? n - base : TILE;
    for (int pos = tid; pos < valid; pos += SORT_BLOCK) {
        const uint32_t key = s_keys[pos];
        const uint32_t d = (key >> shift) & 0xff;
        const uint32_t dst = s_global[d] + (pos - s_tile_off[d]);
        keys_out[dst] = key;
        vals_out[dst] = s_vals[pos];
    }
}

}  // namespace

// Sort n pairs in place on the low `bits` bits of the keys. alt_keys/alt_vals
// are n-element scratch buffers; scratch holds the histogram, tile status and
// counters (size from radix_sort_scratch_bytes).
size_t radix_sort_scratch_bytes(int64_t n) {
    const int64_t tiles = (n + TILE - 1) / TILE;
    return sizeof(uint32_t) * (4 * RADIX + 8 + (size_t)(tiles > 0 ? tiles : 1) * RADIX);
}

rcp_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* alt_keys, uint32_t* alt_vals,
                            int64_t n, int bits, void* scratch, int* d_error, cudaStream_t stream) {
    if (n <= 1) return RCP_OK;
    if (n >= (int64_t)COUNT_MASK) {
        set_error("radix sort: too many keys (limit 2^30)");
        return RCP_ERR_ARG;
    }
    const int passes = (bits + 7) / 8;
    const int64_t tiles = (n + TILE - 1) / TILE;
    uint32_t* hist = (uint32_t*)scratch;
    uint32_t* counters = hist + 4 * RADIX;  // one tile counter per pass
    uint32_t* status = counters + 8;
    RCP_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (4 * RADIX + 8), stream));
    int sms = 0, dev = 0;
    RCP_CUDA(cudaGetDevice(&dev));
    RCP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t hblocks = (n + SORT_BLOCK * 16 - 1) / (SORT_BLOCK * 16);
    if (hblocks > sms * 8) hblocks = sms * 8;
    k_histogram<<<(int)hblocks, SORT_BLOCK, 0, stream>>>(keys, n, passes, hist);
    k_scan_histogram<<<1, RADIX, 0, stream>>>(hist, passes);
    uint32_t *ki = keys, *vi = vals, *ko = alt_keys, *vo = alt_vals;
    for (int p = 0; p < passes; ++p) {
        RCP_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t) * (size_t)tiles * RADIX, stream));
        k_onesweep<<<(int)tiles, SORT_BLOCK, 0, stream>>>(ki, vi, ko, vo, n, 8 * p, hist + p * RADIX, status,
                                                           counters + p, d_error, SPIN_LIMIT);
        uint32_t* t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    if (ki != keys) {
        RCP_CUDA(cudaMemcpyAsync(keys, ki, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, stream));
        RCP_CUDA(cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, stream));
    }
    RCP_CUDA(cudaGetLastError());
    return RCP_OK;
}

}  // namespace rcp

// ---------------------------------------------------------------- allocation-free variant
//
// rcp_sort_pairs_static: the same sort with every scratch buffer (ping-pong
// keys and values, digit histograms, tile status, tile counters, the look-back
// error flag) carved out of one file-scope device array, so the call never
// allocates device memory.

namespace rcp {
namespace {

constexpr int64_t STATIC_MAX = RCP_SORT_STATIC_MAX_PAIRS;
constexpr int64_t STATIC_TILES = (STATIC_MAX + TILE - 1) / TILE;
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_KEYS = 0;
constexpr size_t OFF_VALS = align256(OFF_KEYS + sizeof(uint32_t) * STATIC_MAX);
constexpr size_t OFF_SCRATCH = align256(OFF_VALS + sizeof(uint32_t) * STATIC_MAX);
constexpr size_t SCRATCH_BYTES = sizeof(uint32_t) * (4 * RADIX + 8 + STATIC_TILES * RADIX);
constexpr size_t OFF_ERROR = align256(OFF_SCRATCH + SCRATCH_BYTES);
constexpr size_t STATIC_BYTES = align256(OFF_ERROR + sizeof(int));

}  // namespace
}  // namespace rcp

// Held by every device that loads the library, for the life of the process.
static __device__ __align__(256) unsigned char g_sort_static_scratch[rcp::STATIC_BYTES];

namespace rcp {
namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_static_mu;
void* g_static_ptr[MAX_DEVICES] = {};

// Device address of the static scratch on the current device, looked up once
// per device (host code cannot use the array's name as a device pointer).
rcp_status static_scratch(unsigned char** out) {
    int dev = 0;
    RCP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("rcp_sort_pairs_static: device ordinal out of range");
        return RCP_ERR_STATE;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sort_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_sort_static_scratch)");
        g_static_ptr[dev] = p;
    }
    *out = (unsigned char*)g_static_ptr[dev];
    return RCP_OK;
}

}  // namespace
}  // namespace rcp

extern "C" int64_t rcp_sort_static_capacity(void) { return rcp::STATIC_MAX; }

extern "C" rcp_status rcp_sort_pairs_static(uint32_t* keys, uint32_t* values, int64_t n, int bits, void* stream) {
    using namespace rcp;
    if (n < 0 || bits < 1 || bits > 32 || (n > 0 && (!keys || !values))) {
        set_error("rcp_sort_pairs_static: bad argument");
        return RCP_ERR_ARG;
    }
    if (n > STATIC_MAX) {
        set_error("rcp_sort_pairs_static: n = " + std::to_string(n) +
                  " exceeds the static scratch capacity of RCP_SORT_STATIC_MAX_PAIRS (" + std::to_string(STATIC_MAX) +
                  ") pairs");
        return RCP_ERR_ARG;
    }
    if (n <= 1) return RCP_OK;
    unsigned char* base = nullptr;
    rcp_status r = static_scratch(&base);
    if (r != RCP_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    int* d_err = (int*)(base + OFF_ERROR);
    RCP_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));  // the array keeps the last call's contents
    r = radix_sort_pairs(keys, values, (uint32_t*)(base + OFF_KEYS), (uint32_t*)(base + OFF_VALS), n, bits,
                         base + OFF_SCRATCH, d_err, st);
    if (r != RCP_OK) return r;
    int h = 0;
    RCP_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RCP_CUDA(cudaStreamSynchronize(st));
    if (h) {
        set_error("rcp_sort_pairs_static: look-back wait ran out");
        return RCP_ERR_TIMEOUT;
    }
    return RCP_OK;
}

// ---------------------------------------------------------------- test of the bounded wait
//
// rcp_debug_sort_lookback_timeout: one onesweep block takes tile 1 of a
// two-tile pass while tile 0 never runs, so every one of its look-back waits
// polls a status that nothing publishes. After spin_limit polls each wait
// gives up and sets the error flag, and the block finishes its tile with a
// partial offset. With every key 0 all of the block's keys go to digit 0,
// whose bucket starts at 0, so its writes land at indices [0, TILE) of the
// 2 TILE-element output arrays.

extern "C" rcp_status rcp_debug_sort_lookback_timeout(int64_t spin_limit, void* stream) {
    using namespace rcp;
    if (spin_limit < 1 || spin_limit > (1ll << 20)) {
        set_error("rcp_debug_sort_lookback_timeout: spin_limit outside [1, 2^20]");
        return RCP_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = 2 * (int64_t)TILE;
    DevBuf<uint32_t> keys, vals, ko, vo, scratch;
    DevBuf<int> err;
    RCP_CUDA(keys.alloc(n));
    RCP_CUDA(vals.alloc(n));
    RCP_CUDA(ko.alloc(n));
    RCP_CUDA(vo.alloc(n));
    RCP_CUDA(scratch.alloc(4 * RADIX + 8 + 2 * RADIX));
    RCP_CUDA(err.alloc(1));
    uint32_t* hist = scratch.p;
    uint32_t* counter = hist + 4 * RADIX;
    uint32_t* status = counter + 8;
    RCP_CUDA(cudaMemsetAsync(keys.p, 0, sizeof(uint32_t) * n, st));
    RCP_CUDA(cudaMemsetAsync(vals.p, 0, sizeof(uint32_t) * n, st));
    RCP_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(uint32_t) * (4 * RADIX + 8 + 2 * RADIX), st));
    RCP_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    k_histogram<<<2, SORT_BLOCK, 0, st>>>(keys.p, n, 1, hist);
    k_scan_histogram<<<1, RADIX, 0, st>>>(hist, 1);
    const uint32_t one = 1;  // the block claims tile 1; tile 0 is never claimed
    RCP_CUDA(cudaMemcpyAsync(counter, &one, sizeof(one), cudaMemcpyHostToDevice, st));
    k_onesweep<<<1, SORT_BLOCK, 0, st>>>(keys.p, vals.p, ko.p, vo.p, n, 0, hist, status, counter, err.p,
                                         (long long)spin_limit);
    RCP_CUDA(cudaGetLastError());
    int h = 0;
    RCP_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RCP_CUDA(cudaStreamSynchronize(st));
    if (h) {
        set_error("radix sort: look-back wait ran out");
        return RCP_ERR_TIMEOUT;
    }
    return RCP_OK;
}
