/*
 * rcp.h -- C ABI of the GB300 (sm_103a) recursive-camera-painting renderer.
 *
 * Recursive Camera Painting (Akleman, Mullins, Morrison, Oh; arXiv 2312.12392)
 * renders K passes. Pass n gives every pixel (u,v) its own camera, moved by a
 * function of that pixel's value in the previous pass's image, and ray-traces
 * the scene again:  I_n(u,v) = F(I_{n-1}(u,v), S(n))            (§2, Eq. 1)
 * with I_0 = (0.5, 0.5, 0.5), so pass 1 is a plain ray-traced image (§3).
 *
 * Conventions for every entry point:
 *  - Status codes are returned; nothing aborts or throws across the ABI. The
 *    last error message of the calling thread is in rcp_last_error().
 *  - Input arrays are copied; the caller keeps ownership. Output buffers are
 *    allocated by the caller. "host" buffers are ordinary CPU memory; "device"
 *    buffers are CUDA device pointers on the current device.
 *  - Images are row-major, row 0 at the top. "rgbz" images hold 4 floats per
 *    pixel: linear RGB in [0,1] and the z-depth of the pixel's primary hit,
 *    its distance from the pixel's eye along the base camera's unit view axis
 *    F, t (d . F) for a hit at distance t along the unit ray direction d (0 on
 *    a miss; §4's z-depth). "rgb" images hold 3 floats per pixel.
 *  - Primitive ids: triangles 0..T-1, spheres T..T+S-1; -1 marks a miss.
 *  - Valid arguments: 1 <= width, height <= 8192; 1 <= K <= 16; k >= 0;
 *    focal_dist > 0; finite coordinates. Degenerate (zero-area) triangles are
 *    accepted and never hit.
 *  - A scene may be rendered from several threads at once; rcp_scene_update_*
 *    must not run concurrently with renders of the same scene.
 */
#ifndef RCP_H
#define RCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RCP_OK = 0,
    RCP_ERR_ARG = -1,     /* an argument is out of range or NULL */
    RCP_ERR_OOM = -2,     /* device or host allocation failed, or admission refused for good */
    RCP_ERR_CUDA = -3,    /* a CUDA call failed (message says which) */
    RCP_ERR_STACK = -4,   /* BVH deeper than the traversal stack */
    RCP_ERR_TIMEOUT = -5, /* a bounded wait ran out */
    RCP_ERR_STATE = -6    /* call not valid in the object's current state */
} rcp_status;

typedef enum { RCP_LIGHT_POINT = 0, RCP_LIGHT_DIRECTIONAL = 1 } rcp_light_type;

/* v = light position (point) or direction towards the light (directional;
 * normalised by the library). ambient = the ambient term a of the shading
 * c = albedo * (a + (1 - a) * V * max(0, N.L)) (0.1 in the workloads). The
 * paper does not define a shading model; this Lambert + shadow-ray model is the
 * one the library implements. */
typedef struct {
    int32_t type;
    float v[3];
    float ambient;
} rcp_light;

/* Base pinhole camera: eye P_e, look-at point, up vector, vertical FOV. */
typedef struct {
    float eye[3];
    float look_at[3];
    float up[3];
    float fov_y_deg;
} rcp_camera;

/* Colour-to-camera mapping (§2 Eq. 3-4 displacements V_e, V_p; §3 Eq. 5).
 * With d = 2 * I_{n-1}(u,v) - 1 and V = k * (d.r * right + d.g * up +
 * d.b * forward) in the base camera's frame:
 *  RCP_MAP_EYE:    P'_e = P_e + V, ray re-aimed at the pixel's focal-plane point
 *                  P_p (at focal_dist along the view axis).
 *  RCP_MAP_TARGET: P'_e = P_e, P'_p = P_p + V (the paper's §3 example).
 *  RCP_MAP_DEPTH:  P'_e = P_e, P'_p = P_p + |z - z0| * V, z = the previous
 *                  pass's z-depth (§4, Eq. 7).
 *  RCP_MAP_IMAGE:  the image-space reduction of §6 (V_e = 0): pass 1 is traced;
 *                  every later pass re-samples pass 1's image at the pixel
 *                  displaced by k * (2r - 1) to the right and k * (2g - 1) up
 *                  (k in PIXELS for this mapping), nearest pixel, with the
 *                  screen edges mirrored (§6.1). K-pass device and host renders
 *                  only; it needs no scene work after pass 1.
 *  RCP_MAP_NORMAL: P'_e = P_e, P'_p = P_p + k * (C x N) (§5, Eq. 8): C = the
 *                  pixel's undisplaced pinhole direction, N = the previous
 *                  pass's hit normal (facing its ray). For this mapping the
 *                  fourth float of every rgbz pixel holds, as raw bits, a 32-bit
 *                  octahedral code of that normal instead of the z-depth:
 *                  p = (n.x, n.y) / (|n.x| + |n.y| + |n.z|), folded when n.z < 0
 *                  to ((1 - |p.y|) sgn p.x, (1 - |p.x|) sgn p.y) (sgn 0 = +1);
 *                  q = round(32767 p); bits 0-15 hold q.x + 32768 and bits
 *                  16-31 q.y + 32768. Decoding unfolds p (z = 1 - |p.x| - |p.y|,
 *                  and where z < 0 the same fold) and normalises; the round
 *                  trip is within 1e-4 of the unit normal. Code 0 = no normal
 *                  (I_0, misses); no unit normal encodes to 0. */
typedef enum {
    RCP_MAP_EYE = 0,
    RCP_MAP_TARGET = 1,
    RCP_MAP_DEPTH = 2,
    RCP_MAP_IMAGE = 3,
    RCP_MAP_NORMAL = 4
} rcp_mapping;

/* Samples per pixel (§2: any number of jittered samples per pixel). spp <= 0:
 * one sample at the pixel centre (the default). spp in 1..16: samples at pixel
 * offsets (jitter[2s], jitter[2s+1]) in [0,1)^2; each sample reads the previous
 * image bilinearly at its own position (edges clamped; the normal mapping's
 * code lane from the nearest pixel), is traced and shaded, and the pixel is the
 * mean of its samples (the normal mapping keeps sample 0's normal code; hit ids
 * are sample 0's). Not with RCP_MAP_IMAGE. */
#define RCP_MAX_SPP 16

typedef struct {
    int32_t mapping;  /* rcp_mapping */
    float k;          /* displacement strength lambda (world units) */
    float focal_dist; /* distance f of the focal plane along the view axis */
    float z0;         /* in-focus depth of RCP_MAP_DEPTH (ignored otherwise) */
    int32_t spp;      /* samples per pixel, <= 0 = one at the centre */
    float jitter[2 * RCP_MAX_SPP];
} rcp_params;

typedef struct rcp_scene rcp_scene;

/* Scene statistics (sizes, BVH shape, build time). */
typedef struct {
    int64_t n_tris, n_spheres;
    int64_t n_nodes;      /* 8-wide BVH nodes (208 bytes each) */
    int32_t depth;        /* levels of the 8-wide BVH */
    int32_t max_leaf;     /* largest leaf (primitives) */
    int64_t device_bytes; /* device memory held by the scene */
    float diam;           /* diagonal of the scene's bounding box */
    float build_ms;       /* last BVH build (or refit) time on the device */
    int32_t collapse;     /* rcp_collapse policy the BVH was built with */
    int32_t split_max;    /* references per triangle at most (1: no splitting) */
    int64_t n_records;    /* leaf records (48 bytes each): one per reference */
} rcp_scene_info;

/* How the binary tree is collapsed into 8-wide nodes. The paper is silent on
 * acceleration structures; both are choices of this library and give the
 * same images.
 *  RCP_COLLAPSE_AREA (default): each wide node starts from its binary node's
 *    two children and repeatedly opens the child of largest surface area that
 *    holds more than 3 primitives, until it has 8.
 *  RCP_COLLAPSE_SAH: every wide node's 8 slots are shared out among its
 *    binary subtree by a bottom-up dynamic program that minimises the
 *    surface-area cost (a node visit counted as 3.8 primitive tests). Fewer,
 *    fuller nodes; measured faster on scenes of many separate objects (the
 *    forest), slightly slower on a terrain. */
typedef enum { RCP_COLLAPSE_AREA = 0, RCP_COLLAPSE_SAH = 1 } rcp_collapse;

/* Early split clipping (Ernst and Greiner 2007), also a choice of this
 * library: with split_max = m >= 2, a triangle whose box's half-area exceeds
 * 4 times its own area enters the build as up to m references. Its box is
 * halved at the midpoint of the longest axis, the triangle is clipped to each
 * half, and large halves are halved again. Each reference is bounded by the
 * box of its clipped part, so long thin triangles (a cone's sides from apex
 * to base) no longer bloat the boxes above them. Every reference's leaf
 * record is the whole triangle: images are the same as without splitting. A
 * refit (rcp_scene_update_vertices*) bounds every record by its whole moved
 * triangle, which stays correct but gives the benefit up: splitting is meant
 * for static scenes. split_max 0 or 1: no splitting. */
#define RCP_SPLIT_MAX 8

typedef struct {
    int32_t collapse;  /* rcp_collapse */
    int32_t split_max; /* 0 or 1: no splitting; 2..RCP_SPLIT_MAX: references per triangle at most */
} rcp_build_options;

/* Build a scene and its BVH on the device (the scene S(n) of Eq. 1).
 * tri_xyz: host, T*9 floats (v0 v1 v2 per triangle); spheres: host, S*4 floats
 * (centre, radius), may be NULL when S == 0; albedo: host, (T+S)*3 floats,
 * triangles first. The BVH is built on the device (30-bit Morton codes, radix
 * sort, PLOC clustering into a binary tree) and collapsed to an 8-wide BVH with
 * float child boxes, and validated (as rcp_scene_validate) before it is
 * returned. *out receives a handle owned by the library until
 * rcp_scene_destroy. */
rcp_status rcp_scene_create(const float* tri_xyz, int64_t T, const float* spheres, int64_t S,
                            const float* albedo, const rcp_light* light, rcp_scene** out);
/* The same with build options (NULL = the defaults of rcp_scene_create). An
 * unknown collapse policy or split_max outside [0, RCP_SPLIT_MAX] is
 * RCP_ERR_ARG. */
rcp_status rcp_scene_create_ex(const float* tri_xyz, int64_t T, const float* spheres, int64_t S,
                               const float* albedo, const rcp_light* light, const rcp_build_options* options,
                               rcp_scene** out);

/* Move the triangles' vertices (same count and order; host or device array of
 * T*9 floats) and refit the BVH's boxes bottom-up without rebuilding its
 * topology. The scene's diameter, t_min and shadow offset stay those of the
 * original build. `stream` (cudaStream_t or NULL) orders the device variant. */
rcp_status rcp_scene_update_vertices(rcp_scene* scene, const float* tri_xyz);
rcp_status rcp_scene_update_vertices_device(rcp_scene* scene, const float* d_tri_xyz, void* stream);

rcp_status rcp_scene_get_info(const rcp_scene* scene, rcp_scene_info* info);

/* Check the BVH on the device: every primitive in exactly one leaf, every
 * child's box inside its slot box, every primitive inside its leaf box.
 * RCP_OK when all hold; RCP_ERR_STATE with a message otherwise. */
rcp_status rcp_scene_validate(const rcp_scene* scene);

void rcp_scene_destroy(rcp_scene* scene);

/* K passes I_1..I_K from I_0 = 0.5 (§2-§3); writes I_K's RGB to out_rgb (host,
 * width*height*3 floats, row-major from the top row). Synchronous.
 * Where the device reads and writes pageable host memory coherently (a
 * Grace-class host), the last pass stores the RGB straight into out_rgb while
 * it traces; elsewhere, and for RCP_MAP_IMAGE, the image is packed on the
 * device and copied. Either way the values are the same. Before the render the
 * calling thread reads and writes back one byte of every page of out_rgb, so a
 * bad pointer faults on the host, as a copy into it would. */
rcp_status rcp_render(const rcp_scene* scene, const rcp_camera* cam, int width, int height, int K,
                      const rcp_params* params, float* out_rgb);

/* One pass I_n = F(I_{n-1}, S): in_rgbz (host, width*height*4, NULL = I_0)
 * -> out_rgbz (host, width*height*4); out_prim (host, width*height int32,
 * nullable) receives each pixel's primary-hit id. Synchronous. */
rcp_status rcp_render_pass(const rcp_scene* scene, const rcp_camera* cam, int width, int height,
                           const rcp_params* params, const float* in_rgbz, float* out_rgbz,
                           int32_t* out_prim);

/* Device variant of both: K passes starting from d_in (device rgbz image, NULL =
 * I_0), final image to d_out (device, width*height*4 floats; may equal d_in,
 * except for a one-pass (K = 1) render with spp > 0, whose samples read
 * neighbouring pixels of d_in),
 * last pass's hit ids to d_prim (device, nullable). Enqueued on `stream`
 * (cudaStream_t, NULL = legacy default); the call returns once enqueued. The
 * K-pass sequence is captured once per (scene, shape, K) in a CUDA graph and
 * replayed. Intermediate images live in library-owned device memory. */
rcp_status rcp_render_device(const rcp_scene* scene, const rcp_camera* cam, int width, int height,
                             int K, const rcp_params* params, const float* d_in, float* d_out,
                             int32_t* d_prim, void* stream);

/* One image-space pass (§6, §6.1) on device images (rgbz, width*height*4
 * floats each): out(x,y) = base at the nearest pixel to (x + k_px (2r - 1),
 * y - k_px (2g - 1)), (r, g) = prev(x,y), indices reflected into the image
 * without repeating the edge pixel (-1 -> 0, width -> width-1, repeatedly).
 * The displacement and rounding are computed in float32. out must not alias
 * base or prev. Enqueued on `stream`. */
rcp_status rcp_imagespace_pass_device(const float* d_base, const float* d_prev, float* d_out, int width,
                                      int height, float k_px, void* stream);

/* Many views of one scene in one persistent launch per pass (§2's per-(u,v)
 * cameras for every view at once). cams, widths, heights: host arrays of
 * n_views. d_ins: NULL (every view starts from I_0) or a host array of n_views
 * device pointers, each a view's previous rgbz image or NULL (I_0); the same
 * aliasing rule as rcp_render_device. d_outs: host array of n_views device
 * pointers (rgbz, width*height*4 floats each). d_prims: NULL or a host array of
 * n_views device pointers (width*height int32 each, or NULL) receiving the
 * last pass's hit ids. All views run K passes; the K-pass recursion is
 * captured in a CUDA graph keyed by the view shapes. Enqueued on `stream`. */
rcp_status rcp_render_batch_device(const rcp_scene* scene, int n_views, const rcp_camera* cams,
                                   const int* widths, const int* heights, int K,
                                   const rcp_params* params, const float* const* d_ins,
                                   float* const* d_outs, int32_t* const* d_prims, void* stream);

/* Traversal tuning. block: threads per block (64, 128, 256); blocks_per_sm:
 * resident blocks of the persistent launch (0 = occupancy maximum); chunk:
 * pixels a warp claims per fetch (32 or 64, the rays per warp); fused_camera:
 * 1 = rays are made inside the trace kernel, 0 = a separate camera kernel
 * writes a ray buffer; stack_entries: traversal-stack entries per thread kept
 * in shared memory (0 = one per tree level, the walk's deepest need; fewer
 * entries spill the deeper levels to a library-owned global-memory region);
 * hints: bit 0 = each pixel's walk first tests the primitive its ray hit in the
 * previous pass (a closer far limit from the start), bit 1 = its shadow walk
 * first tests its previous occluder; chain_passes: 1 = one launch runs all K
 * passes, each warp carrying the pixels of its tile from pass to pass in
 * registers (renders of K >= 2 at one sample per pixel with the fused camera
 * and any mapping but RCP_MAP_IMAGE; others run one launch per pass). A new
 * scene starts at {128, 0, 32, 1, 0, 3, 1}. No choice changes any result. */
typedef struct {
    int32_t block;
    int32_t blocks_per_sm;
    int32_t chunk;
    int32_t fused_camera;
    int32_t stack_entries;
    int32_t hints;
    int32_t chain_passes;
} rcp_tuning;

rcp_status rcp_get_tuning(const rcp_scene* scene, rcp_tuning* out);
rcp_status rcp_set_tuning(rcp_scene* scene, const rcp_tuning* tuning);

/* Time every tuning candidate on this scene and view (a K = 4 render each):
 * one launch per pass over block x chunk x fused camera x shared stack depth
 * (the depth a full tree walk needs, or half of it) x hints on or off, and
 * chained passes over block x chunk x stack depth x hints. Keep the fastest in
 * the scene and return it. cache_path (nullable): a
 * JSON file of earlier results, keyed by GPU name, scene size class, tree depth
 * and view size; read before and updated after the search. */
rcp_status rcp_autotune(rcp_scene* scene, const rcp_camera* cam, int width, int height,
                        const rcp_params* params, const char* cache_path, rcp_tuning* out);

/* Work counters of one pass over the given view, from an instrumented copy of
 * the trace kernels: rays traced, 8-wide nodes visited, child boxes tested,
 * triangle and sphere tests. Used for the algorithmic bytes and FLOPs. */
typedef struct {
    int64_t rays, primary_rays, shadow_rays;
    int64_t nodes, box_tests, tri_tests, sphere_tests;
} rcp_counters;

/* Rays traced (primary, shadow) by the scene's most recent rcp_render*
 * call, counted on the device during that render. Read it after the render
 * has completed (synchronise its stream first). */
rcp_status rcp_last_ray_counts(const rcp_scene* scene, int64_t* primary, int64_t* shadow);

/* d_in: previous image (device rgbz, NULL = I_0); d_out: this pass's image
 * (device rgbz, nullable), so that counted passes can be chained. */
rcp_status rcp_count_pass(const rcp_scene* scene, const rcp_camera* cam, int width, int height,
                          const rcp_params* params, const float* d_in, float* d_out, rcp_counters* out);

/* Device time (ms) of each launch of the scene's most recent render, from CUDA
 * events recorded on the render's stream between the launches (inside the
 * captured graph): one per pass, or one for all K passes when they ran
 * chained. Read after the render has completed. */
rcp_status rcp_last_pass_times(const rcp_scene* scene, float* ms, int max_passes, int* n_passes);

/* Bytes that one rcp_render call of K passes over n_views views copies from
 * host to device: the views' per-pass descriptors (camera terms, image
 * pointers), uploaded once per call. The library's own bookkeeping, not part of
 * the method. A render whose passes run chained uploads one descriptor per
 * view: rcp_render_h2d_bytes(n_views, 1). Returns -1 when K or n_views is out
 * of range. */
int64_t rcp_render_h2d_bytes(int n_views, int K);

/* Diagnostics used by the tests (all device pointers, enqueued on `stream`):
 *  rcp_debug_trace: n rays, orig_tmin[n*4] = (origin, t_min), dir_tmax[n*4] =
 *    (unit direction, t_max); any_hit 0 = closest hit (t_out, prim_out), 1 =
 *    any hit (prim_out = 1 occluded / 0 free, t_out unused); brute 1 tests
 *    every primitive instead of walking the BVH; stack_entries: the walk's
 *    stack (0 = 64 entries); a walk that needs more drops the deeper groups and
 *    the call returns RCP_ERR_STACK.
 *  rcp_debug_sort_pairs: stable LSD radix sort of n (key, value) pairs on the
 *    low `bits` bits of the keys, in place.
 *  rcp_debug_morton: 30-bit Morton codes of n points (xyz[n*3]) in the cube
 *    with corner lo[3] and side max_a(hi[a] - lo[a]) (host arrays). */
rcp_status rcp_debug_trace(const rcp_scene* scene, int64_t n, const float* orig_tmin,
                           const float* dir_tmax, int any_hit, int brute, float* t_out,
                           int32_t* prim_out, int stack_entries, void* stream);
rcp_status rcp_debug_sort_pairs(uint32_t* keys, uint32_t* values, int64_t n, int bits, void* stream);
rcp_status rcp_debug_morton(const float* xyz, int64_t n, const float* lo, const float* hi,
                            uint32_t* codes, void* stream);
/* Test of the radix sort's bounded wait: one block of a sort pass takes the
 * second of two tiles while the first never runs, so its look-back waits for
 * counts that are never published. Each wait gives up after spin_limit polls
 * (1 <= spin_limit <= 2^20; a real sort allows 2^26), sets the sort's error
 * flag and the block finishes. Returns RCP_ERR_TIMEOUT when the flag was set,
 * as a sort whose wait ran out does. Synchronous; allocates its own buffers. */
rcp_status rcp_debug_sort_lookback_timeout(int64_t spin_limit, void* stream);

/* Allocation-free sort. The paper has no counterpart: this is a library
 * facility. Some callers cannot allocate device memory at the point where they
 * need to sort: real-time loops that must not allocate once they are running
 * (an allocation can block on the device or fail late), and hosts that own all
 * device memory and hand the library no allocator of its own. This entry
 * point does the same stable LSD radix sort as rcp_debug_sort_pairs (keys and
 * values are device arrays of n uint32, sorted in place on the low `bits` bits
 * of the keys, enqueued on `stream`), but all of its scratch lives in one fixed
 * device array compiled into the library, of about 8.7 MB, which every GPU that
 * loads the library holds until the process exits; it calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *  - n may be at most RCP_SORT_STATIC_MAX_PAIRS (also returned by
 *    rcp_sort_static_capacity); larger n returns RCP_ERR_ARG with a message
 *    saying so.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture begins.
 *  - Every call reuses the same array and clears what must start at zero;
 *    calls whose work overlaps on the GPU (other streams, other host threads)
 *    race on it: serialise them.
 *  - The call waits for the sort to finish before it returns (it reads the
 *    sort's error flag); RCP_ERR_TIMEOUT reports a look-back wait that ran out. */
#define RCP_SORT_STATIC_MAX_PAIRS 1048576
rcp_status rcp_sort_pairs_static(uint32_t* keys, uint32_t* values, int64_t n, int bits, void* stream);
/* The largest n rcp_sort_pairs_static accepts (RCP_SORT_STATIC_MAX_PAIRS of
 * the library as built). */
int64_t rcp_sort_static_capacity(void);

/* ------------------------------------------------------------ serving ---
 * A request = one K-pass render of a resident scene. Requests are admitted
 * (first come first served) while a slot is free and their device memory (two
 * rgbz images, per-pixel hit hints, and an RGB staging buffer unless the last
 * pass writes the caller's buffer) fits the budget; the server backs the
 * device's stream-ordered memory pool with up to 8 GB of it at creation. Each
 * scheduler step advances admitted requests in ONE launch over all of their
 * views, whatever their scene, size or K (continuous batching): in admission
 * order, the oldest always (by one pass at least), each request by as many of
 * its remaining passes as the step's pixel-pass budget still holds
 * (rcp_server_set_step_pixels, at most rcp_server_set_max_chain), which run
 * chained (each pixel carried from pass to pass in registers); a step that
 * holds a multi-sample request advances every request by one pass. A request
 * is finished as soon as its own tiles of its final step are, not at the end
 * of the step's launch (views are queued grouped by scene, oldest first); its
 * image is then in the caller's host buffer. A request whose traversal stack
 * overflowed fails with RCP_ERR_STACK. */
typedef struct rcp_server rcp_server;

typedef struct {
    int64_t submitted, completed, rejected, in_flight, queued;
    int64_t steps;        /* scheduler steps (launches) */
    double p50_ms, p99_ms; /* submit-to-complete latency of completed requests */
    double frames_per_s;  /* completed requests per second since the first submit */
    double mrays_per_s;   /* primary + shadow rays per second over the same span */
    int64_t device_bytes_in_use, device_bytes_peak;
    double device_busy_ms; /* device time of the steps completed so far (CUDA events around each step) */
} rcp_server_stats;

rcp_status rcp_server_create(int64_t mem_budget_bytes, int max_slots, rcp_server** out);
/* out_rgb: host, width*height*3 floats, caller-owned until the request is done.
 * As in rcp_render, a device that reads and writes pageable host memory
 * coherently writes the RGB into out_rgb itself during the request's last
 * pass; the submitting thread touches every page of out_rgb first. */
rcp_status rcp_server_submit(rcp_server* srv, const rcp_scene* scene, const rcp_camera* cam,
                             int width, int height, int K, const rcp_params* params, float* out_rgb,
                             int64_t* ticket);
/* Pixel-passes one scheduler step may hold (default 67,000,000, so that a
 * 3840x2160 K=8 request runs to its end in one step; 0 = every admitted
 * request to its end in every step). The oldest admitted request always
 * advances, whatever its size. */
rcp_status rcp_server_set_step_pixels(rcp_server* srv, int64_t pixels);
/* Passes a request may advance by in one step (1..16, default 16; 1 = one
 * pass per request per step). */
rcp_status rcp_server_set_max_chain(rcp_server* srv, int passes);
/* done = 1 finished, 0 pending; the request's own status is returned. */
rcp_status rcp_server_poll(rcp_server* srv, int64_t ticket, int* done);
rcp_status rcp_server_wait(rcp_server* srv, int64_t ticket, double timeout_s);
/* Submit-to-done latency in ms of a finished request (RCP_ERR_STATE while it
 * is pending). */
rcp_status rcp_server_latency(rcp_server* srv, int64_t ticket, double* ms);
rcp_status rcp_server_stats_get(rcp_server* srv, rcp_server_stats* out);
/* Drop queued requests and stop after the in-flight ones finish. */
void rcp_server_destroy(rcp_server* srv);

/* How rcp_render and the server deliver a frame into a caller's host buffer:
 * the last pass writes the RGB into it directly while it traces, or the image
 * is packed on the device and copied. A page-locked buffer (cudaMallocHost,
 * cudaHostRegister) is mapped in the GPU's page tables and written directly.
 * A pageable buffer can be written directly only where the device reads and
 * writes pageable host memory coherently (a Grace-class host), through the
 * GPU's translation of host addresses: for a buffer the GPU wrote recently
 * that costs nothing, for one it has not (a fresh buffer) it is much slower
 * than packing and copying.
 *  RCP_HOST_OUTPUT_AUTO (default): page-locked buffers directly; pageable ones
 *    directly if one of the last 8 pageable buffers written directly (same
 *    address and size), else pack and copy (a buffer used again is written
 *    directly from its second use on).
 *  RCP_HOST_OUTPUT_DIRECT: directly whenever the device can reach the buffer.
 *  RCP_HOST_OUTPUT_COPY: always pack and copy.
 * Process-wide; the images are the same either way. */
typedef enum { RCP_HOST_OUTPUT_AUTO = 0, RCP_HOST_OUTPUT_DIRECT = 1, RCP_HOST_OUTPUT_COPY = 2 } rcp_host_output;
rcp_status rcp_set_host_output(int mode);
int rcp_get_host_output(void);

/* Message of the calling thread's last failed call ("" if none). */
const char* rcp_last_error(void);
/* Library version string. */
const char* rcp_version(void);

#ifdef __cplusplus
}
#endif
#endif
