/*
 * rcp_oracle.h -- FP64 brute-force CPU oracle for Recursive Camera Painting
 * (Akleman, Mullins, Morrison, Oh; arXiv 2312.12392).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path. Only
 * the test suite, the package smoke check and the benchmark's CPU-baseline leg
 * load it. It shares no code, header or constant with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Everything is computed in double precision from the caller's float32 arrays,
 * widened exactly. Every ray is tested against every primitive (no acceleration
 * structure), so the result is the definition itself.
 *
 * Method (paper §2-§3):
 *   I_n(u,v) = F(I_{n-1}(u,v), S(n))                              (§2, Eq. 1)
 *   F = (1) give every (u,v) its own camera from I_{n-1}(u,v),
 *       (2) render every (u,v) with that camera.                     (§2)
 *   ray direction N = (P'_p - P'_e) / |P'_p - P'_e|                (§2, Eq. 2)
 *   P'_e = P_e + V_e,  P'_p = P_p + V_p                        (§2, Eq. 3-4)
 *   V = lambda * (2 I_{n-1} - 1), in the camera's local frame      (§3, Eq. 5)
 *   I_0 = (0.5, 0.5, 0.5): the first pass is a plain ray-traced image. (§3)
 * Readings where the paper is silent (shading, light, sky, tie-breaking,
 * ambiguity flags) are stated beside each function below.
 *
 * Status codes: 0 ok, -1 bad argument. Nothing here aborts.
 */
#ifndef RCP_ORACLE_H
#define RCP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Colour-to-camera mappings.
 * ORC_MAP_EYE:    V_e = k*(2c-1) in (right, up, forward), V_p = 0: the eye
 *                 moves and the ray is re-aimed at the pixel's focal-plane
 *                 point P_p (a displaced-eye reading of Eq. 3-5).
 * ORC_MAP_TARGET: V_e = 0, V_p = k*(2c-1) in (right, up, forward): the paper's
 *                 own example in §3.
 * ORC_MAP_DEPTH:  V_e = 0, V_p = k*|z - z0|*(2c-1) (§4, Eq. 7); z is the
 *                 previous pass's hit distance, stored beside the colour.
 * ORC_MAP_NORMAL: V_e = 0, V_p = k*(C x N) (§5, Eq. 8); C = the pixel's
 *                 undisplaced pinhole direction, N = the previous pass's hit
 *                 normal (facing its ray), carried in the image's fourth lane
 *                 as a 32-bit octahedral code (0 = no normal: I_0 and misses). */
enum { ORC_MAP_EYE = 0, ORC_MAP_TARGET = 1, ORC_MAP_DEPTH = 2, ORC_MAP_NORMAL = 4 };

/* Octahedral unit-vector code (two 16-bit fields, each q + 32768 with
 * q = round(32767 p) in [-32767, 32767], p the octahedral coordinates), so a
 * real normal never has code 0. */
uint32_t orc_normal_encode(const double n[3]);
/* Returns 0 and zeroes n for code 0, else writes the unit vector and returns 1. */
int orc_normal_decode(uint32_t code, double n[3]);
enum { ORC_LIGHT_POINT = 0, ORC_LIGHT_DIRECTIONAL = 1 };

/* Relative distance under which a ray counts as ambiguous (near an edge, a
 * silhouette, an interval end or a depth tie): distance <= ORC_TOL * (t + |o|). */
#define ORC_TOL 1e-5

typedef struct orc_scene orc_scene;

/* Build an oracle scene. tri: T*9 floats (v0 v1 v2), sph: S*4 floats (centre,
 * radius), albedo: (T+S)*3 floats (triangles first). light: position (point)
 * or direction towards the light (directional; normalised here). The arrays are
 * copied. Returns NULL on a bad argument. */
orc_scene* orc_scene_new(const float* tri, int64_t T, const float* sph, int64_t S,
                         const float* albedo, int light_type, const double light[3],
                         double ambient);
void orc_scene_free(orc_scene* s);
/* Diagonal of the box around all primitives; t_min = 1e-6*diam, shadow offset 1e-4*diam. */
double orc_scene_diam(const orc_scene* s);

/* Per-pixel camera (§2 Eq. 2-4, §3 Eq. 5). cam = eye[3], look_at[3], up[3],
 * fov_y_deg. Pixel (x, y), row 0 at the top; c = previous colour (RGB in [0,1]),
 * z = previous depth (DEPTH mapping only), z0 = focus depth. Writes origin o and
 * unit direction d. Returns 0, or 1 when P'_p == P'_e (direction set to the
 * forward axis). */
int orc_camera_ray(const double cam[10], int W, int H, int x, int y, int mapping,
                   double k, double f, double z0, const double c[3], double z,
                   double o[3], double d[3]);

/* The same camera for a sample at pixel coordinates (px, py) (pixel centre =
 * (x + 0.5, y + 0.5)). */
int orc_camera_ray_at(const double cam[10], int W, int H, double px, double py, int mapping,
                      double k, double f, double z0, const double c[3], double z,
                      double o[3], double d[3]);

/* I_{n-1} as seen by a sample at pixel coordinates (px, py): bilinear between
 * the nearest pixel centres with edge clamping (the normal mapping's code lane
 * from the nearest pixel). */
int orc_sample_image(const float* in, int W, int H, double px, double py, int mapping, double c[4]);

/* Single-primitive tests (exposed for closed-form pins). Return 1 on a hit with
 * t in (tmin, tmax) and write t. */
int orc_hit_triangle(const double v0[3], const double v1[3], const double v2[3],
                     const double o[3], const double d[3], double tmin, double tmax,
                     double* t);
int orc_hit_sphere(const double c[3], double r, const double o[3], const double d[3],
                   double tmin, double tmax, double* t);

/* Closest hit over every primitive, t in (tmin, tmax). Ties in t go to the lower
 * id. prim = -1 on a miss. flag = 1 when the answer is ambiguous at ORC_TOL. */
int orc_trace_closest(const orc_scene* s, const double o[3], const double d[3],
                      double tmin, double tmax, double* t, int64_t* prim, int* flag);
/* Any hit in (tmin, tmax): occluded = 0/1, flag as above; extra_scale is added
 * to (t + |o|) in the ambiguity band (the primary ray's scale, for shadow rays). */
int orc_trace_any(const orc_scene* s, const double o[3], const double d[3], double tmin,
                  double tmax, double extra_scale, int* occluded, int* flag);

/* Shade one primary ray: closest hit, shadow ray, Lambert + ambient, sky on a
 * miss, clamp to [0,1]. rgbz = colour and hit distance (-1 on a miss). */
int orc_shade_ray(const orc_scene* s, const double o[3], const double d[3], double rgbz[4],
                  int64_t* prim, int* flag);

/* One pass I_n = F(I_{n-1}, S) over the listed pixels (pix = NULL: all W*H in
 * row-major order; npix ignored). in_rgbz: H*W*4 floats (RGB + depth) of
 * I_{n-1}, or NULL for I_0 = (0.5,0.5,0.5), depth 0. Outputs per listed pixel:
 * out_rgbz[npix*4], out_prim[npix] (nullable), out_flag[npix] (nullable).
 * nthreads <= 0: all cores. */
int orc_render_pass(const orc_scene* s, const double cam[10], int W, int H, int mapping,
                    double k, double f, double z0, const float* in_rgbz, const int64_t* pix,
                    int64_t npix, double* out_rgbz, int32_t* out_prim, uint8_t* out_flag,
                    int nthreads);

/* K passes from I_0 for the listed pixels. Each pixel's chain depends only on
 * its own previous value (§3), so a subset is exact. Colour is carried in
 * double. Outputs the last pass; out_prim = last pass's prim; out_flag = OR of
 * the flags over all passes. */
int orc_render(const orc_scene* s, const double cam[10], int W, int H, int K, int mapping,
               double k, double f, double z0, const int64_t* pix, int64_t npix,
               double* out_rgbz, int32_t* out_prim, uint8_t* out_flag, int nthreads);

/* Multi-sample pass: spp (1..16) samples per pixel at pixel offsets jitter
 * (2*spp floats in [0,1)); each sample reads in_rgbz (full H*W*4 image or NULL
 * = I_0) at its own position, is traced and shaded; the pixel is the mean
 * (normal mapping: sample 0's code). Outputs per listed pixel as
 * orc_render_pass; out_prim = sample 0's hit. */
int orc_render_pass_ms(const orc_scene* s, const double cam[10], int W, int H, int mapping, double k, double f,
                       double z0, int spp, const float* jitter, const float* in_rgbz, const int64_t* pix,
                       int64_t npix, double* out_rgbz, int32_t* out_prim, uint8_t* out_flag, int nthreads);
/* K multi-sample passes from I_0 over the whole image (W*H*4 doubles out). */
int orc_render_ms(const orc_scene* s, const double cam[10], int W, int H, int K, int mapping, double k, double f,
                  double z0, int spp, const float* jitter, double* out_rgbz, uint8_t* out_flag, int nthreads);

/* Image-space pass (§6: with V_e = 0 a pass reduces to re-sampling the
 * rendered image at a displaced pixel; §6.1: mirrored screen edges). base = the frame's
 * rendered image (H*W*4), prev = I_{n-1} (H*W*4), both float32. For pixel
 * (x, y) with previous colour c, the displacement in pixels is
 *   dx = k_px * (2 c.r - 1),  dy = -k_px * (2 c.g - 1)   (R right, G up: Eq. 5)
 * the sample is the nearest pixel to (x + dx, y + dy), reflected into the
 * image without repeating the edge pixel (-1 -> 0, W -> W-1, repeatedly), and
 * I_n(x, y) = base at that pixel (all four lanes). The displacement and the
 * rounding are done in float32, the precision of the pixel grid decision.
 * Writes npix*4 floats to out (pix = NULL: every pixel). */
int orc_imagespace_pass(const float* base, const float* prev, int W, int H, float k_px, const int64_t* pix,
                        int64_t npix, float* out);
/* The reflection of an integer pixel index into [0, n). */
int64_t orc_mirror_index(int64_t i, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
