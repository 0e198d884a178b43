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
 *                 previous pass's z-depth, stored beside the colour.
 * ORC_MAP_NORMAL: V_e = 0, V_p = k*(C x N) (§5, Eq. 8); C = the pixel's
 *                 undisplaced pinhole direction, N = the previous pass's hit
 *                 normal (facing its ray), carried between passes as a unit
 *                 vector in double precision (the zero vector = no normal: I_0
 *                 and misses). */
enum { ORC_MAP_EYE = 0, ORC_MAP_TARGET = 1, ORC_MAP_DEPTH = 2, ORC_MAP_NORMAL = 4 };
enum { ORC_LIGHT_POINT = 0, ORC_LIGHT_DIRECTIONAL = 1 };

/* Per-ray ambiguity flags (bits). A float32 renderer may legitimately differ
 * from this oracle only where a flag is set:
 *  ORC_FLAG_ID:     the primary hit's primitive may differ (the ray passes near
 *                   an outline or silhouette, near an end of its t interval, or
 *                   two surfaces are hit at nearly the same depth; also a
 *                   degenerate camera, P'_p == P'_e);
 *  ORC_FLAG_SHADOW: the shadow ray's occlusion may differ;
 *  ORC_FLAG_POINT:  the primary hit point itself is ill-conditioned (a sphere
 *                   hit grazing its silhouette or with a root near t_min, or a
 *                   degenerate camera): even the same primitive may then be
 *                   shaded differently. */
#define ORC_FLAG_ID 1
#define ORC_FLAG_SHADOW 2
#define ORC_FLAG_POINT 4

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
 * z = previous z-depth (DEPTH mapping), z0 = focus depth, nrm = previous unit
 * hit normal (NORMAL mapping; NULL or the zero vector = no normal). Writes
 * origin o and unit direction d. Returns 0, or 1 when P'_p == P'_e (direction
 * set to the forward axis). */
int orc_camera_ray(const double cam[10], int W, int H, int x, int y, int mapping,
                   double k, double f, double z0, const double c[3], double z, const double nrm[3],
                   double o[3], double d[3]);

/* The same camera for a sample at pixel coordinates (px, py) (pixel centre =
 * (x + 0.5, y + 0.5)). */
int orc_camera_ray_at(const double cam[10], int W, int H, double px, double py, int mapping,
                      double k, double f, double z0, const double c[3], double z, const double nrm[3],
                      double o[3], double d[3]);

/* I_{n-1} as seen by a sample at pixel coordinates (px, py): bilinear between
 * the four nearest pixel centres (all four lanes), indices clamped to the
 * image. */
int orc_sample_image(const float* in, int W, int H, double px, double py, double c[4]);
/* Index y*W + x of the pixel whose centre is nearest to (px, py), clamped to
 * the image (halves round up): where a sample reads the previous normal. */
int64_t orc_nearest_pixel(int W, int H, double px, double py);

/* Single-primitive tests (exposed for closed-form pins). Return 1 on a hit with
 * t in (tmin, tmax) and write t. */
int orc_hit_triangle(const double v0[3], const double v1[3], const double v2[3],
                     const double o[3], const double d[3], double tmin, double tmax,
                     double* t);
int orc_hit_sphere(const double c[3], double r, const double o[3], const double d[3],
                   double tmin, double tmax, double* t);

/* Closest hit over every primitive, t in (tmin, tmax). Ties in t go to the lower
 * id. prim = -1 on a miss. flag = ORC_FLAG_ID and/or ORC_FLAG_POINT bits. */
int orc_trace_closest(const orc_scene* s, const double o[3], const double d[3],
                      double tmin, double tmax, double* t, int64_t* prim, int* flag);
/* Any hit in (tmin, tmax): occluded = 0/1, flag = 1 when the answer is
 * ambiguous at ORC_TOL; extra_scale is added to (t + |o|) in the ambiguity band
 * (the primary ray's scale, for shadow rays). */
int orc_trace_any(const orc_scene* s, const double o[3], const double d[3], double tmin,
                  double tmax, double extra_scale, int* occluded, int* flag);

/* Shade one primary ray: closest hit, shadow ray, Lambert + ambient, sky on a
 * miss, clamp to [0,1]. rgbt = colour and hit distance t along d (-1 on a
 * miss); nrm (nullable) = the hit's unit normal facing the ray (zero on a
 * miss); flag = ORC_FLAG_* bits. */
int orc_shade_ray(const orc_scene* s, const double o[3], const double d[3], double rgbt[4], double nrm[3],
                  int64_t* prim, int* flag);

/* One pass I_n = F(I_{n-1}, S) over the listed pixels (pix = NULL: all W*H in
 * row-major order; npix ignored). in_rgbz: H*W*4 floats (RGB + z-depth) of
 * I_{n-1}, or NULL for I_0 = (0.5,0.5,0.5), depth 0. in_normal: H*W*3 doubles,
 * the previous pass's hit normals (NORMAL mapping; NULL = none). Outputs per
 * listed pixel: out_rgbz[npix*4] (colour, z-depth of the primary hit along the
 * base camera's view axis, 0 on a miss), out_normal[npix*3] (nullable; zero on
 * a miss), out_prim[npix] (nullable), out_flag[npix] (nullable, ORC_FLAG_*
 * bits). nthreads <= 0: all cores. */
int orc_render_pass(const orc_scene* s, const double cam[10], int W, int H, int mapping,
                    double k, double f, double z0, const float* in_rgbz, const double* in_normal,
                    const int64_t* pix, int64_t npix, double* out_rgbz, double* out_normal,
                    int32_t* out_prim, uint8_t* out_flag, int nthreads);

/* K passes from I_0 for the listed pixels. Each pixel's chain depends only on
 * its own previous value (§3), so a subset is exact. Colour, depth and normal
 * are carried in double. Outputs the last pass; out_prim = last pass's prim;
 * out_flag = OR of the flags over all passes. */
int orc_render(const orc_scene* s, const double cam[10], int W, int H, int K, int mapping,
               double k, double f, double z0, const int64_t* pix, int64_t npix,
               double* out_rgbz, double* out_normal, int32_t* out_prim, uint8_t* out_flag, int nthreads);

/* Multi-sample pass: spp (1..16) samples per pixel at pixel offsets jitter
 * (2*spp floats in [0,1)); each sample reads in_rgbz (full H*W*4 image or NULL
 * = I_0) bilinearly at its own position and in_normal (H*W*3 or NULL) at the
 * nearest pixel, is traced and shaded; the pixel is the mean of its samples
 * (colour and depth; the normal is sample 0's). Outputs per listed pixel as
 * orc_render_pass; out_prim = sample 0's hit. */
int orc_render_pass_ms(const orc_scene* s, const double cam[10], int W, int H, int mapping, double k, double f,
                       double z0, int spp, const float* jitter, const float* in_rgbz, const double* in_normal,
                       const int64_t* pix, int64_t npix, double* out_rgbz, double* out_normal, int32_t* out_prim,
                       uint8_t* out_flag, int nthreads);
/* K multi-sample passes from I_0 over the whole image (W*H*4 doubles out;
 * out_normal W*H*3, nullable). */
int orc_render_ms(const orc_scene* s, const double cam[10], int W, int H, int K, int mapping, double k, double f,
                  double z0, int spp, const float* jitter, double* out_rgbz, double* out_normal, uint8_t* out_flag,
                  int nthreads);

/* Image-space pass (§6: with V_e = 0 a pass reduces to re-sampling the
 * rendered image at a displaced pixel; §6.1: mirrored screen edges). base = the
 * frame's rendered image (H*W*4), prev = I_{n-1} (H*W*4), both float32,
 * widened exactly. For pixel (x, y) with previous colour c, in double:
 *   sx = x + k_px * (2 c.r - 1),  sy = y - k_px * (2 c.g - 1)  (R right, G up: Eq. 5)
 * the sample is the nearest pixel (floor(s + 1/2)) to (sx, sy), reflected into
 * the image without repeating the edge pixel (-1 -> 0, W -> W-1, repeatedly),
 * and I_n(x, y) = base at that pixel (all four lanes).
 * out_flag (nullable) = 1 where sx or sy lies within ORC_IMG_TOL * (|x| or |y|
 * + k_px + 1) of a rounding boundary (a half-integer): there a renderer that
 * evaluates the displacement in float32 may take the neighbouring pixel.
 * Writes npix*4 floats to out (pix = NULL: every pixel). */
#define ORC_IMG_TOL 4.76837158203125e-07 /* 2^-21 */
int orc_imagespace_pass(const float* base, const float* prev, int W, int H, double k_px, const int64_t* pix,
                        int64_t npix, float* out, uint8_t* out_flag);
/* The reflection of an integer pixel index into [0, n). */
int64_t orc_mirror_index(int64_t i, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
