/*
 * rcp_oracle.c -- FP64 brute-force CPU oracle for Recursive Camera Painting
 * (arXiv 2312.12392). TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke
 * check and the benchmark's CPU-baseline leg, never by the CUDA library.
 *
 * Plain C99 + pthreads. Every function states the passage it follows; the
 * paper's notation is kept (P_e eye, P_p texture-coordinate point, V_e / V_p
 * displacements, lambda = k, I_n images). Where the paper is silent the chosen
 * reading is stated at the function.
 */
#include "rcp_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

struct orc_scene {
    int64_t T, S;
    double* v;      /* T*9: v0 v1 v2, exact copies of the float input */
    double* n;      /* T*3: unnormalised geometric normal (v1-v0) x (v2-v0) */
    double* rad;    /* T: largest vertex distance from the centroid */
    double* sph;    /* S*4 */
    double* albedo; /* (T+S)*3 */
    int light_type;
    double light[3];
    double ambient;
    double diam;
};

/* ---------------------------------------------------------------- vectors */

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double a[3], const double b[3], double r[3]) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static void cross3(const double a[3], const double b[3], double r[3]) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    r[0] = x; r[1] = y; r[2] = z;
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void normalize3(double a[3]) { double l = norm3(a); a[0] /= l; a[1] /= l; a[2] /= l; }

/* ---------------------------------------------------------------- scene */

orc_scene* orc_scene_new(const float* tri, int64_t T, const float* sph, int64_t S,
                         const float* albedo, int light_type, const double light[3],
                         double ambient) {
    if (T < 0 || S < 0 || (T > 0 && !tri) || (S > 0 && !sph) || (T + S > 0 && !albedo) || !light)
        return NULL;
    if (light_type != ORC_LIGHT_POINT && light_type != ORC_LIGHT_DIRECTIONAL) return NULL;
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    if (!s) return NULL;
    s->T = T;
    s->S = S;
    s->v = (double*)malloc(sizeof(double) * (size_t)(T * 9 + 1));
    s->n = (double*)malloc(sizeof(double) * (size_t)(T * 3 + 1));
    s->rad = (double*)malloc(sizeof(double) * (size_t)(T + 1));
    s->sph = (double*)malloc(sizeof(double) * (size_t)(S * 4 + 1));
    s->albedo = (double*)malloc(sizeof(double) * (size_t)((T + S) * 3 + 1));
    if (!s->v || !s->n || !s->rad || !s->sph || !s->albedo) { orc_scene_free(s); return NULL; }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < T * 9; ++i) s->v[i] = (double)tri[i];
    for (int64_t i = 0; i < T; ++i) {
        const double* v = s->v + 9 * i;
        double e1[3], e2[3];
        sub3(v + 3, v, e1);
        sub3(v + 6, v, e2);
        cross3(e1, e2, s->n + 3 * i);
        double cen[3] = {(v[0] + v[3] + v[6]) / 3, (v[1] + v[4] + v[7]) / 3, (v[2] + v[5] + v[8]) / 3};
        s->rad[i] = 0.0;
        for (int j = 0; j < 3; ++j) {
            double w[3];
            sub3(v + 3 * j, cen, w);
            if (norm3(w) > s->rad[i]) s->rad[i] = norm3(w);
        }
        s->rad[i] *= 1.0 + 1e-12;
        for (int j = 0; j < 3; ++j)
            for (int a = 0; a < 3; ++a) {
                if (v[3 * j + a] < lo[a]) lo[a] = v[3 * j + a];
                if (v[3 * j + a] > hi[a]) hi[a] = v[3 * j + a];
            }
    }
    for (int64_t i = 0; i < S * 4; ++i) s->sph[i] = (double)sph[i];
    for (int64_t i = 0; i < S; ++i) {
        const double* c = s->sph + 4 * i;
        for (int a = 0; a < 3; ++a) {
            if (c[a] - c[3] < lo[a]) lo[a] = c[a] - c[3];
            if (c[a] + c[3] > hi[a]) hi[a] = c[a] + c[3];
        }
    }
    for (int64_t i = 0; i < (T + S) * 3; ++i) s->albedo[i] = (double)albedo[i];
    s->light_type = light_type;
    memcpy(s->light, light, sizeof(double) * 3);
    if (light_type == ORC_LIGHT_DIRECTIONAL) {
        if (norm3(s->light) == 0.0) { orc_scene_free(s); return NULL; }
        normalize3(s->light);
    }
    s->ambient = ambient;
    if (T + S > 0) {
        double d[3];
        sub3(hi, lo, d);
        s->diam = norm3(d);
    } else {
        s->diam = 0.0;
    }
    return s;
}

void orc_scene_free(orc_scene* s) {
    if (!s) return;
    free(s->v);
    free(s->n);
    free(s->rad);
    free(s->sph);
    free(s->albedo);
    free(s);
}

double orc_scene_diam(const orc_scene* s) { return s ? s->diam : 0.0; }

/* ---------------------------------------------------------------- camera */

/*
 * Per-pixel camera: §2 (Eq. 2-4) and §3 (Eq. 5).
 *
 * Base pinhole frame (reading: right-handed, +R screen-right, +U screen-up, so
 * that red moves a pixel right and green moves it up, as §3 states): F = normalize(look_at -
 * eye), R = normalize(F x up), U = R x F. Pixel (x, y) is sampled at its centre
 * (u, v) = ((x+.5)/W, (y+.5)/H), row 0 at the top. P_p is the pixel's point on
 * the focal plane at distance f along F (reading of §2's 3D point of the
 * texture coordinate (u,v)):
 *     P_p = P_e + f * (F + (2u-1) tan(fov/2) (W/H) R + (1-2v) tan(fov/2) U).
 * The colour mapping of Eq. 5, with (R, G, B) along (right, up, forward):
 *     V = k * ((2r-1) R + (2g-1) U + (2b-1) F).
 * EYE:    P'_e = P_e + V, P'_p = P_p       (V_e = V, V_p = 0; Eq. 3-4, whose
 *                                          first line the paper prints as P'_p)
 * TARGET: P'_e = P_e,     P'_p = P_p + V   (V_e = 0; §3's example)
 * DEPTH:  P'_e = P_e,     P'_p = P_p + |z - z0| V   (§4, Eq. 7)
 * NORMAL: P'_e = P_e,     P'_p = P_p + k (C x N)    (§5, Eq. 8), C = the unit
 *         pinhole direction (P_p - P_e)/|P_p - P_e|, N = the previous normal
 * Ray: origin P'_e, direction (P'_p - P'_e) / |P'_p - P'_e|   (Eq. 2).
 */
int orc_camera_ray(const double cam[10], int W, int H, int x, int y, int mapping,
                   double k, double f, double z0, const double c[3], double z, const double nrm[3],
                   double o[3], double d[3]) {
    return orc_camera_ray_at(cam, W, H, (double)x + 0.5, (double)y + 0.5, mapping, k, f, z0, c, z, nrm, o, d);
}

/* The same camera for a sample at pixel coordinates (px, py): (u, v) =
 * (px/W, py/H); the pixel centre is (x + 0.5, y + 0.5) (§2 allows any number
 * of jittered samples per pixel). */
int orc_camera_ray_at(const double cam[10], int W, int H, double px, double py, int mapping,
                      double k, double f, double z0, const double c[3], double z, const double nrm[3],
                      double o[3], double d[3]) {
    const double* Pe = cam;
    double F[3], R[3], U[3];
    sub3(cam + 3, cam, F);
    normalize3(F);
    cross3(F, cam + 6, R);
    normalize3(R);
    cross3(R, F, U);
    const double tn = tan(cam[9] * M_PI / 360.0);
    const double aspect = (double)W / (double)H;
    const double u = px / (double)W;
    const double v = py / (double)H;
    const double sx = (2.0 * u - 1.0) * tn * aspect;
    const double sy = (1.0 - 2.0 * v) * tn;
    double Pp[3], V[3], Pe2[3], Pp2[3];
    for (int a = 0; a < 3; ++a) Pp[a] = Pe[a] + f * (F[a] + sx * R[a] + sy * U[a]);
    const double dr = 2.0 * c[0] - 1.0, dg = 2.0 * c[1] - 1.0, db = 2.0 * c[2] - 1.0;
    for (int a = 0; a < 3; ++a) V[a] = k * (dr * R[a] + dg * U[a] + db * F[a]);
    if (mapping == ORC_MAP_NORMAL) {
        /* §5, Eq. 8: V_p = k (C x N), C the undisplaced pinhole direction and
           N the previous pass's hit normal (none: no displacement) */
        double N[3] = {0.0, 0.0, 0.0}, C[3], X[3];
        if (nrm) memcpy(N, nrm, sizeof(N));
        sub3(Pp, Pe, C);
        normalize3(C);
        cross3(C, N, X);
        for (int a = 0; a < 3; ++a) V[a] = k * X[a];
    }
    if (mapping == ORC_MAP_EYE) {
        for (int a = 0; a < 3; ++a) { Pe2[a] = Pe[a] + V[a]; Pp2[a] = Pp[a]; }
    } else if (mapping == ORC_MAP_TARGET || mapping == ORC_MAP_NORMAL) {
        for (int a = 0; a < 3; ++a) { Pe2[a] = Pe[a]; Pp2[a] = Pp[a] + V[a]; }
    } else {
        const double m = fabs(z - z0);
        for (int a = 0; a < 3; ++a) { Pe2[a] = Pe[a]; Pp2[a] = Pp[a] + m * V[a]; }
    }
    double N[3];
    sub3(Pp2, Pe2, N);
    double len = norm3(N);
    memcpy(o, Pe2, sizeof(double) * 3);
    if (len == 0.0) {
        memcpy(d, F, sizeof(double) * 3);
        return 1;
    }
    for (int a = 0; a < 3; ++a) d[a] = N[a] / len;
    return 0;
}

/* ---------------------------------------------------------------- primitives */

/* Unclipped Moller-Trumbore: returns 1 if the ray's line meets the triangle's
 * plane inside the closed triangle (u >= 0, v >= 0, u + v <= 1), writing t (any
 * sign). A degenerate triangle (zero normal) or a ray parallel to the plane
 * (det == 0) gives 0. */
static int mt_raw(const double* v, const double* n, const double o[3], const double d[3], double* t) {
    if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) return 0;
    double e1[3], e2[3], P[3], Tv[3], Q[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(d, e2, P);
    const double det = dot3(e1, P);
    if (det == 0.0) return 0;
    const double inv = 1.0 / det;
    sub3(o, v, Tv);
    const double uu = dot3(Tv, P) * inv;
    cross3(Tv, e1, Q);
    const double vv = dot3(d, Q) * inv;
    *t = dot3(e2, Q) * inv;
    return uu >= 0.0 && vv >= 0.0 && uu + vv <= 1.0;
}

int orc_hit_triangle(const double v0[3], const double v1[3], const double v2[3],
                     const double o[3], const double d[3], double tmin, double tmax, double* t) {
    double v[9], e1[3], e2[3], n[3], tt;
    memcpy(v, v0, 24); memcpy(v + 3, v1, 24); memcpy(v + 6, v2, 24);
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    if (mt_raw(v, n, o, d, &tt) && tt > tmin && tt < tmax) { *t = tt; return 1; }
    return 0;
}

/* Analytic ray-sphere (d unit): the roots of |o + t d - c| = r, taken as
 * -b -/+ sqrt(r^2 - |oc - b d|^2) with oc = o - c, b = oc . d; the nearer root
 * inside (tmin, tmax), else the farther one. */
static int sphere_roots(const double* s, const double o[3], const double d[3], double* t0, double* t1,
                        double* perp_len) {
    double oc[3], perp[3];
    sub3(o, s, oc);
    const double b = dot3(oc, d);
    for (int a = 0; a < 3; ++a) perp[a] = oc[a] - b * d[a];
    const double p2 = dot3(perp, perp);
    *perp_len = sqrt(p2);
    const double disc = s[3] * s[3] - p2;
    if (disc < 0.0) return 0;
    const double q = sqrt(disc);
    *t0 = -b - q;
    *t1 = -b + q;
    return 1;
}

int orc_hit_sphere(const double c[3], double r, const double o[3], const double d[3],
                   double tmin, double tmax, double* t) {
    double s[4] = {c[0], c[1], c[2], r}, t0, t1, pl;
    if (!sphere_roots(s, o, d, &t0, &t1, &pl)) return 0;
    if (t0 > tmin && t0 < tmax) { *t = t0; return 1; }
    if (t1 > tmin && t1 < tmax) { *t = t1; return 1; }
    return 0;
}

/* Geometric unit normal at a hit (triangle: normalised (v1-v0)x(v2-v0); sphere:
 * (p - c)/r), flipped to face the ray (two-sided surfaces). */
static void hit_normal(const orc_scene* s, int64_t id, const double p[3], const double d[3], double N[3]) {
    if (id < s->T) {
        memcpy(N, s->n + 3 * id, 24);
        normalize3(N);
    } else {
        const double* c = s->sph + 4 * (id - s->T);
        for (int a = 0; a < 3; ++a) N[a] = (p[a] - c[a]) / c[3];
    }
    if (dot3(N, d) > 0.0) { N[0] = -N[0]; N[1] = -N[1]; N[2] = -N[2]; }
}

/* ---------------------------------------------------------------- ambiguity */

/*
 * The GPU traces in float32, so rays within a rounding error of a decision
 * boundary may legitimately resolve differently from this oracle. Such rays are
 * flagged. A decision is ambiguous when the ray passes within
 *     band = ORC_TOL * (t + |o| + extra)
 * of it, measured perpendicular to the ray (float32 rounding of the ray scales
 * with the ray's length and the magnitude of its origin). The boundaries are:
 * a triangle's edges (distance from the ray to the triangle's outline in the
 * plane perpendicular to d), a sphere's silhouette (| |oc x d| - r |), the ends
 * of the t interval, and two surfaces hit at nearly the same depth.
 */

static double band_at(double t, double onorm, double extra) { return ORC_TOL * (fabs(t) + onorm + extra); }

/* Does the ray pass within the band of triangle v's outline at a depth in
 * [lo - band, hi + band]? The distance is taken in the plane perpendicular to
 * unit d; the depth is that of the outline point nearest to the ray. `rad` is
 * the triangle's radius about its centroid (an exact early-out: a triangle whose
 * bounding sphere stays farther than the band from the ray cannot be near). */
static int outline_near(const double* v, double rad, const double o[3], const double d[3],
                        double onorm, double extra, double lo, double hi) {
    double cen[3] = {(v[0] + v[3] + v[6]) / 3, (v[1] + v[4] + v[7]) / 3, (v[2] + v[5] + v[8]) / 3};
    double w[3];
    sub3(cen, o, w);
    const double cd = dot3(w, d);
    double perp2 = dot3(w, w) - cd * cd;
    if (perp2 < 0.0) perp2 = 0.0;
    const double reach = rad + band_at(fabs(cd) + rad, onorm, extra);
    if (sqrt(perp2) > reach) return 0;
    if (cd + rad < lo - band_at(fabs(cd) + rad, onorm, extra)) return 0;
    if (cd - rad > hi + band_at(fabs(cd) + rad, onorm, extra)) return 0;
    double a[3], b[3], ax[3] = {1, 0, 0};
    if (fabs(d[0]) > 0.5) { ax[0] = 0; ax[1] = 1; }
    cross3(d, ax, a);
    normalize3(a);
    cross3(d, a, b);
    double q[3][3];
    for (int j = 0; j < 3; ++j) {
        sub3(v + 3 * j, o, w);
        q[j][0] = dot3(w, a);
        q[j][1] = dot3(w, b);
        q[j][2] = dot3(w, d);
    }
    for (int j = 0; j < 3; ++j) {
        const double* p0 = q[j];
        const double* p1 = q[(j + 1) % 3];
        const double wx = p1[0] - p0[0], wy = p1[1] - p0[1];
        const double ww = wx * wx + wy * wy;
        double tt = 0.0;
        if (ww > 0.0) {
            tt = -(p0[0] * wx + p0[1] * wy) / ww;
            if (tt < 0.0) tt = 0.0;
            if (tt > 1.0) tt = 1.0;
        }
        const double px = p0[0] + tt * wx, py = p0[1] + tt * wy;
        const double depth = p0[2] + tt * (p1[2] - p0[2]);
        const double bd = band_at(depth, onorm, extra);
        if (sqrt(px * px + py * py) <= bd && depth >= lo - bd && depth <= hi + bd) return 1;
    }
    return 0;
}

/* |cos| of the angle between the ray and the surface normal at a hit, floored
 * at 1e-3 so a grazing hit widens the depth band by at most 1000x. */
static double hit_cos(const orc_scene* s, int64_t id, const double o[3], const double d[3], double t) {
    double p[3], N[3];
    for (int a = 0; a < 3; ++a) p[a] = o[a] + t * d[a];
    hit_normal(s, id, p, d, N);
    double c = fabs(dot3(N, d));
    return c < 1e-3 ? 1e-3 : c;
}

/* ---------------------------------------------------------------- tracing */

/*
 * Closest hit (the rays of §3's second stage): every primitive is tested and
 * the smallest t in (tmin, tmax) wins; equal t goes to the lower id (reading:
 * the paper has no tie rule). Triangles have ids 0..T-1, spheres T..T+S-1.
 */
int orc_trace_closest(const orc_scene* s, const double o[3], const double d[3],
                      double tmin, double tmax, double* t_out, int64_t* prim, int* flag) {
    double best = tmax;
    int64_t best_id = -1;
    for (int64_t i = 0; i < s->T; ++i) {
        double t;
        if (mt_raw(s->v + 9 * i, s->n + 3 * i, o, d, &t) && t > tmin && t < best) { best = t; best_id = i; }
    }
    for (int64_t j = 0; j < s->S; ++j) {
        double t0, t1, pl;
        const double* sp = s->sph + 4 * j;
        if (!sphere_roots(sp, o, d, &t0, &t1, &pl)) continue;
        double t = (t0 > tmin) ? t0 : t1;
        if (t > tmin && t < best) { best = t; best_id = s->T + j; }
    }
    *t_out = best_id >= 0 ? best : INFINITY;
    *prim = best_id;

    /* ambiguity: outlines and silhouettes in front of (or at) the hit, hits at
     * the t_min end, and other surfaces within the depth band of the hit */
    const double on = norm3(o);
    const double tb = best_id >= 0 ? best : tmax;
    const double cos_b = best_id >= 0 ? hit_cos(s, best_id, o, d, best) : 1.0;
    const double band_b = band_at(best_id >= 0 ? best : 0.0, on, 0.0);
    int amb = 0;
    for (int64_t i = 0; i < s->T && !amb; ++i) {
        const double* v = s->v + 9 * i;
        const double* n = s->n + 3 * i;
        if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) continue;
        if (outline_near(v, s->rad[i], o, d, on, 0.0, tmin, tb)) { amb = 1; break; }
        double t;
        if (!mt_raw(v, n, o, d, &t)) continue;
        const double cz = hit_cos(s, i, o, d, t);
        if (fabs(t - tmin) <= band_at(t, on, 0.0) / cz) { amb = 1; break; }
        if (best_id >= 0 && i != best_id && t > tmin && t - tb <= band_b * (1.0 / cos_b + 1.0 / cz)) {
            amb = 1;
            break;
        }
    }
    for (int64_t j = 0; j < s->S && !amb; ++j) {
        double t0, t1, pl;
        const double* sp = s->sph + 4 * j;
        double oc[3];
        sub3(o, sp, oc);
        const double tca = -dot3(oc, d);
        const double bc = band_at(tca, on, 0.0);
        const int real = sphere_roots(sp, o, d, &t0, &t1, &pl);
        if (fabs(pl - sp[3]) <= bc && tca >= tmin - bc && tca <= tb + bc) { amb = 1; break; }
        if (!real) continue;
        const double ts[2] = {t0, t1};
        for (int r = 0; r < 2; ++r) {
            const double cz = hit_cos(s, s->T + j, o, d, ts[r]);
            if (fabs(ts[r] - tmin) <= band_at(ts[r], on, 0.0) / cz) amb = 1;
            if (best_id >= 0 && s->T + j != best_id && ts[r] > tmin &&
                ts[r] - tb <= band_b * (1.0 / cos_b + 1.0 / cz)) amb = 1;
        }
    }
    int fl = amb ? ORC_FLAG_ID : 0;
    /* The hit point of the best primitive itself: a sphere hit near its
     * silhouette (the two roots nearly meet) or with a root near t_min (the
     * near and far roots may swap) is ill-conditioned, so even the same sphere
     * may be hit at another point and shaded differently. */
    if (best_id >= s->T) {
        const double* sp = s->sph + 4 * (best_id - s->T);
        double t0, t1, pl, oc[3];
        sub3(o, sp, oc);
        const double bc = band_at(-dot3(oc, d), on, 0.0);
        sphere_roots(sp, o, d, &t0, &t1, &pl);
        int ill = fabs(pl - sp[3]) <= bc;
        const double ts[2] = {t0, t1};
        for (int r = 0; r < 2; ++r)
            if (fabs(ts[r] - tmin) <= band_at(ts[r], on, 0.0) / hit_cos(s, best_id, o, d, ts[r])) ill = 1;
        if (ill) fl |= ORC_FLAG_ID | ORC_FLAG_POINT;
    }
    *flag = fl;
    return 0;
}

/*
 * Any hit in (tmin, tmax) (the shadow ray). A hit well inside a primitive and
 * well inside the interval decides "occluded" on its own; otherwise the answer
 * is flagged when any primitive lies within the band of a boundary.
 */
int orc_trace_any(const orc_scene* s, const double o[3], const double d[3], double tmin,
                  double tmax, double extra, int* occluded, int* flag) {
    const double on = norm3(o);
    int occ = 0, robust = 0, amb = 0;
    for (int64_t i = 0; i < s->T && !robust; ++i) {
        const double* v = s->v + 9 * i;
        const double* n = s->n + 3 * i;
        if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) continue;
        double t;
        const int inside = mt_raw(v, n, o, d, &t);
        const int near_edge = outline_near(v, s->rad[i], o, d, on, extra, tmin, tmax);
        if (inside) {
            const double bt = band_at(t, on, extra) / hit_cos(s, i, o, d, t);
            const int near_end = fabs(t - tmin) <= bt || fabs(t - tmax) <= bt;
            if (t > tmin && t < tmax) {
                occ = 1;
                if (!near_edge && !near_end) robust = 1;
            }
            if (near_end) amb = 1;
        }
        if (near_edge) amb = 1;
    }
    for (int64_t j = 0; j < s->S && !robust; ++j) {
        double t0, t1, pl;
        const double* sp = s->sph + 4 * j;
        double oc[3];
        sub3(o, sp, oc);
        const double tca = -dot3(oc, d);
        const double bc = band_at(tca, on, extra);
        const int real = sphere_roots(sp, o, d, &t0, &t1, &pl);
        const int near_sil = fabs(pl - sp[3]) <= bc && tca >= tmin - bc && tca <= tmax + bc;
        if (near_sil) amb = 1;
        if (!real) continue;
        const double ts[2] = {t0, t1};
        for (int r = 0; r < 2; ++r) {
            const double bt = band_at(ts[r], on, extra) / hit_cos(s, s->T + j, o, d, ts[r]);
            const int near_end = fabs(ts[r] - tmin) <= bt || fabs(ts[r] - tmax) <= bt;
            if (ts[r] > tmin && ts[r] < tmax) {
                occ = 1;
                if (!near_end && !near_sil) robust = 1;
            }
            if (near_end) amb = 1;
        }
    }
    *occluded = occ;
    *flag = robust ? 0 : amb;
    return 0;
}

/* ---------------------------------------------------------------- shading */

/*
 * Render one primary ray (§2 stage 2, the new image of the pass). The paper does
 * not state a shading model; the reading used here:
 *  - hit: c = albedo * (a + (1 - a) * V * max(0, N . L)), with ambient a, a
 *    white light of intensity 1 and no distance falloff; V = 1 unless the
 *    shadow ray is blocked. N faces the ray. L points from the hit point p to
 *    the light (point) or is the given direction (directional). The shadow ray
 *    is only cast when N . L > 0; it starts at p + eps N (eps = 1e-4 * diam)
 *    and runs over (0, |light - (p + eps N)|) (point) or (0, inf).
 *  - miss: sky(d) = (1 - s) (1,1,1) + s (0.5, 0.7, 1.0), s = (d_y + 1) / 2.
 *  - each channel clamped to [0, 1] (the paper's low-dynamic-range images, §3).
 * rgbz[3] = hit distance along d, or -1 on a miss; nrm (nullable) = the unit
 * normal N facing the ray (zero on a miss).
 */
int orc_shade_ray(const orc_scene* s, const double o[3], const double d[3], double rgbz[4], double nrm[3],
                  int64_t* prim, int* flag) {
    const double tmin = 1e-6 * s->diam;
    const double eps = 1e-4 * s->diam;
    double t;
    int64_t id;
    int amb = 0;
    orc_trace_closest(s, o, d, tmin, INFINITY, &t, &id, &amb);
    *prim = id;
    if (nrm) nrm[0] = nrm[1] = nrm[2] = 0.0;
    if (id < 0) {
        const double sv = 0.5 * (d[1] + 1.0);
        rgbz[0] = (1.0 - sv) + sv * 0.5;
        rgbz[1] = (1.0 - sv) + sv * 0.7;
        rgbz[2] = (1.0 - sv) + sv * 1.0;
        rgbz[3] = -1.0;
    } else {
        double p[3], N[3], L[3];
        for (int a = 0; a < 3; ++a) p[a] = o[a] + t * d[a];
        hit_normal(s, id, p, d, N);
        if (nrm) memcpy(nrm, N, sizeof(N));
        if (s->light_type == ORC_LIGHT_POINT) {
            sub3(s->light, p, L);
            normalize3(L);
        } else {
            memcpy(L, s->light, 24);
        }
        const double ndl = dot3(N, L);
        double vis = 1.0;
        if (ndl > 0.0) {
            double ps[3], ls[3], tmax = INFINITY;
            for (int a = 0; a < 3; ++a) ps[a] = p[a] + eps * N[a];
            if (s->light_type == ORC_LIGHT_POINT) {
                sub3(s->light, ps, ls);
                tmax = norm3(ls);
                for (int a = 0; a < 3; ++a) ls[a] /= tmax;
            } else {
                memcpy(ls, s->light, 24);
            }
            int occ = 0, samb = 0;
            orc_trace_any(s, ps, ls, 0.0, tmax, t + norm3(o), &occ, &samb);
            vis = occ ? 0.0 : 1.0;
            if (samb) amb |= ORC_FLAG_SHADOW;
        }
        const double lam = ndl > 0.0 ? ndl : 0.0;
        const double* alb = s->albedo + 3 * id;
        for (int a = 0; a < 3; ++a) rgbz[a] = alb[a] * (s->ambient + (1.0 - s->ambient) * vis * lam);
        rgbz[3] = t;
    }
    for (int a = 0; a < 3; ++a) rgbz[a] = rgbz[a] < 0.0 ? 0.0 : (rgbz[a] > 1.0 ? 1.0 : rgbz[a]);
    *flag = amb;
    return 0;
}

/* ---------------------------------------------------------------- passes */

typedef struct {
    const orc_scene* s;
    const double* cam;
    int W, H, K, mapping;
    double k, f, z0;
    const float* in;       /* previous image (float32 H*W*4), NULL = I_0 */
    const double* in_d;    /* previous image in double (multi-sample chains) */
    const double* in_n;    /* previous hit normals (H*W*3), NULL = none */
    int spp;               /* samples per pixel, 0 = one at the centre */
    const float* jitter;   /* spp (dx, dy) offsets inside the pixel */
    const int64_t* pix;
    int64_t npix;
    double* out;
    double* out_n;
    int32_t* prim;
    uint8_t* flag;
    int64_t next, chunk;
    pthread_mutex_t mu;
} job_t;

/* Unit view axis F = (look_at - eye)/|look_at - eye| of the base camera. */
static void camera_forward(const double cam[10], double F[3]) {
    sub3(cam + 3, cam, F);
    normalize3(F);
}

/*
 * z-depth of a primary hit (reading of §4 and §6: "z-depth" is depth along the
 * camera's view axis, as a game engine's scene depth is): the hit point's
 * distance from the pixel's eye measured along the base camera's forward axis
 * F, z = t (d . F); 0 on a miss.
 */
static double z_depth(const double d[3], const double F[3], int64_t id, double t) {
    return id < 0 ? 0.0 : t * dot3(d, F);
}

/*
 * The previous image seen by a sample at pixel coordinates (px, py): bilinear
 * between the four nearest pixel centres, indices clamped at the edges (§2's
 * (u,v) need not sit on a pixel centre). in_f or in_d (float or double H*W*4
 * image); both NULL = I_0.
 */
static void sample_prev(const float* in_f, const double* in_d, int W, int H, double px, double py, double c[4]) {
    if (!in_f && !in_d) {
        c[0] = c[1] = c[2] = 0.5;
        c[3] = 0.0;
        return;
    }
    const double qx = px - 0.5, qy = py - 0.5;
    const double fx0 = floor(qx), fy0 = floor(qy);
    const double wx = qx - fx0, wy = qy - fy0;
    int64_t xs[2] = {(int64_t)fx0, (int64_t)fx0 + 1}, ys[2] = {(int64_t)fy0, (int64_t)fy0 + 1};
    for (int j = 0; j < 2; ++j) {
        xs[j] = xs[j] < 0 ? 0 : (xs[j] >= W ? W - 1 : xs[j]);
        ys[j] = ys[j] < 0 ? 0 : (ys[j] >= H ? H - 1 : ys[j]);
    }
    const double w[2][2] = {{(1.0 - wx) * (1.0 - wy), wx * (1.0 - wy)}, {(1.0 - wx) * wy, wx * wy}};
    for (int a = 0; a < 4; ++a) {
        double acc = 0.0;
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 2; ++q) {
                const int64_t idx = 4 * (ys[r] * W + xs[q]) + a;
                acc += w[r][q] * (in_f ? (double)in_f[idx] : in_d[idx]);
            }
        c[a] = acc;
    }
}

/* The pixel whose centre is nearest to (px, py), clamped to the image: a
 * normal is a direction, not a quantity to blend, so a sample takes its
 * nearest pixel's. */
int64_t orc_nearest_pixel(int W, int H, double px, double py) {
    int64_t nx = (int64_t)floor(px), ny = (int64_t)floor(py);
    nx = nx < 0 ? 0 : (nx >= W ? W - 1 : nx);
    ny = ny < 0 ? 0 : (ny >= H ? H - 1 : ny);
    return ny * W + nx;
}

int orc_sample_image(const float* in, int W, int H, double px, double py, double c[4]) {
    if (!in || W < 1 || H < 1) return -1;
    sample_prev(in, NULL, W, H, px, py, c);
    return 0;
}

/* One pass of one pixel with J->spp jittered samples: each sample reads I_{n-1}
 * at its own (u,v), gets its own camera and is traced and shaded; the pixel is
 * the mean of its samples (colour and depth; the normal is sample 0's).
 * Reading: §2's anti-aliasing samples are averaged. */
static void run_pixel_ms(const job_t* J, int64_t i) {
    const int64_t p = J->pix ? J->pix[i] : i;
    const int x = (int)(p % J->W), y = (int)(p / J->W);
    double F[3];
    camera_forward(J->cam, F);
    double acc[4] = {0, 0, 0, 0}, n0[3] = {0, 0, 0};
    uint8_t fl = 0;
    int64_t id0 = -1;
    for (int s = 0; s < J->spp; ++s) {
        const double px = (double)x + (double)J->jitter[2 * s], py = (double)y + (double)J->jitter[2 * s + 1];
        double c[4], o[3], d[3], rgbt[4], ns[3];
        const double* nin = J->in_n ? J->in_n + 3 * orc_nearest_pixel(J->W, J->H, px, py) : NULL;
        sample_prev(J->in, J->in_d, J->W, J->H, px, py, c);
        int amb = 0;
        int64_t id = -1;
        if (orc_camera_ray_at(J->cam, J->W, J->H, px, py, J->mapping, J->k, J->f, J->z0, c, c[3], nin, o, d))
            fl |= ORC_FLAG_ID | ORC_FLAG_POINT;
        orc_shade_ray(J->s, o, d, rgbt, ns, &id, &amb);
        fl |= (uint8_t)amb;
        for (int a = 0; a < 3; ++a) acc[a] += rgbt[a];
        acc[3] += z_depth(d, F, id, rgbt[3]);
        if (s == 0) {
            id0 = id;
            memcpy(n0, ns, sizeof(n0));
        }
    }
    for (int a = 0; a < 4; ++a) J->out[4 * i + a] = acc[a] / (double)J->spp;
    if (J->out_n) memcpy(J->out_n + 3 * i, n0, sizeof(n0));
    if (J->prim) J->prim[i] = (int32_t)id0;
    if (J->flag) J->flag[i] = fl;
}

/* One pixel's chain of `passes` passes starting from I_{n-1} = (c, nrm):
 * colour and z-depth in c, the hit normal in nrm. */
static void run_pixel(const job_t* J, int64_t i, double c[4], double nrm[3], int passes) {
    const int64_t p = J->pix ? J->pix[i] : i;
    const int x = (int)(p % J->W), y = (int)(p / J->W);
    double F[3];
    camera_forward(J->cam, F);
    uint8_t fl = 0;
    int64_t id = -1;
    for (int n = 0; n < passes; ++n) {
        double o[3], d[3], rgbt[4];
        int amb = 0;
        if (orc_camera_ray(J->cam, J->W, J->H, x, y, J->mapping, J->k, J->f, J->z0, c, c[3], nrm, o, d))
            fl |= ORC_FLAG_ID | ORC_FLAG_POINT;
        orc_shade_ray(J->s, o, d, rgbt, nrm, &id, &amb);
        fl |= (uint8_t)amb;
        memcpy(c, rgbt, sizeof(double) * 3);
        c[3] = z_depth(d, F, id, rgbt[3]);
    }
    memcpy(J->out + 4 * i, c, sizeof(double) * 4);
    if (J->out_n) memcpy(J->out_n + 3 * i, nrm, sizeof(double) * 3);
    if (J->prim) J->prim[i] = (int32_t)id;
    if (J->flag) J->flag[i] = fl;
}

static void* worker(void* arg) {
    job_t* J = (job_t*)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i0 = J->next;
        J->next += J->chunk;
        pthread_mutex_unlock(&J->mu);
        if (i0 >= J->npix) break;
        int64_t i1 = i0 + J->chunk < J->npix ? i0 + J->chunk : J->npix;
        if (J->spp > 0) {
            for (int64_t i = i0; i < i1; ++i) run_pixel_ms(J, i);
            continue;
        }
        for (int64_t i = i0; i < i1; ++i) {
            const int64_t p = J->pix ? J->pix[i] : i;
            double c[4] = {0.5, 0.5, 0.5, 0.0}, nrm[3] = {0.0, 0.0, 0.0};
            if (J->in)
                for (int a = 0; a < 4; ++a) c[a] = (double)J->in[4 * p + a];
            if (J->in_n) memcpy(nrm, J->in_n + 3 * p, sizeof(nrm));
            run_pixel(J, i, c, nrm, J->K);
        }
    }
    return NULL;
}

static int run_job(job_t* J, int nthreads) {
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    pthread_mutex_init(&J->mu, NULL);
    J->next = 0;
    /* pixels per claim: up to 64, but small enough that every thread gets
       several claims when the sample is small */
    J->chunk = J->npix / (8 * (int64_t)nthreads);
    if (J->chunk > 64) J->chunk = 64;
    if (J->chunk < 1) J->chunk = 1;
    int started = 0;
    for (int i = 0; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, worker, J) == 0) ++started;
    if (started == 0) worker(J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J->mu);
    return 0;
}

static int check_common(const orc_scene* s, const double* cam, int W, int H, int mapping, double k, double f) {
    if (!s || !cam || W < 1 || H < 1 || k < 0.0 || !(f > 0.0)) return -1;
    if (mapping != ORC_MAP_EYE && mapping != ORC_MAP_TARGET && mapping != ORC_MAP_DEPTH && mapping != ORC_MAP_NORMAL)
        return -1;
    return 0;
}

static int check_pix(const int64_t* pix, int64_t npix, int W, int H) {
    for (int64_t i = 0; pix && i < npix; ++i)
        if (pix[i] < 0 || pix[i] >= (int64_t)W * H) return -1;
    return 0;
}

int orc_render_pass(const orc_scene* s, const double cam[10], int W, int H, int mapping,
                    double k, double f, double z0, const float* in_rgbz, const double* in_normal,
                    const int64_t* pix, int64_t npix, double* out_rgbz, double* out_normal,
                    int32_t* out_prim, uint8_t* out_flag, int nthreads) {
    if (check_common(s, cam, W, H, mapping, k, f) || !out_rgbz) return -1;
    if (!pix) npix = (int64_t)W * H;
    if (check_pix(pix, npix, W, H)) return -1;
    job_t J;
    memset(&J, 0, sizeof(J));
    J.s = s; J.cam = cam; J.W = W; J.H = H; J.K = 1; J.mapping = mapping; J.k = k; J.f = f; J.z0 = z0;
    J.in = in_rgbz; J.in_n = in_normal; J.pix = pix; J.npix = npix; J.out = out_rgbz; J.out_n = out_normal;
    J.prim = out_prim; J.flag = out_flag;
    return run_job(&J, nthreads);
}

int orc_render(const orc_scene* s, const double cam[10], int W, int H, int K, int mapping,
               double k, double f, double z0, const int64_t* pix, int64_t npix,
               double* out_rgbz, double* out_normal, int32_t* out_prim, uint8_t* out_flag, int nthreads) {
    if (check_common(s, cam, W, H, mapping, k, f) || !out_rgbz || K < 1) return -1;
    if (!pix) npix = (int64_t)W * H;
    if (check_pix(pix, npix, W, H)) return -1;
    job_t J;
    memset(&J, 0, sizeof(J));
    J.s = s; J.cam = cam; J.W = W; J.H = H; J.K = K; J.mapping = mapping; J.k = k; J.f = f; J.z0 = z0;
    J.pix = pix; J.npix = npix; J.out = out_rgbz; J.out_n = out_normal; J.prim = out_prim; J.flag = out_flag;
    return run_job(&J, nthreads);
}

static int check_jitter(int spp, const float* jitter) {
    if (spp < 1 || spp > 16 || !jitter) return -1;
    for (int i = 0; i < 2 * spp; ++i)
        if (!(jitter[i] >= 0.0f && jitter[i] < 1.0f)) return -1;
    return 0;
}

int orc_render_pass_ms(const orc_scene* s, const double cam[10], int W, int H, int mapping, double k, double f,
                       double z0, int spp, const float* jitter, const float* in_rgbz, const double* in_normal,
                       const int64_t* pix, int64_t npix, double* out_rgbz, double* out_normal, int32_t* out_prim,
                       uint8_t* out_flag, int nthreads) {
    if (check_common(s, cam, W, H, mapping, k, f) || !out_rgbz || check_jitter(spp, jitter)) return -1;
    if (!pix) npix = (int64_t)W * H;
    if (check_pix(pix, npix, W, H)) return -1;
    job_t J;
    memset(&J, 0, sizeof(J));
    J.s = s; J.cam = cam; J.W = W; J.H = H; J.K = 1; J.mapping = mapping; J.k = k; J.f = f; J.z0 = z0;
    J.in = in_rgbz; J.in_n = in_normal; J.spp = spp; J.jitter = jitter;
    J.pix = pix; J.npix = npix; J.out = out_rgbz; J.out_n = out_normal; J.prim = out_prim; J.flag = out_flag;
    return run_job(&J, nthreads);
}

/* K multi-sample passes from I_0 over the whole image (a sample reads its
 * neighbours' previous values, so chains are no longer per pixel); the image
 * and the normals are carried in double between passes. out_flag = OR over
 * the passes. */
int orc_render_ms(const orc_scene* s, const double cam[10], int W, int H, int K, int mapping, double k, double f,
                  double z0, int spp, const float* jitter, double* out_rgbz, double* out_normal, uint8_t* out_flag,
                  int nthreads) {
    if (check_common(s, cam, W, H, mapping, k, f) || !out_rgbz || K < 1 || check_jitter(spp, jitter)) return -1;
    const int64_t P = (int64_t)W * H;
    double* prev = (double*)malloc(sizeof(double) * 4 * P);
    double* nprev = (double*)malloc(sizeof(double) * 3 * P);
    double* ncur = (double*)malloc(sizeof(double) * 3 * P);
    uint8_t* fl = (uint8_t*)calloc((size_t)P, 1);
    if (!prev || !nprev || !ncur || !fl) {
        free(prev);
        free(nprev);
        free(ncur);
        free(fl);
        return -1;
    }
    if (out_flag) memset(out_flag, 0, (size_t)P);
    for (int n = 0; n < K; ++n) {
        job_t J;
        memset(&J, 0, sizeof(J));
        J.s = s; J.cam = cam; J.W = W; J.H = H; J.K = 1; J.mapping = mapping; J.k = k; J.f = f; J.z0 = z0;
        J.in_d = n == 0 ? NULL : prev; J.in_n = n == 0 ? NULL : nprev; J.spp = spp; J.jitter = jitter;
        J.npix = P; J.out = out_rgbz; J.out_n = ncur; J.flag = fl;
        run_job(&J, nthreads);
        memcpy(prev, out_rgbz, sizeof(double) * 4 * P);
        memcpy(nprev, ncur, sizeof(double) * 3 * P);
        for (int64_t i = 0; out_flag && i < P; ++i) out_flag[i] |= fl[i];
    }
    if (out_normal) memcpy(out_normal, ncur, sizeof(double) * 3 * P);
    free(prev);
    free(nprev);
    free(ncur);
    free(fl);
    return 0;
}

/* ---------------------------------------------------------------- image space */

/*
 * Mirror ("reflect") edge rule of §6.1: an index past an edge is reflected
 * back into the image about that edge, the edge pixel itself not repeated
 * (-1 -> 0, -2 -> 1, n -> n-1, n+1 -> n-2), again and again for offsets of more
 * than one image width. Reading: the paper names mirroring but not its exact
 * form; this is the reflection that keeps the sample nearest to its original.
 */
int64_t orc_mirror_index(int64_t i, int64_t n) {
    if (n <= 1) return 0;
    const int64_t period = 2 * n;
    int64_t m = i % period;
    if (m < 0) m += period;
    return m < n ? m : period - 1 - m;
}

/*
 * One image-space pass (§6, §6.1). Reading: the displacement is Eq. 5's
 * k (2c - 1) restricted to the screen plane (B moves along the view axis and
 * does not move a pixel), k_px being k in pixels, red to the right and green
 * up (towards row 0); the sample is the nearest pixel, halves rounding up.
 * Computed in double from the float32 inputs.
 *
 * The flag marks samples whose displaced coordinate lies within
 * ORC_IMG_TOL (|x| + k_px + 1) of a half-integer, the boundary between two
 * nearest pixels: evaluating x + k (2c - 1) and the rounding in float32 errs by
 * at most a few units of 2^-24 of those magnitudes, so outside the band every
 * correct float32 evaluation takes the same pixel.
 */
static int near_half(double s, double band) {
    const double frac = s - floor(s); /* in [0, 1) */
    return fabs(frac - 0.5) <= band;
}

int orc_imagespace_pass(const float* base, const float* prev, int W, int H, double k_px, const int64_t* pix,
                        int64_t npix, float* out, uint8_t* out_flag) {
    if (!base || !prev || !out || W < 1 || H < 1 || !(k_px >= 0.0)) return -1;
    if (!pix) npix = (int64_t)W * H;
    for (int64_t i = 0; i < npix; ++i) {
        const int64_t p = pix ? pix[i] : i;
        if (p < 0 || p >= (int64_t)W * H) return -1;
        const int64_t x = p % W, y = p / W;
        const float* c = prev + 4 * p;
        const double sx = (double)x + k_px * (2.0 * (double)c[0] - 1.0);
        const double sy = (double)y - k_px * (2.0 * (double)c[1] - 1.0);
        const int64_t ix = orc_mirror_index((int64_t)floor(sx + 0.5), W);
        const int64_t iy = orc_mirror_index((int64_t)floor(sy + 0.5), H);
        if (ix < 0 || ix >= W || iy < 0 || iy >= H) return -1;
        memcpy(out + 4 * i, base + 4 * (iy * W + ix), 4 * sizeof(float));
        if (out_flag)
            out_flag[i] = (uint8_t)(near_half(sx, ORC_IMG_TOL * ((double)x + k_px + 1.0)) ||
                                    near_half(sy, ORC_IMG_TOL * ((double)y + k_px + 1.0)));
    }
    return 0;
}
