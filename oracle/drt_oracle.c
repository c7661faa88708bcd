/*
 * drt_oracle.c -- plain, slow FP64 CPU oracle of the Dynamic Ray Tracing (DRT) hot path of
 * Bilibashi, Vitucci, Degli-Esposti, "On Dynamic Ray Tracing and Anticipative Channel Prediction
 * for Dynamic Environments".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this library.  It shares no code, header, table or helper with the CUDA library.
 *
 * Two independent geometric solvers fill the same per-(path, time-step) record:
 *
 *   O-DRT      the paper's procedure.  Per wall a local frame attached to the moving body with the
 *              wall on y^I = 0 (Eq. coordinate_transf); TX/RX states carried into it with the
 *              relative-motion transforms (Eqs. relative_vel, relative_acc) and back with their
 *              inverses (Eqs. global_vel_ref_point, global_acc_ref_point); image chain and
 *              back-tracking for multiple reflections (Sec. III-A.2); the reflection point of
 *              Eq. ref_point; the diffraction point of Eq. diff_point in an edge frame with z along
 *              the edge (Sec. III-B); scattering tiles as rigid body points (Sec. III-C,
 *              Eq. RigidBodyMotion).  Velocities and accelerations of the interaction points are
 *              the chain rule of App. B / App. C, evaluated by second-order forward differentiation
 *              (value, d/dt, d^2/dt^2) of Eqs. ref_point and diff_point.  A segment with two or more
 *              diffractions (called "straightforward" in Sec. III-B but not given) is solved by
 *              damped Newton on the unfolded length with finite-difference velocities.
 *   O-RESOLVE  the brute-force snapshot solve the paper validates against (Sec. IV-A.2): every
 *              primitive posed at t, every interaction parameter solved from scratch (face centre /
 *              edge midpoint start) by damped Newton on the total path length, velocities by
 *              5-point finite differences in time.
 *
 * Both feed one coefficient module (Fresnel reflection, Kouyoumjian-Pathak UTD with Luebbers'
 * dielectric heuristic, Effective-Roughness directive scattering, ray spreading, polarisation
 * tracking), the Doppler product of App. A Eq. doppler_freq, and the direct FP64 sum
 * H(t,f) = sum_p a_p(t) exp(-j 2 pi f tau_p(t)).
 *
 * Parity pins live in the CPU tests; no function here is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_C0 299792458.0
#define OR_EPS0 8.8541878128e-12
#define OR_PI 3.14159265358979323846
#define OR_MAXI 4

enum { OR_T_NONE = 0, OR_T_R = 1, OR_T_D = 2, OR_T_S = 3 };
/* flag bits of one path-step; 0 means the path exists at that instant */
enum { OR_F_FACE = 1, OR_F_EDGE = 2, OR_F_SIDE = 4, OR_F_NOCONV = 8, OR_F_DEGEN = 16 };

/* ---------------------------------------------------------------- scene records (byte layouts of
 * the shared input generator) */
typedef struct { double o[3], v[3], a[3], k[3], w0, wdot; } or_body;
typedef struct { double r[3], v[3], a[3]; } or_term;
typedef struct { double eps_r, sigma, rough_s, pec; } or_mat;
typedef struct { int32_t body, material; double c[3], n[3], u[3], hu, hw; } or_face;
typedef struct { int32_t body, material; double a[3], b[3], n0[3], nn[3], wedge_n; } or_edge;
typedef struct { int32_t body, material; double c[3], n[3], area, s, alpha_r, phase; } or_tile;

typedef struct {
    or_term tx, rx;
    int32_t n_bodies, n_materials, n_faces, n_edges, n_tiles, pad_;
    const or_body *bodies;
    const or_mat *mats;
    const or_face *faces;
    const or_edge *edges;
    const or_tile *tiles;
} or_scene;

typedef struct { int n; int type[OR_MAXI]; int prim[OR_MAXI]; double s0[OR_MAXI]; } or_path;

/* ---------------------------------------------------------------- 3-vectors */
typedef struct { double x, y, z; } v3;
static v3 V(const double *p) { v3 r = {p[0], p[1], p[2]}; return r; }
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 crs(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static double nrm(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / nrm(a)); }
static v3 matv(const double R[3][3], v3 a) {
    return mk(R[0][0] * a.x + R[0][1] * a.y + R[0][2] * a.z, R[1][0] * a.x + R[1][1] * a.y + R[1][2] * a.z,
              R[2][0] * a.x + R[2][1] * a.y + R[2][2] * a.z);
}

/* kinematic state of a point: position, velocity, acceleration (world components) */
typedef struct { v3 p, v, a; } kst;

/* ---------------------------------------------------------------- kinematics (Eq. Taylor, Sec. III-A) */
typedef struct { double R[3][3]; v3 O, vO, aO, w, wd, o0; } or_pose;

/* Rotation by angle th about the fixed unit axis k (Rodrigues' formula). */
static void rodrigues(v3 k, double th, double R[3][3]) {
    double c = cos(th), s = sin(th), C = 1.0 - c;
    R[0][0] = c + k.x * k.x * C;       R[0][1] = k.x * k.y * C - k.z * s; R[0][2] = k.x * k.z * C + k.y * s;
    R[1][0] = k.y * k.x * C + k.z * s; R[1][1] = c + k.y * k.y * C;       R[1][2] = k.y * k.z * C - k.x * s;
    R[2][0] = k.z * k.x * C - k.y * s; R[2][1] = k.z * k.y * C + k.x * s; R[2][2] = c + k.z * k.z * C;
}

/* Body pose at dt = t - t0: reference point by Eq. Taylor, theta(t) = w0 dt + wdot dt^2/2 about the
 * fixed axis, omega(t) = omega(t0) + omega_dot dt (Sec. III-A). */
static void body_pose(const or_body *b, double t, or_pose *P) {
    double th = b->w0 * t + 0.5 * b->wdot * t * t, ws = b->w0 + b->wdot * t;
    v3 k = V(b->k);
    rodrigues(k, th, P->R);
    P->o0 = V(b->o);
    P->O = add(add(V(b->o), scl(V(b->v), t)), scl(V(b->a), 0.5 * t * t));
    P->vO = add(V(b->v), scl(V(b->a), t));
    P->aO = V(b->a);
    P->w = scl(k, ws);
    P->wd = scl(k, b->wdot);
}

/* State of the body point that sat at p0 at t0: v = v_O + w x O^I Q (Eq. RigidBodyMotion), and its
 * time derivative a = a_O + w_dot x r + w x (w x r). */
static kst pose_point(const or_pose *P, v3 p0) {
    kst s;
    v3 r = matv(P->R, sub(p0, P->o0));
    s.p = add(P->O, r);
    s.v = add(P->vO, crs(P->w, r));
    s.a = add(add(P->aO, crs(P->wd, r)), crs(P->w, crs(P->w, r)));
    return s;
}

static kst terminal_state(const or_term *T, double t) {   /* Eq. Taylor */
    kst s;
    s.p = add(add(V(T->r), scl(V(T->v), t)), scl(V(T->a), 0.5 * t * t));
    s.v = add(V(T->v), scl(V(T->a), t));
    s.a = V(T->a);
    return s;
}

/* ---------------------------------------------------------------- local frames (Eq. coordinate_transf) */
typedef struct { kst O; v3 w, wd; v3 ex, ey, ez; } or_frame;

/* Frame attached to a face: origin at the face centre, y^I along the face normal, so the wall lies
 * on y^I = 0 as Eq. ref_point assumes; x^I along the face's first in-plane axis. */
static void face_frame(const or_scene *S, int f, double t, or_frame *F) {
    const or_face *fc = &S->faces[f];
    or_pose P;
    body_pose(&S->bodies[fc->body], t, &P);
    F->O = pose_point(&P, V(fc->c));
    F->w = P.w; F->wd = P.wd;
    F->ex = matv(P.R, V(fc->u));
    F->ey = matv(P.R, V(fc->n));
    F->ez = crs(F->ex, F->ey);
}

/* Frame attached to an edge: origin at edge point a, z^I along the edge (Sec. III-B), x^I along the
 * 0-face tangent t0 = n0 x e pointing away from the edge, y^I = n0. */
static void edge_frame(const or_scene *S, int e, double t, or_frame *F, double *len, double *wn) {
    const or_edge *ed = &S->edges[e];
    or_pose P;
    body_pose(&S->bodies[ed->body], t, &P);
    v3 e0 = sub(V(ed->b), V(ed->a));
    *len = nrm(e0);
    e0 = scl(e0, 1.0 / *len);
    F->O = pose_point(&P, V(ed->a));
    F->w = P.w; F->wd = P.wd;
    F->ez = matv(P.R, e0);
    F->ex = matv(P.R, crs(V(ed->n0), e0));
    F->ey = crs(F->ez, F->ex);
    *wn = ed->wedge_n;
}

/* World state -> local frame: inverse of Eq. coordinate_transf for positions and the relative-motion
 * transforms Eqs. relative_vel and relative_acc (Euler, Coriolis and centrifugal terms), expressed in
 * local components. */
static kst to_local(const or_frame *F, kst X) {
    v3 r = sub(X.p, F->O.p);
    v3 vrel = sub(sub(X.v, F->O.v), crs(F->w, r));
    v3 arel = sub(sub(sub(sub(X.a, F->O.a), crs(F->wd, r)), scl(crs(F->w, vrel), 2.0)), crs(F->w, crs(F->w, r)));
    kst L;
    L.p = mk(dot(r, F->ex), dot(r, F->ey), dot(r, F->ez));
    L.v = mk(dot(vrel, F->ex), dot(vrel, F->ey), dot(vrel, F->ez));
    L.a = mk(dot(arel, F->ex), dot(arel, F->ey), dot(arel, F->ez));
    return L;
}

/* Local state -> world: Eq. coordinate_transf and the inverse relative-motion transforms
 * Eqs. global_vel_ref_point and global_acc_ref_point. */
static kst from_local(const or_frame *F, kst L) {
    v3 r = add(add(scl(F->ex, L.p.x), scl(F->ey, L.p.y)), scl(F->ez, L.p.z));
    v3 vrel = add(add(scl(F->ex, L.v.x), scl(F->ey, L.v.y)), scl(F->ez, L.v.z));
    v3 arel = add(add(scl(F->ex, L.a.x), scl(F->ey, L.a.y)), scl(F->ez, L.a.z));
    kst X;
    X.p = add(F->O.p, r);
    X.v = add(add(F->O.v, vrel), crs(F->w, r));
    X.a = add(add(add(add(F->O.a, arel), crs(F->wd, r)), scl(crs(F->w, vrel), 2.0)), crs(F->w, crs(F->w, r)));
    return X;
}

/* Image through the wall of frame F (Sec. III-A.2): same x^I, z^I, opposite y^I, for position,
 * velocity and acceleration alike. */
static kst image_local(kst L) { L.p.y = -L.p.y; L.v.y = -L.v.y; L.a.y = -L.a.y; return L; }
static kst image_world(const or_scene *S, int f, double t, kst X) {
    or_frame F;
    face_frame(S, f, t, &F);
    return from_local(&F, image_local(to_local(&F, X)));
}

/* ---------------------------------------------------------------- second-order jets (value, d/dt, d2/dt2) */
typedef struct { double f, d, dd; } jet;
static jet J(double f, double d, double dd) { jet r = {f, d, dd}; return r; }
static jet jadd(jet a, jet b) { return J(a.f + b.f, a.d + b.d, a.dd + b.dd); }
static jet jsub(jet a, jet b) { return J(a.f - b.f, a.d - b.d, a.dd - b.dd); }
static jet jmul(jet a, jet b) { return J(a.f * b.f, a.d * b.f + a.f * b.d, a.dd * b.f + 2.0 * a.d * b.d + a.f * b.dd); }
static jet jdiv(jet a, jet b) {
    double q = a.f / b.f;
    double qd = (a.d - q * b.d) / b.f;
    double qdd = (a.dd - 2.0 * qd * b.d - q * b.dd) / b.f;
    return J(q, qd, qdd);
}
static jet jsqrt(jet a) {
    double r = sqrt(a.f);
    double rd = a.d / (2.0 * r);
    double rdd = (a.dd - 2.0 * rd * rd) / (2.0 * r);
    return J(r, rd, rdd);
}
static jet jx(kst s) { return J(s.p.x, s.v.x, s.a.x); }
static jet jy(kst s) { return J(s.p.y, s.v.y, s.a.y); }
static jet jz(kst s) { return J(s.p.z, s.v.z, s.a.z); }

/* Eq. ref_point in the wall frame (wall on y = 0, T and R on the y > 0 side):
 *   x_Q = x_T + (x_R - x_T) y_T / (y_R + y_T),  z_Q likewise,  y_Q = 0.
 * Carried on jets, this is App. B: the first-order part is Eq. ref_point_velo with the partials of
 * App. B, the second-order part is Eq. ref_point_acc. */
static kst ref_point_local(kst T, kst R) {
    jet g = jdiv(jy(T), jadd(jy(T), jy(R)));
    jet xq = jadd(jx(T), jmul(jsub(jx(R), jx(T)), g));
    jet zq = jadd(jz(T), jmul(jsub(jz(R), jz(T)), g));
    kst Q;
    Q.p = mk(xq.f, 0.0, zq.f); Q.v = mk(xq.d, 0.0, zq.d); Q.a = mk(xq.dd, 0.0, zq.dd);
    return Q;
}

/* Eq. diff_point in the edge frame (edge on the z axis), with the 2D distances of Eq. dist2D_TXRX:
 *   z_QD = z_RX + d_RX (z_TX - z_RX) / (d_TX + d_RX).
 * On jets the first-order part is App. C (Eqs. diff_point_velo .. diff_point_velo4). */
static kst diff_point_local(kst T, kst R) {
    jet dT = jsqrt(jadd(jmul(jx(T), jx(T)), jmul(jy(T), jy(T))));
    jet dR = jsqrt(jadd(jmul(jx(R), jx(R)), jmul(jy(R), jy(R))));
    jet zq = jadd(jz(R), jdiv(jmul(dR, jsub(jz(T), jz(R))), jadd(dT, dR)));
    kst Q;
    Q.p = mk(0.0, 0.0, zq.f); Q.v = mk(0.0, 0.0, zq.d); Q.a = mk(0.0, 0.0, zq.dd);
    return Q;
}

/* ---------------------------------------------------------------- O-DRT */
typedef struct { kst V[OR_MAXI + 2]; int flags; } or_geom;

/* Back-tracking over the reflections strictly between vertices a and b (Sec. III-A.2): the source
 * V[a] is imaged through the walls in order; then, from the receiver V[b] and the last wall back
 * towards the source, each reflection point is Eq. ref_point between the source imaged through the
 * preceding walls and the (virtual) receiver found at the previous step. */
static void odrt_backtrack(const or_scene *S, const or_path *pa, double t, or_geom *G, int a, int b) {
    int m = b - a - 1;
    if (m <= 0) return;
    kst img[OR_MAXI + 1];
    img[0] = G->V[a];
    for (int j = 1; j < m; ++j) img[j] = image_world(S, pa->prim[a + j - 1], t, img[j - 1]);
    kst next = G->V[b];
    for (int j = m; j >= 1; --j) {
        or_frame F;
        face_frame(S, pa->prim[a + j - 1], t, &F);
        kst Q = from_local(&F, ref_point_local(to_local(&F, img[j - 1]), to_local(&F, next)));
        G->V[a + j] = Q;
        next = Q;
    }
}

/* Position of the D vertex at index d on its edge for a given edge parameter. */
static v3 edge_point(const or_scene *S, int e, double t, double s) {
    or_frame F;
    double L, wn;
    edge_frame(S, e, t, &F, &L, &wn);
    return add(F.O.p, scl(F.ez, s));
}

/* Reflect a world point across a face plane posed at t. */
static v3 mirror_point(const or_scene *S, int f, double t, v3 X) {
    or_frame F;
    face_frame(S, f, t, &F);
    double h = dot(sub(X, F.O.p), F.ey);
    return sub(X, scl(F.ey, 2.0 * h));
}
static v3 mirror_dir(const or_scene *S, int f, double t, v3 d) {
    or_frame F;
    face_frame(S, f, t, &F);
    return sub(d, scl(F.ey, 2.0 * dot(d, F.ey)));
}

static int solve_linear(int n, double *A, double *b) {  /* Gaussian elimination, partial pivoting */
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (fabs(A[p * n + c]) < 1e-300) return -1;
        if (p != c) {
            for (int k = 0; k < n; ++k) { double tmp = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = tmp; }
            double tmp = b[c]; b[c] = b[p]; b[p] = tmp;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
        b[c] = s / A[c * n + c];
    }
    return 0;
}

/* Damped Newton minimisation of a convex path-length function f(x) (Fermat: a ray is the stationary,
 * here minimal, total length through its sequence of planes and lines), continued over a smoothing
 * parameter: each segment length |d| is replaced by sqrt(|d|^2 + delta^2) with delta = 1 m, 0.1 m,
 * ..., 1e-5 m and finally 0, each stage starting from the previous minimiser, so no iterate gets
 * caught on the kink where two vertices meet.  Hessian by central differences of the analytic
 * gradient.  Returns 1 when the final gradient is below 1e-9. */
typedef double (*or_objfn)(const void *ctx, const double *x, double delta, double *g);
static int or_minimize(or_objfn fn, const void *ctx, int n, double *x) {
    static const double deltas[] = {1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 0.0};
    double g[2 * OR_MAXI], gp[2 * OR_MAXI], gm[2 * OR_MAXI], tmp[2 * OR_MAXI], st[2 * OR_MAXI];
    double H[4 * OR_MAXI * OR_MAXI];
    if (n == 0) return 1;
    for (int stage = 0; stage < 7; ++stage) {
        double delta = deltas[stage], tol = delta > 0 ? 1e-11 : 1e-14;
        double h = delta > 0 ? fmin(1e-6, 0.01 * delta) : 1e-6;
        for (int it = 0; it < 100; ++it) {
            double f = fn(ctx, x, delta, g);
            double gmax = 0.0;
            for (int j = 0; j < n; ++j) gmax = fmax(gmax, fabs(g[j]));
            if (gmax < tol) break;
            for (int c = 0; c < n; ++c) {
                memcpy(tmp, x, sizeof(double) * n);
                tmp[c] = x[c] + h; fn(ctx, tmp, delta, gp);
                tmp[c] = x[c] - h; fn(ctx, tmp, delta, gm);
                for (int r = 0; r < n; ++r) H[r * n + c] = (gp[r] - gm[r]) / (2 * h);
            }
            for (int j = 0; j < n; ++j) st[j] = -g[j];
            if (solve_linear(n, H, st) != 0) for (int j = 0; j < n; ++j) st[j] = -g[j];
            double gd = 0.0, smax = 0.0;
            for (int j = 0; j < n; ++j) gd += g[j] * st[j];
            if (!(gd < 0)) for (int j = 0; j < n; ++j) st[j] = -g[j];
            for (int j = 0; j < n; ++j) smax = fmax(smax, fabs(st[j]));
            double alpha = 1.0;
            for (int ls = 0; ls < 80; ++ls) {
                for (int j = 0; j < n; ++j) tmp[j] = x[j] + alpha * st[j];
                if (fn(ctx, tmp, delta, NULL) <= f + 1e-13 * fabs(f)) break;
                alpha *= 0.5;
            }
            memcpy(x, tmp, sizeof(double) * n);
            if (alpha * smax < 1e-15) break;
        }
    }
    double gmax = 0.0;
    fn(ctx, x, 0.0, g);
    for (int j = 0; j < n; ++j) gmax = fmax(gmax, fabs(g[j]));
    return gmax < 1e-9;
}

static double smooth_len(v3 d, double delta) { return sqrt(dot(d, d) + delta * delta); }

/* Unfolded length of the segment between anchors a and b with edge parameters s[] of its D
 * vertices (reflections unfolded by imaging the start of each sub-segment through its walls), and
 * its gradient with respect to s[]. */
static double multid_length(const or_scene *S, const or_path *pa, double t, int a, int b, v3 Pa, v3 Pb,
                            const double *s, double delta, double *grad) {
    int didx[OR_MAXI], m = 0;
    for (int i = a + 1; i < b; ++i)
        if (pa->type[i - 1] == OR_T_D) didx[m++] = i;
    double L = 0.0;
    if (grad)
        for (int j = 0; j < m; ++j) grad[j] = 0.0;
    for (int j = 0; j <= m; ++j) {       /* sub-segment j: from point j-1 to point j */
        int i0 = (j == 0) ? a : didx[j - 1];
        int i1 = (j == m) ? b : didx[j];
        v3 X = (j == 0) ? Pa : edge_point(S, pa->prim[i0 - 1], t, s[j - 1]);
        v3 Y = (j == m) ? Pb : edge_point(S, pa->prim[i1 - 1], t, s[j]);
        v3 ex = mk(0, 0, 0);
        if (j > 0) {
            or_frame F;
            double len, wn;
            edge_frame(S, pa->prim[i0 - 1], t, &F, &len, &wn);
            ex = F.ez;
        }
        for (int i = i0 + 1; i < i1; ++i) {
            X = mirror_point(S, pa->prim[i - 1], t, X);
            ex = mirror_dir(S, pa->prim[i - 1], t, ex);
        }
        v3 r = sub(X, Y);
        double l = smooth_len(r, delta);
        L += l;
        if (!grad) continue;
        v3 rh = scl(r, 1.0 / l);
        if (j > 0) grad[j - 1] += dot(rh, ex);
        if (j < m) {
            or_frame F;
            double len, wn;
            edge_frame(S, pa->prim[i1 - 1], t, &F, &len, &wn);
            grad[j] -= dot(rh, F.ez);
        }
    }
    return L;
}

/* Edge parameters of a segment with >= 2 diffractions: minimum of the unfolded length (convex in
 * the edge parameters), started from the t0 parameters of the ray-tracing run. */
typedef struct { const or_scene *S; const or_path *pa; double t; int a, b; v3 Pa, Pb; } or_md_ctx;
static double md_obj(const void *c, const double *x, double delta, double *g) {
    const or_md_ctx *C = (const or_md_ctx *)c;
    return multid_length(C->S, C->pa, C->t, C->a, C->b, C->Pa, C->Pb, x, delta, g);
}
static int multid_newton(const or_scene *S, const or_path *pa, double t, int a, int b, v3 Pa, v3 Pb, double *s) {
    int m = 0;
    for (int i = a + 1; i < b; ++i)
        if (pa->type[i - 1] == OR_T_D) s[m++] = pa->s0[i - 1];
    or_md_ctx C = {S, pa, t, a, b, Pa, Pb};
    return or_minimize(md_obj, &C, m, s);
}

static void odrt_anchor_states(const or_scene *S, const or_path *pa, double t, or_geom *G) {
    G->V[0] = terminal_state(&S->tx, t);
    G->V[pa->n + 1] = terminal_state(&S->rx, t);
    for (int i = 1; i <= pa->n; ++i)
        if (pa->type[i - 1] == OR_T_S) {
            const or_tile *tl = &S->tiles[pa->prim[i - 1]];
            or_pose P;
            body_pose(&S->bodies[tl->body], t, &P);
            G->V[i] = pose_point(&P, V(tl->c));  /* Sec. III-C: tile centroid moves rigidly */
        }
}

/* O-DRT geometry of one path at t (positions, sliding velocities, accelerations of all vertices). */
static void odrt_solve(const or_scene *S, const or_path *pa, double t, or_geom *G) {
    G->flags = 0;
    odrt_anchor_states(S, pa, t, G);
    int a = 0;
    for (int b = 1; b <= pa->n + 1; ++b) {
        if (b <= pa->n && pa->type[b - 1] != OR_T_S) continue;
        int nd = 0, dpos = -1;
        for (int i = a + 1; i < b; ++i)
            if (pa->type[i - 1] == OR_T_D) { ++nd; dpos = i; }
        if (nd == 0) {
            odrt_backtrack(S, pa, t, G, a, b);
        } else if (nd == 1) {
            /* virtual source: V[a] imaged through the walls before the edge; virtual receiver: V[b]
             * imaged through the walls after it, last wall first (reflections unfolded) */
            kst src = G->V[a], rcv = G->V[b];
            for (int i = a + 1; i < dpos; ++i) src = image_world(S, pa->prim[i - 1], t, src);
            for (int i = b - 1; i > dpos; --i) rcv = image_world(S, pa->prim[i - 1], t, rcv);
            or_frame F;
            double len, wn;
            edge_frame(S, pa->prim[dpos - 1], t, &F, &len, &wn);
            kst Tl = to_local(&F, src), Rl = to_local(&F, rcv);
            double dT = hypot(Tl.p.x, Tl.p.y), dR = hypot(Rl.p.x, Rl.p.y);
            if (dT + dR < 1e-12) { G->flags |= OR_F_DEGEN; G->V[dpos] = G->V[a]; }
            else G->V[dpos] = from_local(&F, diff_point_local(Tl, Rl));
            odrt_backtrack(S, pa, t, G, a, dpos);
            odrt_backtrack(S, pa, t, G, dpos, b);
        } else {
            /* >= 2 diffractions: Newton on the unfolded length at t + k h, k = -2..2, then
             * 5-point finite differences for velocity and acceleration of the D vertices */
            const double h = 1e-3;
            double sk[5][OR_MAXI];
            int conv = 1;
            for (int k = -2; k <= 2; ++k) {
                double tk = t + k * h;
                or_geom Gk;
                odrt_anchor_states(S, pa, tk, &Gk);
                conv &= multid_newton(S, pa, tk, a, b, Gk.V[a].p, Gk.V[b].p, sk[k + 2]);
            }
            if (!conv) G->flags |= OR_F_NOCONV;
            int j = 0;
            for (int i = a + 1; i < b; ++i) {
                if (pa->type[i - 1] != OR_T_D) continue;
                v3 P[5];
                for (int k = 0; k < 5; ++k) P[k] = edge_point(S, pa->prim[i - 1], t + (k - 2) * h, sk[k][j]);
                kst Q;
                Q.p = P[2];
                Q.v = scl(add(sub(scl(P[3], 8.0), scl(P[1], 8.0)), sub(P[0], P[4])), 1.0 / (12.0 * h));
                Q.a = scl(add(add(scl(add(P[3], P[1]), 16.0), scl(P[2], -30.0)), scl(add(P[0], P[4]), -1.0)),
                          1.0 / (12.0 * h * h));
                G->V[i] = Q;
                ++j;
            }
            int prev = a;
            for (int i = a + 1; i <= b; ++i)
                if (i == b || pa->type[i - 1] == OR_T_D) { odrt_backtrack(S, pa, t, G, prev, i); prev = i; }
        }
        a = b;
    }
}

/* ---------------------------------------------------------------- O-RESOLVE */
typedef struct {
    int np;                 /* number of unknowns */
    int off[OR_MAXI];       /* first unknown of each vertex, -1 for tiles */
    v3 base[OR_MAXI], ax1[OR_MAXI], ax2[OR_MAXI];
    v3 P0, Pn;
} or_resolve_ctx;

static void resolve_setup(const or_scene *S, const or_path *pa, double t, or_resolve_ctx *C, double *x0) {
    C->np = 0;
    C->P0 = terminal_state(&S->tx, t).p;
    C->Pn = terminal_state(&S->rx, t).p;
    for (int i = 0; i < pa->n; ++i) {
        int ty = pa->type[i], pr = pa->prim[i];
        if (ty == OR_T_R) {
            or_frame F;
            face_frame(S, pr, t, &F);
            C->base[i] = F.O.p; C->ax1[i] = F.ex; C->ax2[i] = F.ez;
            C->off[i] = C->np; x0[C->np] = 0.0; x0[C->np + 1] = 0.0; C->np += 2;
        } else if (ty == OR_T_D) {
            or_frame F;
            double len, wn;
            edge_frame(S, pr, t, &F, &len, &wn);
            C->base[i] = F.O.p; C->ax1[i] = F.ez;
            C->off[i] = C->np; x0[C->np] = 0.5 * len; C->np += 1;
        } else {
            const or_tile *tl = &S->tiles[pr];
            or_pose P;
            body_pose(&S->bodies[tl->body], t, &P);
            C->base[i] = pose_point(&P, V(tl->c)).p;
            C->off[i] = -1;
        }
    }
}

static void resolve_points(const or_path *pa, const or_resolve_ctx *C, const double *x, v3 *P) {
    P[0] = C->P0;
    P[pa->n + 1] = C->Pn;
    for (int i = 0; i < pa->n; ++i) {
        int ty = pa->type[i];
        if (ty == OR_T_R) P[i + 1] = add(add(C->base[i], scl(C->ax1[i], x[C->off[i]])), scl(C->ax2[i], x[C->off[i] + 1]));
        else if (ty == OR_T_D) P[i + 1] = add(C->base[i], scl(C->ax1[i], x[C->off[i]]));
        else P[i + 1] = C->base[i];
    }
}

/* total length and its gradient: dL/dP_i = k_i - k_{i+1} with k_i the unit vector of segment i */
static double resolve_length(const or_path *pa, const or_resolve_ctx *C, const double *x, double delta, double *g) {
    v3 P[OR_MAXI + 2], k[OR_MAXI + 2];
    resolve_points(pa, C, x, P);
    double L = 0.0;
    for (int i = 1; i <= pa->n + 1; ++i) {
        v3 d = sub(P[i], P[i - 1]);
        double l = smooth_len(d, delta);
        L += l;
        k[i] = scl(d, 1.0 / l);
    }
    if (g) {
        for (int i = 0; i < pa->n; ++i) {
            if (C->off[i] < 0) continue;
            v3 dLdP = sub(k[i + 1], k[i + 2]);
            g[C->off[i]] = dot(dLdP, C->ax1[i]);
            if (pa->type[i] == OR_T_R) g[C->off[i] + 1] = dot(dLdP, C->ax2[i]);
        }
    }
    return L;
}

typedef struct { const or_path *pa; const or_resolve_ctx *C; } or_rs_ctx;
static double rs_obj(const void *c, const double *x, double delta, double *g) {
    const or_rs_ctx *R = (const or_rs_ctx *)c;
    return resolve_length(R->pa, R->C, x, delta, g);
}
static int resolve_positions(const or_scene *S, const or_path *pa, double t, v3 *P) {
    or_resolve_ctx C;
    double x[2 * OR_MAXI];
    resolve_setup(S, pa, t, &C, x);
    or_rs_ctx R = {pa, &C};
    int conv = or_minimize(rs_obj, &R, C.np, x);
    resolve_points(pa, &C, x, P);
    return conv;
}

/* O-RESOLVE geometry: positions solved from scratch at t and at t +- h, t +- 2h; velocities and
 * accelerations by 5-point central differences. */
static void resolve_solve(const or_scene *S, const or_path *pa, double t, or_geom *G) {
    const double h = 1e-3;
    v3 P[5][OR_MAXI + 2];
    int conv = 1;
    for (int k = 0; k < 5; ++k) conv &= resolve_positions(S, pa, t + (k - 2) * h, P[k]);
    G->flags = conv ? 0 : OR_F_NOCONV;
    for (int i = 0; i <= pa->n + 1; ++i) {
        G->V[i].p = P[2][i];
        G->V[i].v = scl(add(sub(scl(P[3][i], 8.0), scl(P[1][i], 8.0)), sub(P[0][i], P[4][i])), 1.0 / (12.0 * h));
        G->V[i].a = scl(add(add(scl(add(P[3][i], P[1][i]), 16.0), scl(P[2][i], -30.0)), scl(add(P[0][i], P[4][i]), -1.0)),
                        1.0 / (12.0 * h * h));
    }
    /* terminals and tiles are known exactly */
    kst tx = terminal_state(&S->tx, t), rx = terminal_state(&S->rx, t);
    G->V[0] = tx;
    G->V[pa->n + 1] = rx;
}

/* ---------------------------------------------------------------- validity (T_C) */
static double wrap2pi(double a) { a = fmod(a, 2 * OR_PI); return a < 0 ? a + 2 * OR_PI : a; }

/* Validity of a path-step from its vertices (Sec. II: DRT holds while the multipath structure does):
 * each reflection point inside its face and both neighbours on the face's front side; each
 * diffraction point on its edge segment and both neighbours in the wedge's exterior; each tile lit
 * from and seen from its front side.  *margin is the smallest distance (m) of any of these tests to
 * its decision boundary. */
static int path_flags(const or_scene *S, const or_path *pa, double t, const v3 *P, double *margin) {
    int fl = 0;
    double mg = INFINITY;
    for (int i = 1; i <= pa->n + 1; ++i)
        if (nrm(sub(P[i], P[i - 1])) < 1e-9) fl |= OR_F_DEGEN;
    for (int i = 1; i <= pa->n; ++i) {
        int ty = pa->type[i - 1], pr = pa->prim[i - 1];
        if (ty == OR_T_R) {
            or_frame F;
            face_frame(S, pr, t, &F);
            const or_face *fc = &S->faces[pr];
            v3 r = sub(P[i], F.O.p);
            double al = dot(r, F.ex), be = dot(r, F.ez);
            if (fabs(al) > fc->hu || fabs(be) > fc->hw) fl |= OR_F_FACE;
            if (isfinite(fc->hu)) mg = fmin(mg, fabs(fc->hu - fabs(al)));
            if (isfinite(fc->hw)) mg = fmin(mg, fabs(fc->hw - fabs(be)));
            double dp = dot(sub(P[i - 1], F.O.p), F.ey), dn = dot(sub(P[i + 1], F.O.p), F.ey);
            if (!(dp > 0) || !(dn > 0)) fl |= OR_F_SIDE;
            mg = fmin(mg, fmin(fabs(dp), fabs(dn)));
        } else if (ty == OR_T_D) {
            or_frame F;
            double len, wn;
            edge_frame(S, pr, t, &F, &len, &wn);
            double s = dot(sub(P[i], F.O.p), F.ez);
            if (s < 0 || s > len) fl |= OR_F_EDGE;
            mg = fmin(mg, fmin(fabs(s), fabs(len - s)));
            for (int side = -1; side <= 1; side += 2) {
                v3 r = sub(P[i + side], P[i]);
                v3 rp = sub(r, scl(F.ez, dot(r, F.ez)));
                double ph = wrap2pi(atan2(dot(rp, F.ey), dot(rp, F.ex)));
                if (!(ph > 0 && ph < wn * OR_PI)) fl |= OR_F_SIDE;
                /* angular distance to the two wedge faces (angles 0 and n pi) */
                double amg = fmin(fmin(ph, 2 * OR_PI - ph), fabs(ph - wn * OR_PI));
                mg = fmin(mg, nrm(rp) * sin(fmin(amg, 0.5 * OR_PI)));
            }
        } else {
            const or_tile *tl = &S->tiles[pr];
            or_pose Pp;
            body_pose(&S->bodies[tl->body], t, &Pp);
            v3 n = matv(Pp.R, V(tl->n));
            double dp = dot(sub(P[i - 1], P[i]), n), dn = dot(sub(P[i + 1], P[i]), n);
            if (!(dp > 0) || !(dn > 0)) fl |= OR_F_SIDE;
            mg = fmin(mg, fmin(fabs(dp), fabs(dn)));
        }
    }
    *margin = mg;
    return fl;
}

/* ---------------------------------------------------------------- coefficient module */

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton on P_n (Golub-Welsch-free textbook method). */
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) { double p3 = p2; p2 = p1; p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j; }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}
static double GLX[32], GLW[32];
static pthread_once_t gl_once = PTHREAD_ONCE_INIT;
static void gl_init(void) { gauss_legendre(32, GLX, GLW); }

/* exp(j x^2) G(x) with G(x) = int_x^inf exp(-j tau^2) dtau, x >= 0, by quadrature along the rotated
 * ray tau = x + exp(-j pi/4) r, r >= 0 (Cauchy's theorem).  There -j tau^2 = -j x^2 - sqrt2 x r (1+j)
 * - r^2, so the factor exp(-j x^2) comes out exactly and the rest decays like exp(-r^2 - sqrt2 x r);
 * composite 32-point Gauss-Legendre over 8 panels up to where the exponent reaches -42. */
static double complex fresnel_G_scaled(double x) {
    pthread_once(&gl_once, gl_init);
    double b = sqrt(2.0) * x;
    double R = 0.5 * (-b + sqrt(b * b + 4 * 42.0));
    const int panels = 8;
    double complex acc = 0.0;
    for (int p = 0; p < panels; ++p) {
        double lo = R * p / panels, hi = R * (p + 1) / panels, c = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
        for (int i = 0; i < 32; ++i) {
            double r = c + hw * GLX[i];
            acc += hw * GLW[i] * cexp(-r * r - b * r * (1.0 + I));
        }
    }
    return cexp(-I * OR_PI / 4) * acc;
}
double complex or_fresnel_G(double x) { return cexp(-I * x * x) * fresnel_G_scaled(x); }

/* UTD transition function F(X) = 2j sqrt(X) exp(jX) int_sqrt(X)^inf exp(-j tau^2) dtau
 * (Kouyoumjian-Pathak 1974). */
double complex or_transition_F(double X) {
    if (X <= 0) return 0.0;
    double s = sqrt(X);
    return 2.0 * I * s * fresnel_G_scaled(s);
}

/* Fresnel reflection coefficients (e^{+j w t}, eps_c = eps_r - j sigma / (w eps0)) for the
 * perpendicular (TE) and parallel (TM) components at incidence cosine ct (Sec. III-A, "Fresnel's
 * reflection coefficients as usually done in standard RT").  PEC: -1 and +1. */
static void fresnel(const or_mat *m, double fc, double ct, double complex *rte, double complex *rtm) {
    if (m->pec != 0.0) { *rte = -1.0; *rtm = 1.0; return; }
    double complex ec = m->eps_r - I * m->sigma / (2 * OR_PI * fc * OR_EPS0);
    double complex sq = csqrt(ec - 1.0 + ct * ct);
    *rte = (ct - sq) / (ct + sq);
    *rtm = (ec * ct - sq) / (ec * ct + sq);
}

/* One Kouyoumjian-Pathak term cot((pi +- beta)/(2n)) F(kL a+-(beta)), written with
 * eps = (pi +- beta) - 2 pi n N+- so that cot(.) = cot(eps/(2n)) and a+-(beta) = 2 sin^2(eps/2);
 * at eps -> 0 it tends to n sqrt(2 pi k L) sgn(eps) exp(j pi/4). */
static double complex utd_term(double eps, double n, double kL) {
    if (fabs(eps) < 1e-9) return n * sqrt(2 * OR_PI * kL) * (eps >= 0 ? 1.0 : -1.0) * cexp(I * OR_PI / 4);
    double sh = sin(0.5 * eps);
    return (cos(eps / (2 * n)) / sin(eps / (2 * n))) * or_transition_F(2.0 * kL * sh * sh);
}

/* Soft and hard UTD wedge diffraction coefficients (Kouyoumjian-Pathak; the distance parameter L is
 * the caller's, see path_amplitude), with Luebbers' heuristic for lossy wedges: the two
 * reflection-type terms are weighted by the 0-face and n-face Fresnel coefficients (-1 / +1 for a
 * perfect conductor recovers the "-/+" of the PEC form). */
void or_utd(double n, double phi, double phip, double sinb0, double L, double k, const or_mat *m, double fc,
            double complex *Ds, double complex *Dh) {
    double kL = k * L;
    double complex C = -cexp(-I * OR_PI / 4) / (2.0 * n * sqrt(2 * OR_PI * k) * sinb0);
    double bm = phi - phip, bp = phi + phip;
    double Np_m = round((bm + OR_PI) / (2 * OR_PI * n)), Nm_m = round((bm - OR_PI) / (2 * OR_PI * n));
    double Np_p = round((bp + OR_PI) / (2 * OR_PI * n)), Nm_p = round((bp - OR_PI) / (2 * OR_PI * n));
    double complex t1 = utd_term(OR_PI + bm - 2 * OR_PI * n * Np_m, n, kL);   /* cot((pi+(phi-phi'))/2n) */
    double complex t2 = utd_term(OR_PI - bm + 2 * OR_PI * n * Nm_m, n, kL);   /* cot((pi-(phi-phi'))/2n) */
    double complex t3 = utd_term(OR_PI - bp + 2 * OR_PI * n * Nm_p, n, kL);   /* cot((pi-(phi+phi'))/2n): 0-face */
    double complex t4 = utd_term(OR_PI + bp - 2 * OR_PI * n * Np_p, n, kL);   /* cot((pi+(phi+phi'))/2n): n-face */
    double complex r0s, r0h, rns, rnh;
    fresnel(m, fc, fabs(sin(phip)), &r0s, &r0h);
    fresnel(m, fc, fabs(sin(n * OR_PI - phi)), &rns, &rnh);
    *Ds = C * (t1 + t2 + r0s * t3 + rns * t4);
    *Dh = C * (t1 + t2 + r0h * t3 + rnh * t4);
}

/* Hemispheric normalisation of the ER directive lobe:
 * F(alpha, theta_i) = int_{hemisphere} ((1 + cos psi_R)/2)^alpha dOmega, psi_R measured from the
 * specular direction; tensor Gauss-Legendre quadrature in polar angle and azimuth. */
double or_er_norm(double alpha, double cti) {
    pthread_once(&gl_once, gl_init);
    double sti = sqrt(fmax(0.0, 1.0 - cti * cti));
    v3 r = mk(sti, 0.0, cti);   /* specular direction in a frame with the normal along z */
    double acc = 0.0;
    for (int i = 0; i < 32; ++i) {
        double th = 0.25 * OR_PI * (GLX[i] + 1.0), wt = 0.25 * OR_PI * GLW[i];
        for (int j = 0; j < 32; ++j) {
            double ph = OR_PI * (GLX[j] + 1.0), wp = OR_PI * GLW[j];
            v3 s = mk(sin(th) * cos(ph), sin(th) * sin(ph), cos(th));
            acc += wt * wp * sin(th) * pow(0.5 * (1.0 + dot(s, r)), alpha);
        }
    }
    return acc;
}

/* Effective-Roughness directive scattering (Sec. III-C) of a tile of area dA and scattering parameter
 * S: field magnitude factor at unit distance, relative to the incident field magnitude at the tile,
 * S sqrt(dA cos(theta_i) / F(alpha, theta_i)) ((1 + cos psi_R)/2)^(alpha/2), so that the scattered
 * power over the front hemisphere is S^2 times the power intercepted by the tile. */
double or_er_amp(double alpha, double S, double area, double cti, double cpsi) {
    double Fa = or_er_norm(alpha, cti);
    return S * sqrt(area * cti / Fa) * pow(0.5 * (1.0 + cpsi), 0.5 * alpha);
}

typedef struct { double complex x, y, z; } c3;
static double complex cdot(c3 E, v3 e) { return E.x * e.x + E.y * e.y + E.z * e.z; }
static c3 c3s(v3 e, double complex s) { c3 r = {s * e.x, s * e.y, s * e.z}; return r; }
static c3 c3add(c3 a, c3 b) { c3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static double c3norm(c3 E) { return sqrt(creal(E.x * conj(E.x) + E.y * conj(E.y) + E.z * conj(E.z))); }

/* linear polarisation vector transverse to k: the vertical (z) direction projected off k, x if k is
 * vertical; used for the isotropic "vertically polarised" TX and RX antennas */
static v3 vertical_pol(v3 k) {
    v3 p = sub(mk(0, 0, 1), scl(k, k.z));
    if (nrm(p) < 1e-9) p = sub(mk(1, 0, 0), scl(k, k.x));
    return unit(p);
}

/* Complex amplitude a_p of one path-step, excluding the propagation phase exp(-jkd) that H(t,f)
 * applies: (lambda/4pi) x ray spreading x polarimetric chain of Fresnel / UTD / ER factors, TX
 * polarised along vertical_pol(k_1), RX projecting on vertical_pol(k_{n+1}).  Line of sight gives
 * lambda/(4 pi d) (Friis). */
static double complex path_amplitude(const or_scene *S, const or_path *pa, double t, const v3 *P, double fc) {
    int n = pa->n;
    double k = 2 * OR_PI * fc / OR_C0, lam = OR_C0 / fc;
    v3 kd[OR_MAXI + 2];
    double len[OR_MAXI + 2];
    for (int i = 1; i <= n + 1; ++i) {
        v3 d = sub(P[i], P[i - 1]);
        len[i] = nrm(d);
        kd[i] = scl(d, 1.0 / len[i]);
    }
    /* Ray spreading (Sec. III-A "ray divergence factor") and the UTD distance parameters
     * (Sec. III-B, Kouyoumjian-Pathak), per anchor segment between point sources (TX, tiles, RX):
     *  - from a point source the wave is spherical, principal radii rho1 = rho2 = distance; without
     *    diffraction the segment spreads as 1 / (unfolded length);
     *  - a planar reflection keeps the principal radii and mirrors their directions;
     *  - at an edge the incident wavefront's radius of curvature rho_e in the plane of the incident ray
     *    and the edge follows from its principal radii (Euler: 1/rho_e = cos^2 g / rho1 + sin^2 g / rho2,
     *    g the angle between that plane and the first principal direction); for a straight edge the
     *    diffracted ray's second caustic lies rho_e behind the edge, so it spreads as
     *    sqrt(rho_e / (s (rho_e + s))) up to the next diffraction or point source at distance s, and
     *    its wavefront has one caustic on the edge (principal direction e x k_out, radius s) and the
     *    other radius rho_e + s;
     *  - the distance parameter of the transition function is
     *    L = s (rho_e + s) rho1 rho2 sin^2 b0 / (rho_e (rho1 + s) (rho2 + s)),
     *    which for a spherical incident wave is s s' sin^2 b0 / (s + s'). */
    double spread = 1.0;
    double rho1[OR_MAXI + 1], rho2[OR_MAXI + 1], rhoe[OR_MAXI + 1], snext[OR_MAXI + 1];
    int a = 0;
    for (int b = 1; b <= n + 1; ++b) {
        if (b <= n && pa->type[b - 1] != OR_T_S) continue;
        int last = a;            /* the point source or the latest diffraction */
        double d = 0.0;          /* distance travelled since `last` */
        v3 X1 = mk(0, 0, 0);     /* after a diffraction: principal direction of its caustic on the edge */
        for (int i = a + 1; i <= b; ++i) {
            d += len[i];
            if (i < b && pa->type[i - 1] == OR_T_R) {
                if (last != a) {
                    or_frame F;
                    face_frame(S, pa->prim[i - 1], t, &F);
                    X1 = sub(X1, scl(F.ey, 2.0 * dot(X1, F.ey)));
                }
                continue;
            }
            if (last == a) spread *= 1.0 / d;
            else {
                snext[last] = d;
                spread *= sqrt(rhoe[last] / (d * (rhoe[last] + d)));
            }
            if (i == b) break;
            or_frame F;
            double elen, wn;
            edge_frame(S, pa->prim[i - 1], t, &F, &elen, &wn);
            if (last == a) {
                rho1[i] = rho2[i] = rhoe[i] = d;
            } else {
                rho1[i] = d;
                rho2[i] = rhoe[last] + d;
                v3 u = sub(F.ez, scl(kd[i], dot(F.ez, kd[i])));
                double cg = nrm(u) > 1e-12 ? dot(unit(u), X1) : 0.0;
                rhoe[i] = 1.0 / (cg * cg / rho1[i] + (1.0 - cg * cg) / rho2[i]);
            }
            X1 = unit(crs(F.ez, kd[i + 1]));
            last = i;
            d = 0.0;
        }
        a = b;
    }
    c3 E = c3s(vertical_pol(kd[1]), 1.0);
    for (int i = 1; i <= n; ++i) {
        int ty = pa->type[i - 1], pr = pa->prim[i - 1];
        v3 kin = kd[i], kout = kd[i + 1];
        if (ty == OR_T_R) {
            const or_face *fc_ = &S->faces[pr];
            const or_mat *m = &S->mats[fc_->material];
            or_frame F;
            face_frame(S, pr, t, &F);
            v3 nf = F.ey;
            if (dot(nf, kin) > 0) nf = scl(nf, -1.0);
            double ct = -dot(nf, kin);
            v3 ep = crs(kin, nf);
            if (nrm(ep) < 1e-12) { ep = crs(nf, mk(1, 0, 0)); if (nrm(ep) < 1e-6) ep = crs(nf, mk(0, 1, 0)); }
            ep = unit(ep);
            v3 epin = crs(ep, kin), epout = crs(ep, kout);
            double complex rte, rtm;
            fresnel(m, fc, ct, &rte, &rtm);
            double rough = sqrt(fmax(0.0, 1.0 - m->rough_s * m->rough_s));
            E = c3add(c3s(ep, rough * rte * cdot(E, ep)), c3s(epout, rough * rtm * cdot(E, epin)));
        } else if (ty == OR_T_D) {
            const or_edge *ed = &S->edges[pr];
            const or_mat *m = &S->mats[ed->material];
            or_frame F;
            double elen, wn;
            edge_frame(S, pr, t, &F, &elen, &wn);
            v3 e = F.ez;
            v3 wi = sub(scl(kin, -1.0), scl(e, dot(scl(kin, -1.0), e)));
            v3 wo = sub(kout, scl(e, dot(kout, e)));
            double phip = wrap2pi(atan2(dot(wi, F.ey), dot(wi, F.ex)));
            double phi = wrap2pi(atan2(dot(wo, F.ey), dot(wo, F.ex)));
            double sinb0 = nrm(crs(kin, e));
            double sd = snext[i];
            double L = sd * (rhoe[i] + sd) * rho1[i] * rho2[i] * sinb0 * sinb0 / (rhoe[i] * (rho1[i] + sd) * (rho2[i] + sd));
            double complex Ds, Dh;
            or_utd(wn, phi, phip, sinb0, L, k, m, fc, &Ds, &Dh);
            v3 php = unit(scl(crs(e, kin), -1.0)), bp = crs(php, kin);
            v3 ph = unit(crs(e, kout)), b = crs(ph, kout);
            E = c3add(c3s(b, -Ds * cdot(E, bp)), c3s(ph, -Dh * cdot(E, php)));
        } else {
            const or_tile *tl = &S->tiles[pr];
            or_pose Pp;
            body_pose(&S->bodies[tl->body], t, &Pp);
            v3 nt = matv(Pp.R, V(tl->n));
            if (dot(nt, kin) > 0) nt = scl(nt, -1.0);
            double cti = -dot(nt, kin);
            v3 kspec = add(kin, scl(nt, 2.0 * cti));
            double cpsi = dot(kspec, kout);
            double amp = or_er_amp(tl->alpha_r, tl->s, tl->area, cti, cpsi);
            double complex ph = cexp(I * tl->phase);
            /* the scattered wave keeps the incident polarisation projected transverse to k_out,
             * rescaled to the incident magnitude */
            double nE = c3norm(E);
            c3 Ep = c3add(E, c3s(kout, -cdot(E, kout)));
            double nEp = c3norm(Ep);
            if (nEp < 1e-12 * nE || nE == 0.0) Ep = c3s(vertical_pol(kout), nE);
            else Ep = (c3){Ep.x * (nE / nEp), Ep.y * (nE / nEp), Ep.z * (nE / nEp)};
            E = (c3){Ep.x * amp * ph, Ep.y * amp * ph, Ep.z * amp * ph};
        }
    }
    return (lam / (4 * OR_PI)) * spread * cdot(E, vertical_pol(kd[n + 1]));
}

/* App. A, Eq. doppler_freq: f' = f0 prod_{i=1}^{n+1} (c - v_i.k_i) / (c - v_{i-1}.k_i), with v_0 the TX
 * and v_{n+1} the RX velocity and v_i the velocity of the i-th interaction point; f_D = f' - f0. */
static double path_doppler(int n, const kst *Vx, double fc) {
    double prod = 1.0;
    for (int i = 1; i <= n + 1; ++i) {
        v3 k = unit(sub(Vx[i].p, Vx[i - 1].p));
        prod *= (OR_C0 - dot(Vx[i].v, k)) / (OR_C0 - dot(Vx[i - 1].v, k));
    }
    return fc * (prod - 1.0);
}

/* ---------------------------------------------------------------- per path-step record */
typedef struct {
    const or_scene *S;
    int32_t n_paths;
    const uint8_t *n_int, *types;
    const int32_t *prims;
    const double *s0;
    double t_start, dt;
    int32_t n_steps;
    double fc;
    int32_t method;
    double *tau, *amp, *fd, *ang, *margin, *pts, *vel;
    uint8_t *flags;
    int64_t next;
    pthread_mutex_t mu;
} or_job;

static void load_path(const or_job *J, int p, or_path *pa) {
    pa->n = J->n_int[p];
    for (int i = 0; i < OR_MAXI; ++i) {
        pa->type[i] = J->types[p * OR_MAXI + i];
        pa->prim[i] = J->prims[p * OR_MAXI + i];
        pa->s0[i] = J->s0 ? J->s0[p * OR_MAXI + i] : 0.0;
    }
}

static void eval_one(const or_job *J, int64_t idx) {
    int ti = (int)(idx / J->n_paths), p = (int)(idx % J->n_paths);
    double t = J->t_start + ti * J->dt;
    or_path pa;
    load_path(J, p, &pa);
    or_geom G;
    if (J->method == 0) odrt_solve(J->S, &pa, t, &G);
    else resolve_solve(J->S, &pa, t, &G);
    v3 P[OR_MAXI + 2];
    for (int i = 0; i <= pa.n + 1; ++i) P[i] = G.V[i].p;
    double mg;
    int fl = G.flags | path_flags(J->S, &pa, t, P, &mg);
    double d = 0.0;
    for (int i = 1; i <= pa.n + 1; ++i) d += nrm(sub(P[i], P[i - 1]));
    double complex a = (fl & OR_F_DEGEN) ? 0.0 : path_amplitude(J->S, &pa, t, P, J->fc);
    J->tau[idx] = d / OR_C0;
    J->amp[2 * idx] = creal(a);
    J->amp[2 * idx + 1] = cimag(a);
    J->fd[idx] = path_doppler(pa.n, G.V, J->fc);
    v3 kdep = unit(sub(P[1], P[0])), karr = unit(sub(P[pa.n], P[pa.n + 1]));
    J->ang[4 * idx + 0] = atan2(kdep.y, kdep.x);
    J->ang[4 * idx + 1] = atan2(kdep.z, hypot(kdep.x, kdep.y));
    J->ang[4 * idx + 2] = atan2(karr.y, karr.x);
    J->ang[4 * idx + 3] = atan2(karr.z, hypot(karr.x, karr.y));
    J->flags[idx] = (uint8_t)fl;
    J->margin[idx] = mg;
    if (J->pts)
        for (int i = 0; i < OR_MAXI; ++i) {
            v3 q = (i < pa.n) ? P[i + 1] : mk(NAN, NAN, NAN);
            J->pts[(idx * OR_MAXI + i) * 3 + 0] = q.x;
            J->pts[(idx * OR_MAXI + i) * 3 + 1] = q.y;
            J->pts[(idx * OR_MAXI + i) * 3 + 2] = q.z;
        }
    if (J->vel)
        for (int i = 0; i < OR_MAXI + 2; ++i) {
            v3 q = (i <= pa.n + 1) ? G.V[i].v : mk(NAN, NAN, NAN);
            J->vel[(idx * (OR_MAXI + 2) + i) * 3 + 0] = q.x;
            J->vel[(idx * (OR_MAXI + 2) + i) * 3 + 1] = q.y;
            J->vel[(idx * (OR_MAXI + 2) + i) * 3 + 2] = q.z;
        }
}

static void *worker(void *arg) {
    or_job *J = (or_job *)arg;
    int64_t total = (int64_t)J->n_steps * J->n_paths;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t lo = J->next;
        J->next += 64;
        pthread_mutex_unlock(&J->mu);
        if (lo >= total) break;
        int64_t hi = lo + 64 < total ? lo + 64 : total;
        for (int64_t i = lo; i < hi; ++i) eval_one(J, i);
    }
    return NULL;
}

/* Per (time-step, path) record over t_n = t_start + n dt (seconds after t0), [T][P] row-major:
 * tau (s), amp (re, im), fD (Hz), angles (AoD az, el, AoA az, el; rad), flags, margin (m);
 * optional pts [T][P][4][3] (interaction points, NaN past n_int) and vel [T][P][6][3] (vertex
 * velocities TX, points, RX).  method 0 = O-DRT, 1 = O-RESOLVE.  Returns 0. */
int or_extrapolate(const or_scene *S, int32_t n_paths, const uint8_t *n_int, const uint8_t *types,
                   const int32_t *prims, const double *s0, double t_start, double dt, int32_t n_steps,
                   double fc, int32_t method, int32_t n_threads, double *tau, double *amp, double *fd,
                   double *ang, uint8_t *flags, double *margin, double *pts, double *vel) {
    pthread_once(&gl_once, gl_init);
    or_job J = {S, n_paths, n_int, types, prims, s0, t_start, dt, n_steps, fc, method,
                tau, amp, fd, ang, margin, pts, vel, flags, 0, PTHREAD_MUTEX_INITIALIZER};
    if (n_threads <= 1) {
        for (int64_t i = 0; i < (int64_t)n_steps * n_paths; ++i) eval_one(&J, i);
        return 0;
    }
    pthread_t th[256];
    int nt = n_threads > 256 ? 256 : n_threads;
    for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, worker, &J);
    for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* H(t_n, f_k) = sum over valid paths of a_p(t_n) exp(-j 2 pi f_k tau_p(t_n)), f_k = fc - B/2 + k B/N,
 * direct FP64 sum in path order; H is [T][F] (re, im). */
typedef struct {
    int32_t n_steps, n_paths, n_bins;
    const double *tau, *amp;
    const uint8_t *flags;
    double fc, bw;
    double *H;
    int32_t next;
    pthread_mutex_t mu;
} or_hjob;

static void h_row(const or_hjob *J, int t) {
    for (int kb = 0; kb < J->n_bins; ++kb) {
        double f = J->fc - 0.5 * J->bw + kb * (J->bw / J->n_bins);
        double complex h = 0.0;
        for (int p = 0; p < J->n_paths; ++p) {
            int64_t i = (int64_t)t * J->n_paths + p;
            if (J->flags[i]) continue;
            double complex a = J->amp[2 * i] + I * J->amp[2 * i + 1];
            h += a * cexp(-I * 2 * OR_PI * f * J->tau[i]);
        }
        J->H[2 * ((int64_t)t * J->n_bins + kb)] = creal(h);
        J->H[2 * ((int64_t)t * J->n_bins + kb) + 1] = cimag(h);
    }
}

static void *h_worker(void *arg) {
    or_hjob *J = (or_hjob *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int t = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (t >= J->n_steps) break;
        h_row(J, t);
    }
    return NULL;
}

int or_synthesize_H(int32_t n_steps, int32_t n_paths, const double *tau, const double *amp, const uint8_t *flags,
                    double fc, double bw, int32_t n_bins, int32_t n_threads, double *H) {
    or_hjob J = {n_steps, n_paths, n_bins, tau, amp, flags, fc, bw, H, 0, PTHREAD_MUTEX_INITIALIZER};
    if (n_threads <= 1) {
        for (int t = 0; t < n_steps; ++t) h_row(&J, t);
        return 0;
    }
    pthread_t th[256];
    int nt = n_threads > 256 ? 256 : n_threads;
    for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, h_worker, &J);
    for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* ---------------------------------------------------------------- conventional ray tracing at t (Sec. II)
 * DRT starts from the ray chains of one conventional ray-tracing run at t0 and re-runs it at every
 * multipath-lifetime boundary (Sec. II, Sec. IV-B).  This is that run by brute-force image-tree
 * enumeration: every chain of at most max_order reflections / diffractions (no primitive twice in a
 * row) and, if with_tiles, every single-tile scattering chain, posed at t, solved with the O-DRT
 * geometry (Newton for two diffractions in one segment, from the edge midpoints), kept when the chain
 * is valid (path_flags, as for the extrapolation) and no face blocks any of its segments. */

/* Does face f block the segment A -> B?  It does when the segment crosses the face's plane strictly
 * between its ends at a point inside the rectangle; a face whose plane holds A or B (the face a
 * reflection point or a tile lies on, the faces of a diffracting edge, faces coplanar with those)
 * does not.  *mg is lowered to the distance of this decision from its boundary (m). */
static int face_blocks(const or_scene *S, int f, double t, v3 A, v3 B, double *mg) {
    or_frame F;
    face_frame(S, f, t, &F);
    const or_face *fc = &S->faces[f];
    double ha = dot(sub(A, F.O.p), F.ey), hb = dot(sub(B, F.O.p), F.ey);
    if (fabs(ha) < 1e-9 || fabs(hb) < 1e-9) return 0;
    if ((ha > 0) == (hb > 0)) return 0;
    v3 X = add(A, scl(sub(B, A), ha / (ha - hb)));
    v3 r = sub(X, F.O.p);
    double al = dot(r, F.ex), be = dot(r, F.ez);
    double m = fmin(fabs(ha), fabs(hb));
    if (isfinite(fc->hu)) m = fmin(m, fabs(fc->hu - fabs(al)));
    if (isfinite(fc->hw)) m = fmin(m, fabs(fc->hw - fabs(be)));
    *mg = fmin(*mg, m);
    return fabs(al) <= fc->hu && fabs(be) <= fc->hw;
}

/* candidate k of the enumeration: 0 = line of sight; then the single interactions (faces as
 * reflections, edges as diffractions, tiles as scatterers); then the ordered pairs (a, b), a != b, of
 * faces and edges.  Returns 0 for a skipped index (a == b). */
static int trace_candidate(const or_scene *S, int64_t k, int with_tiles, or_path *pa) {
    const int NP = S->n_faces + S->n_edges, NT = with_tiles ? S->n_tiles : 0;
    memset(pa, 0, sizeof(*pa));
    if (k == 0) return 1;
    k -= 1;
    int code[2], n = 0;
    if (k < NP + NT) {
        code[n++] = (int)k;
    } else {
        k -= NP + NT;
        code[0] = (int)(k / NP);
        code[1] = (int)(k % NP);
        if (code[0] == code[1]) return 0;
        n = 2;
    }
    pa->n = n;
    for (int j = 0; j < n; ++j) {
        int c = code[j];
        if (c < S->n_faces) { pa->type[j] = OR_T_R; pa->prim[j] = c; }
        else if (c < NP) {
            const or_edge *e = &S->edges[c - S->n_faces];
            pa->type[j] = OR_T_D;
            pa->prim[j] = c - S->n_faces;
            pa->s0[j] = 0.5 * nrm(sub(V(e->b), V(e->a)));
        } else { pa->type[j] = OR_T_S; pa->prim[j] = c - NP; }
    }
    return 1;
}

int64_t or_trace_candidates(const or_scene *S, int32_t max_order, int32_t with_tiles) {
    const int64_t NP = S->n_faces + S->n_edges, NT = with_tiles ? S->n_tiles : 0;
    return 1 + (max_order >= 1 ? NP + NT : 0) + (max_order >= 2 ? NP * NP : 0);
}

/* Decision of candidate k at t: 1 when it is a ray; *margin is the smallest distance (m) of any of the
 * decisions (validity, occlusion) from its boundary; the chain and its diffraction parameters at t go
 * to *pa. */
static int trace_one(const or_scene *S, double t, int64_t k, int with_tiles, or_path *pa, double *margin) {
    *margin = INFINITY;
    if (!trace_candidate(S, k, with_tiles, pa)) return 0;
    or_geom G;
    odrt_solve(S, pa, t, &G);
    v3 P[OR_MAXI + 2];
    for (int i = 0; i <= pa->n + 1; ++i) P[i] = G.V[i].p;
    double mg;
    int fl = G.flags | path_flags(S, pa, t, P, &mg);
    *margin = mg;
    for (int i = 1; i <= pa->n; ++i)
        if (pa->type[i - 1] == OR_T_D) {
            or_frame F;
            double len, wn;
            edge_frame(S, pa->prim[i - 1], t, &F, &len, &wn);
            pa->s0[i - 1] = dot(sub(P[i], F.O.p), F.ez);
        }
    for (int i = 0; i <= pa->n + 1; ++i)
        if (!(isfinite(P[i].x) && isfinite(P[i].y) && isfinite(P[i].z))) fl |= OR_F_DEGEN;
    if (fl) return 0;
    int blocked = 0;
    for (int i = 1; i <= pa->n + 1; ++i)
        for (int f = 0; f < S->n_faces; ++f) blocked |= face_blocks(S, f, t, P[i - 1], P[i], margin);
    return !blocked;
}

typedef struct {
    const or_scene *S;
    double t;
    int32_t with_tiles, cap;
    int64_t total, next;
    double report;
    int32_t count;
    uint8_t *n_int, *types, *found;
    int32_t *prims;
    double *s0, *margin;
    int64_t *index;
    pthread_mutex_t mu;
} or_trjob;

static void *trace_worker(void *arg) {
    or_trjob *J = (or_trjob *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t lo = J->next;
        J->next += 256;
        pthread_mutex_unlock(&J->mu);
        if (lo >= J->total) break;
        int64_t hi = lo + 256 < J->total ? lo + 256 : J->total;
        for (int64_t k = lo; k < hi; ++k) {
            or_path pa;
            double mg;
            int ray = trace_one(J->S, J->t, k, J->with_tiles, &pa, &mg);
            if (!ray && !(mg < J->report)) continue;
            pthread_mutex_lock(&J->mu);
            int slot = J->count++;
            pthread_mutex_unlock(&J->mu);
            if (slot >= J->cap) continue;
            J->index[slot] = k;
            J->found[slot] = (uint8_t)ray;
            J->margin[slot] = mg;
            J->n_int[slot] = (uint8_t)pa.n;
            for (int j = 0; j < OR_MAXI; ++j) {
                J->types[slot * OR_MAXI + j] = (uint8_t)(j < pa.n ? pa.type[j] : 0);
                J->prims[slot * OR_MAXI + j] = j < pa.n ? pa.prim[j] : -1;
                J->s0[slot * OR_MAXI + j] = j < pa.n ? pa.s0[j] : 0.0;
            }
        }
    }
    return NULL;
}

/* Ray tracing at t: writes (in no particular order) every candidate that is a ray (found = 1) and every
 * other candidate whose decision margin is below `report` m (found = 0: a run at this instant could
 * decide it either way), with its enumeration index, margin, chain and diffraction parameters at t.
 * Returns the number of such candidates (only the first cap are written). */
int32_t or_trace(const or_scene *S, double t, int32_t max_order, int32_t with_tiles, double report, int32_t n_threads,
                 int32_t cap, int64_t *index, uint8_t *found, double *margin, uint8_t *n_int, uint8_t *types,
                 int32_t *prims, double *s0) {
    pthread_once(&gl_once, gl_init);
    or_trjob J;
    memset(&J, 0, sizeof(J));
    J.S = S; J.t = t; J.with_tiles = with_tiles; J.cap = cap; J.report = report;
    J.total = or_trace_candidates(S, max_order, with_tiles);
    J.n_int = n_int; J.types = types; J.found = found; J.prims = prims; J.s0 = s0; J.margin = margin; J.index = index;
    pthread_mutex_init(&J.mu, NULL);
    int nt = n_threads < 1 ? 1 : n_threads > 256 ? 256 : n_threads;
    pthread_t th[256];
    for (int i = 0; i < nt; ++i) pthread_create(&th[i], NULL, trace_worker, &J);
    for (int i = 0; i < nt; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.mu);
    return J.count;
}

/* ---------------------------------------------------------------- unit-level entry points for pins */
void or_fresnel_coeffs(double eps_r, double sigma, double pec, double fc, double ct, double *out4) {
    or_mat m = {eps_r, sigma, 0.0, pec};
    double complex a, b;
    fresnel(&m, fc, ct, &a, &b);
    out4[0] = creal(a); out4[1] = cimag(a); out4[2] = creal(b); out4[3] = cimag(b);
}
void or_fresnel_G_ri(double x, double *out2) { double complex g = or_fresnel_G(x); out2[0] = creal(g); out2[1] = cimag(g); }
void or_transition_F_ri(double X, double *out2) { double complex g = or_transition_F(X); out2[0] = creal(g); out2[1] = cimag(g); }
void or_utd_ri(double n, double phi, double phip, double sinb0, double L, double k, double eps_r, double sigma,
               double pec, double fc, double *out4) {
    or_mat m = {eps_r, sigma, 0.0, pec};
    double complex a, b;
    or_utd(n, phi, phip, sinb0, L, k, &m, fc, &a, &b);
    out4[0] = creal(a); out4[1] = cimag(a); out4[2] = creal(b); out4[3] = cimag(b);
}
/* Body-point state at t (pins of Eq. RigidBodyMotion against differentiated poses). */
void or_body_point(const or_body *b, const double *p0, double t, double *out9) {
    or_pose P;
    body_pose(b, t, &P);
    kst s = pose_point(&P, V(p0));
    out9[0] = s.p.x; out9[1] = s.p.y; out9[2] = s.p.z;
    out9[3] = s.v.x; out9[4] = s.v.y; out9[5] = s.v.z;
    out9[6] = s.a.x; out9[7] = s.a.y; out9[8] = s.a.z;
}
/* Round trip world -> face frame -> world of a kinematic state (Eqs. relative_vel/acc followed by
 * global_vel/acc_ref_point). */
void or_frame_roundtrip(const or_scene *S, int32_t face, double t, const double *in9, double *local9, double *out9) {
    or_frame F;
    face_frame(S, face, t, &F);
    kst X = {V(in9), V(in9 + 3), V(in9 + 6)};
    kst L = to_local(&F, X), Y = from_local(&F, L);
    double *o = local9;
    o[0] = L.p.x; o[1] = L.p.y; o[2] = L.p.z; o[3] = L.v.x; o[4] = L.v.y; o[5] = L.v.z; o[6] = L.a.x; o[7] = L.a.y; o[8] = L.a.z;
    o = out9;
    o[0] = Y.p.x; o[1] = Y.p.y; o[2] = Y.p.z; o[3] = Y.v.x; o[4] = Y.v.y; o[5] = Y.v.z; o[6] = Y.a.x; o[7] = Y.a.y; o[8] = Y.a.z;
}
/* Eq. ref_point on jets in a wall frame given local states of T and R (9 doubles each). */
void or_ref_point_local(const double *t9, const double *r9, double *q9) {
    kst T = {V(t9), V(t9 + 3), V(t9 + 6)}, R = {V(r9), V(r9 + 3), V(r9 + 6)};
    kst Q = ref_point_local(T, R);
    q9[0] = Q.p.x; q9[1] = Q.p.y; q9[2] = Q.p.z; q9[3] = Q.v.x; q9[4] = Q.v.y; q9[5] = Q.v.z; q9[6] = Q.a.x; q9[7] = Q.a.y; q9[8] = Q.a.z;
}
void or_diff_point_local(const double *t9, const double *r9, double *q9) {
    kst T = {V(t9), V(t9 + 3), V(t9 + 6)}, R = {V(r9), V(r9 + 3), V(r9 + 6)};
    kst Q = diff_point_local(T, R);
    q9[0] = Q.p.x; q9[1] = Q.p.y; q9[2] = Q.p.z; q9[3] = Q.v.x; q9[4] = Q.v.y; q9[5] = Q.v.z; q9[6] = Q.a.x; q9[7] = Q.a.y; q9[8] = Q.a.z;
}
/* Doppler of an explicit vertex chain (positions + velocities, n+2 vertices). */
double or_doppler_chain(int32_t n, const double *pos, const double *vel, double fc) {
    kst Vx[OR_MAXI + 2];
    for (int i = 0; i <= n + 1; ++i) { Vx[i].p = V(pos + 3 * i); Vx[i].v = V(vel + 3 * i); Vx[i].a = mk(0, 0, 0); }
    return path_doppler(n, Vx, fc);
}
