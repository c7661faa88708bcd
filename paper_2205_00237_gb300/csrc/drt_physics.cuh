// drt_physics.cuh -- per-(path, time-step) device work of the DRT hot path: posing primitives on
// moving bodies, the interaction points (image method and back-tracking, Keller cone, rigid
// tiles, Newton for several diffractions in one segment), validity, Doppler and the field
// coefficients.  Templated on the working precision T; positions carry their time derivative as
// dual numbers so interaction-point velocities come out of the same arithmetic.
#pragma once
// rarely executed code (multi-diffraction Newton, the transition function near shadow boundaries,
// user-output writes) is kept out of line so the hot per-step code stays dense in the instruction
// cache (canyon FP32-bulk step 0.36 -> 0.27 ms)
#define DRT_OUTLINE __host__ __device__ __noinline__
#include <type_traits>
#include "drt_internal.h"
#include "drt_fnodes.h"
#include "drt_math.cuh"

namespace drt {

constexpr double C0 = 299792458.0;
constexpr double EPS0 = 8.8541878128e-12;
constexpr double PI = 3.14159265358979323846;

enum : uint32_t { F_FACE = 1, F_EDGE = 2, F_SIDE = 4, F_NOCONV = 8, F_DEGEN = 16 };
// internal: the FP32-bulk solve met a geometry it cannot resolve in FP32 (near-grazing Keller cone,
// unconverged Newton, non-finite value); the path-step is redone in FP64.  Never written out.
constexpr uint32_t F_REDO64 = 128;
// internal: some FP32 validity margin lies within 100x the FP32 error bound (fp32_margin_tol)
constexpr uint32_t F_NEAR100 = 64;

enum : int { T_NONE = 0, T_R = 1, T_D = 2, T_S = 3 };

// ------------------------------------------------------------------------------------------------
// posing (Sec. III-A: rotation about a fixed axis, Eq. RigidBodyMotion for body-point velocity)
template <class T> struct Pose { v3<T> R0, R1, R2, O, vO, w; };   // rows of R

template <class T> DRT_HD Pose<T> load_pose(const double *P) {
    Pose<T> q;
    q.R0 = V3<T>(P[0], P[1], P[2]);
    q.R1 = V3<T>(P[3], P[4], P[5]);
    q.R2 = V3<T>(P[6], P[7], P[8]);
    q.O = V3<T>(P[9], P[10], P[11]);
    q.vO = V3<T>(P[12], P[13], P[14]);
    q.w = V3<T>(P[15], P[16], P[17]);
    return q;
}
template <class T> DRT_HD v3<T> rot(const Pose<T> &q, const double *a) {
    v3<T> x = V3<T>(a[0], a[1], a[2]);
    return V3<T>(dot(q.R0, x), dot(q.R1, x), dot(q.R2, x));
}
// body point that sat at o + rel at t0: position O + R rel, velocity v_O + w x (R rel)
template <class T> DRT_HD v3<dl<T>> pose_point(const Pose<T> &q, const double *rel) {
    v3<T> r = rot(q, rel);
    return dual(q.O + r, q.vO + cross(q.w, r));
}
// body-fixed direction: R d0, derivative w x (R d0)
template <class T> DRT_HD v3<dl<T>> pose_dir(const Pose<T> &q, const double *d0) {
    v3<T> n = rot(q, d0);
    return dual(n, cross(q.w, n));
}

// pose record of one body at time t (seconds after t0): theta(t) = w0 t + wdot t^2 / 2 about the fixed
// axis k (Rodrigues), O(t) by Eq. Taylor, v_O(t) = v + a t, omega(t) = (w0 + wdot t) k
DRT_HD void body_pose_row(const BodyD &B, double t, double *P) {
    double th = B.w0 * t + 0.5 * B.wdot * t * t, ws = B.w0 + B.wdot * t;
    double s = sin(th), c = cos(th);
    double C1 = 1.0 - c, kx = B.k[0], ky = B.k[1], kz = B.k[2];
    P[0] = c + kx * kx * C1;      P[1] = kx * ky * C1 - kz * s; P[2] = kx * kz * C1 + ky * s;
    P[3] = ky * kx * C1 + kz * s; P[4] = c + ky * ky * C1;      P[5] = ky * kz * C1 - kx * s;
    P[6] = kz * kx * C1 - ky * s; P[7] = kz * ky * C1 + kx * s; P[8] = c + kz * kz * C1;
    for (int j = 0; j < 3; ++j) {
        P[9 + j] = B.o[j] + B.v[j] * t + 0.5 * B.a[j] * t * t;
        P[12 + j] = B.v[j] + B.a[j] * t;
        P[15 + j] = B.k[j] * ws;
    }
}

// terminal state (Eq. Taylor)
template <class T> DRT_HD v3<dl<T>> terminal(const TermD &m, T t) {
    v3<T> r = V3<T>(m.r[0], m.r[1], m.r[2]), v = V3<T>(m.v[0], m.v[1], m.v[2]), a = V3<T>(m.a[0], m.a[1], m.a[2]);
    return dual(r + v * t + a * (T(0.5) * t * t), v + a * t);
}

// ------------------------------------------------------------------------------------------------
// interaction points, generic over the scalar S (dl<double> for the FP64 form, dd for FP32-bulk)
// Eq. ref_point in vector form: tangential coordinates interpolated between source S and
// receiver R with weight h_S / (h_S + h_R) (h = height above the wall), normal coordinate 0.
template <class S> DRT_HD v3<S> refl_point(v3<S> Sv, v3<S> Rv, v3<S> c, v3<S> n) {
    S hs = dot(Sv - c, n), hr = dot(Rv - c, n);
    S g = hs / (hs + hr);
    v3<S> Q = Sv + (Rv - Sv) * g;
    return Q - n * dot(Q - c, n);
}
// image of X across the wall (c, n)
template <class S> DRT_HD v3<S> mirror(v3<S> X, v3<S> c, v3<S> n) {
    S h = dot(X - c, n);
    return X - n * (h + h);
}
template <class S> DRT_HD v3<S> mirror_dir(v3<S> d, v3<S> n) {
    S h = dot(d, n);
    return d - n * (h + h);
}

// posed primitives of one chain vertex
template <class S> struct Prim {
    typedef typename ST<S>::R T;
    int type, mat;
    v3<S> p;        // R: face centre, D: edge point a, S: tile centroid
    v3<S> a;        // R: face normal, D: edge direction, S: tile normal
    v3<T> b;        // R: face axis u, D: 0-face tangent t0 = n0 x e
    v3<T> c;        // D: 0-face normal n0
    T h1, h2;       // R: hu, hw; D: length, wedge n
    T h3, h4;       // D: sin(n pi), cos(n pi) (the n-face direction in the (t0, n0) plane)
    int idx;
};

// pose table layout [body][time-step][POSE_W]: the 32 lanes of a warp (consecutive time steps of
// one path) read one contiguous 4.6 KB stretch per body
DRT_HD const double *pose_at(const double *pose, int n_steps, int body, int ti) {
    return pose + ((size_t)body * n_steps + ti) * POSE_W;
}

// FP64 form: primitive posed from the pose record `P` of its body
template <class T>
DRT_HD Prim<dl<T>> load_prim_row(const LinkDev &L, const double *Prow, int type, int idx) {
    Prim<dl<T>> q;
    q.type = type;
    q.idx = idx;
    Pose<T> P = load_pose<T>(Prow);
    if (type == T_R) {
        const FaceD &f = L.faces[idx];
        q.p = pose_point(P, f.c);
        q.a = pose_dir(P, f.n);
        q.b = rot(P, f.u);
        q.h1 = T(f.hu);
        q.h2 = T(f.hw);
        q.mat = f.mat;
    } else if (type == T_D) {
        const EdgeD &e = L.edges[idx];
        q.p = pose_point(P, e.a);
        q.a = pose_dir(P, e.e);
        q.b = rot(P, e.t0);
        q.c = rot(P, e.n0);
        q.h1 = T(e.len);
        q.h2 = T(e.wn);
        q.h3 = T(e.snp);
        q.h4 = T(e.cnp);
        q.mat = e.mat;
    } else {
        const TileD &tl = L.tiles[idx];
        q.p = pose_point(P, tl.c);
        q.a = pose_dir(P, tl.n);
        q.mat = tl.mat;
    }
    return q;
}

DRT_HD int prim_body(const LinkDev &L, int type, int idx) {
    return type == T_R ? L.faces[idx].body : type == T_D ? L.edges[idx].body : L.tiles[idx].body;
}

// A primitive of a body at rest: its t0 placement at every instant, with zero rates.  This is what
// posing gives for such a body (identity rotation, O = o, no velocity) without the pose record or
// the rotations: most primitives of the synthetic scenes (facades, their edges and tiles, the ground)
// are at rest.
template <class T> DRT_HD Prim<dl<T>> load_prim_fixed(const LinkDev &L, int type, int idx) {
    Prim<dl<T>> q;
    q.type = type;
    q.idx = idx;
    const double *o = L.bodies[prim_body(L, type, idx)].o;
    const v3<T> zero = V3<T>(T(0), T(0), T(0));
    auto at = [&](const double *rel) { return dual(V3<T>(o[0] + rel[0], o[1] + rel[1], o[2] + rel[2]), zero); };
    auto dir = [&](const double *d) { return dual(V3<T>(d[0], d[1], d[2]), zero); };
    if (type == T_R) {
        const FaceD &f = L.faces[idx];
        q.p = at(f.c);
        q.a = dir(f.n);
        q.b = V3<T>(f.u[0], f.u[1], f.u[2]);
        q.h1 = T(f.hu);
        q.h2 = T(f.hw);
        q.mat = f.mat;
    } else if (type == T_D) {
        const EdgeD &e = L.edges[idx];
        q.p = at(e.a);
        q.a = dir(e.e);
        q.b = V3<T>(e.t0[0], e.t0[1], e.t0[2]);
        q.c = V3<T>(e.n0[0], e.n0[1], e.n0[2]);
        q.h1 = T(e.len);
        q.h2 = T(e.wn);
        q.h3 = T(e.snp);
        q.h4 = T(e.cnp);
        q.mat = e.mat;
    } else {
        const TileD &tl = L.tiles[idx];
        q.p = at(tl.c);
        q.a = dir(tl.n);
        q.mat = tl.mat;
    }
    return q;
}

// FP64 form: primitives posed from the pose table
template <class T>
DRT_HD Prim<dl<T>> load_prim(const LinkDev &L, const double *pose, int n_steps, int ti, int type, int idx) {
    const int body = prim_body(L, type, idx);
    if (L.body_fixed[body]) return load_prim_fixed<T>(L, type, idx);
    return load_prim_row<T>(L, pose_at(pose, n_steps, body, ti), type, idx);
}

// FP64 primitive posed directly from the body kinematics at time t (FP32-bulk redo path)
template <class T>
DRT_HD Prim<dl<T>> load_prim_direct(const LinkDev &L, double t, int type, int idx) {
    const int body = prim_body(L, type, idx);
    if (L.body_fixed[body]) return load_prim_fixed<T>(L, type, idx);
    double P[POSE_W];
    body_pose_row(L.bodies[body], t, P);
    return load_prim_row<T>(L, P, type, idx);
}

// Keller-cone point on the edge line (A, e) between a virtual source and a virtual receiver:
// s = s_A + (s_B - s_A) rho_A / (rho_A + rho_B), the 3D form of Eq. diff_point.
template <class S>
DRT_HD S keller_s(v3<S> Sv, v3<S> Rv, const Prim<S> &e, uint32_t &fl) {
    typedef typename ST<S>::R T;
    v3<S> wa = Sv - e.p, wb = Rv - e.p;
    S sa = dot(wa, e.a), sb = dot(wb, e.a);
    v3<S> pa = wa - e.a * sa, pb = wb - e.a * sb;
    T ra2 = dot(val(pa), val(pa)), rb2 = dot(val(pb), val(pb));
    if (!(ra2 > T(1e-24)) || !(rb2 > T(1e-24))) {
        fl |= F_DEGEN;
        return sa;
    }
    // near grazing (a virtual terminal within 1 mm of the edge line) FP32 cannot resolve the cone
    if (sizeof(T) == 4 && (ra2 < T(1e-6) || rb2 < T(1e-6))) fl |= F_REDO64;
    S ra = norm(pa), rb = norm(pb);
    return sa + (sb - sa) * ra / (ra + rb);
}

template <class S> DRT_HD void clamp_positive(S &x, typename ST<S>::R eps);
template <> DRT_HD void clamp_positive<dl<double>>(dl<double> &x, double eps) {
    if (!(x.v > eps)) x.v = eps;
}
template <> DRT_HD void clamp_positive<double>(double &x, double eps) {
    if (!(x > eps)) x = eps;
}
template <> DRT_HD void clamp_positive<float>(float &x, float eps) {
    if (!(x > eps)) x = eps;
}
template <> DRT_HD void clamp_positive<de>(de &x, float eps) {
    if (!(x.b + x.d > eps)) {
        x.b = eps;
        x.d = 0.f;
    }
}
template <> DRT_HD void clamp_positive<dd>(dd &x, float eps) {
    if (!(x.b + x.d > eps)) {
        x.b = eps;
        x.d = 0.f;
    }
}

// Newton start for an edge parameter from its value `base` + `delta` and rate: for delta numbers
// the base part is `base` (the chunk-base solution) and the delta `delta`
template <class S> DRT_HD S newton_start(double base, double delta, double rate);
template <> DRT_HD double newton_start<double>(double base, double delta, double) { return base + delta; }
template <> DRT_HD float newton_start<float>(double base, double delta, double) { return (float)(base + delta); }
template <> DRT_HD dl<double> newton_start<dl<double>>(double base, double delta, double rate) {
    return {base + delta, rate};
}
template <> DRT_HD de newton_start<de>(double base, double delta, double) { return {(float)base, (float)delta}; }
template <> DRT_HD dd newton_start<dd>(double base, double delta, double rate) {
    return {(float)base, (float)delta, (float)rate};
}

// the same from an FP32 offset and rate (the FP32-bulk steps' warm starts): no FP64 arithmetic
template <class S> DRT_HD S newton_start_f(double base, float delta, float rate);
template <> DRT_HD de newton_start_f<de>(double base, float delta, float) { return {(float)base, delta}; }
template <> DRT_HD dd newton_start_f<dd>(double base, float delta, float rate) { return {(float)base, delta, rate}; }

// chain length of path p (vertices before the first empty type byte)
DRT_HD int chain_length(const LinkDev &L, int p) {
    const uint32_t c = L.ptypes[p];
    return (c & 0xffu) == 0 ? 0 : (c & 0xff00u) == 0 ? 1 : (c & 0xff0000u) == 0 ? 2 : (c & 0xff000000u) == 0 ? 3 : 4;
}

// The solvers below run on chains of N vertices, N known at compile time: every vertex loop has a
// fixed bound and unrolls, so the per-vertex arrays (positions, images, Newton state) are indexed by
// constants and stay in registers; the chain's interaction types are read at run time.

// tile centroids move rigidly with their bodies (Sec. III-C)
template <int N, class S> DRT_HD void place_tiles(const Prim<S> *pr, v3<S> *V) {
#pragma unroll
    for (int i = 1; i <= N; ++i)
        if (pr[i - 1].type == T_S) V[i] = pr[i - 1].p;
}

// Keller-cone points of the diffractions that are alone between their point sources: each lies on
// the cone between its virtual source (the segment's left point source imaged through the
// reflections in between) and its virtual receiver (the right point source imaged backwards through
// the reflections after it).  Vertices with nv[i] set were placed by the Newton solve.
template <int N, class S>
DRT_HD void place_keller(const Prim<S> *pr, v3<S> *V, uint32_t &fl, const bool *nv) {
    v3<S> img[N > 0 ? N : 1];
    v3<S> cur = V[0];
#pragma unroll
    for (int i = 1; i <= N; ++i) {
        const Prim<S> &q = pr[i - 1];
        if (q.type == T_D) img[i - 1] = cur;
        else if (q.type == T_R) cur = mirror(cur, q.p, q.a);
        else cur = V[i];
    }
    cur = V[N + 1];
#pragma unroll
    for (int i = N; i >= 1; --i) {
        const Prim<S> &q = pr[i - 1];
        if (q.type == T_D && !(nv && nv[i])) V[i] = q.p + q.a * keller_s(img[i - 1], cur, q, fl);
        else if (q.type == T_R) cur = mirror(cur, q.p, q.a);
        else cur = V[i];
    }
}

// reflection points by back-tracking (Sec. III-A.2) between the known points (point sources and
// diffraction points): a wall's source image is the last known point imaged through the walls
// before it; the points are placed from the right, each by Eq. ref_point towards the point placed
// before it
template <int N, class S> DRT_HD void place_reflections(const Prim<S> *pr, v3<S> *V) {
    v3<S> img[N > 0 ? N : 1];
    v3<S> cur = V[0];
#pragma unroll
    for (int i = 1; i <= N; ++i) {
        const Prim<S> &q = pr[i - 1];
        if (q.type == T_R) {
            img[i - 1] = cur;
            cur = mirror(cur, q.p, q.a);
        } else {
            cur = V[i];
        }
    }
    v3<S> next = V[N + 1];
#pragma unroll
    for (int i = N; i >= 1; --i) {
        const Prim<S> &q = pr[i - 1];
        if (q.type == T_R) V[i] = refl_point(img[i - 1], next, q.p, q.a);
        next = V[i];
    }
}

// Edge parameters of the diffractions of a segment with two or more of them (the reading of Sec.
// III-B for multiple diffraction): Newton on the unfolded length of the segment -- the stationary,
// here minimal, path, with the reflections between diffraction points unfolded by imaging -- using
// its analytic tridiagonal Hessian, started from s0 (+ ds0, at rate rate0).  The length is convex in
// the edge parameters, so a step that lengthens the path is halved until it does not (backtracking
// line search).  Carried on dual numbers, the converged iterate's derivative is the implicit-function
// derivative, so the diffraction points' sliding velocities come out of the same solve.
// The unknowns are indexed by their vertex (nv[i]).  One sweep over the vertices meets the legs of
// the unfolded path in order (a leg runs from an anchor -- point source or unknown diffraction point
// -- to the next, through the reflections in between) and eliminates each unknown of the
// tridiagonal system at the anchor that closes its outgoing leg; the back substitution runs the
// other way.  Nothing is indexed at run time.
template <int N, class S, class D = double>
DRT_HD void newton_diffractions(const Prim<S> *pr, v3<S> *V, const bool *nv, const double *s0, const D *ds0,
                                const D *rate0, uint32_t &fl) {
    typedef typename ST<S>::R T;
    // convergence threshold on the Newton step (m): near round-off of the working precision
    const T tol = sizeof(T) == 8 ? T(1e-10) : T(1e-4);
    // below this step (m) the length change of a Newton step is at round-off of the ~100 m path
    // length, so the backtracking test is only applied to larger steps
    const T ls_min = sizeof(T) == 8 ? T(1e-4) : T(1e-2);
    const S zero = scst<S>(T(0)), one = scst<S>(T(1));
    S s[N + 1], step[N + 1];
#pragma unroll
    for (int i = 1; i <= N; ++i)
        if (nv[i]) {
            if constexpr (std::is_same<D, float>::value)
                s[i] = newton_start_f<S>(s0[i - 1], ds0 ? ds0[i - 1] : 0.f, rate0 ? rate0[i - 1] : 0.f);
            else
                s[i] = newton_start<S>(s0[i - 1], ds0 ? ds0[i - 1] : 0.0, rate0 ? rate0[i - 1] : 0.0);
            step[i] = zero;
        }
    bool conv = false;
    int halvings = 0;
    T Lprev = T(0), smax_prev = T(0);
    bool have_prev = false;
    for (int it = 0; it < 64; ++it) {
        // cpS[i], dpS[i]: elimination of the unknown whose outgoing leg ends at anchor i (cl[i])
        S cpS[N + 2], dpS[N + 2];
        bool cl[N + 2];
        v3<S> X = V[0], ex = V[0];   // the leg's start imaged through its walls so far; its edge alike
        bool startN = false, first = true;
        // gk, hk: gradient and Hessian diagonal of the unknown starting the current leg; hop: its
        // coupling to the unknown before it; cpP, dpP: elimination of that previous unknown
        S Lc = zero, gk = zero, hk = zero, hop = zero, cpP = zero, dpP = zero;
#pragma unroll
        for (int i = 1; i <= N + 1; ++i) {
            cl[i] = false;
            const int ty = i <= N ? pr[i - 1].type : T_S;   // vertex N + 1 is RX, a point source
            const bool var = i <= N && nv[i];
            if (ty == T_R) {
                X = mirror(X, pr[i - 1].p, pr[i - 1].a);
                if (startN) ex = mirror_dir(ex, pr[i - 1].a);
                continue;
            }
            if (ty == T_D && !var) {   // a Keller diffraction: its segment has no unknowns
                startN = false;
                continue;
            }
            const v3<S> Y = var ? pr[i - 1].p + pr[i - 1].a * s[i] : V[i];
            if (startN || var) {
                const v3<S> r = X - Y;
                const S l = norm(r);
                Lc = Lc + l;
                const S il = one / l;
                const v3<S> rh = r * il;
                S qs = zero, gi = zero, hi = zero, hoi = zero;
                if (startN) {
                    qs = dot(rh, ex);
                    gk = gk + qs;
                    hk = hk + (one - qs * qs) * il;
                }
                if (var) {
                    const S q = dot(rh, pr[i - 1].a);
                    gi = zero - q;
                    hi = (one - q * q) * il;
                    if (startN) hoi = (qs * q - dot(ex, pr[i - 1].a)) * il;
                }
                if (startN) {   // the unknown starting this leg has all its terms: eliminate it
                    clamp_positive(hk, T(1e-12));
                    S cp, dp;
                    if (first) {
                        cp = hoi / hk;
                        dp = -gk / hk;
                    } else {
                        const S den = hk - hop * cpP;
                        cp = hoi / den;
                        dp = (-gk - hop * dpP) / den;
                    }
                    first = false;
                    cpS[i] = cp;
                    dpS[i] = dp;
                    cl[i] = true;
                    cpP = cp;
                    dpP = dp;
                }
                if (var) {
                    gk = gi;
                    hk = hi;
                    hop = hoi;
                }
            }
            X = Y;
            if (var) ex = pr[i - 1].a;
            startN = var;
        }
        if (have_prev && smax_prev > ls_min && !(sval(Lc) <= Lprev) && halvings < 40) {
#pragma unroll
            for (int i = 1; i <= N; ++i)
                if (nv[i]) {   // backtrack: s_prev + step / 2
                    step[i] = step[i] * T(0.5);
                    s[i] = s[i] - step[i];
                }
            smax_prev *= T(0.5);
            ++halvings;
            continue;
        }
        halvings = 0;
        Lprev = sval(Lc);
        have_prev = true;
        // back substitution from the right: the step computed at the anchor closing an unknown's
        // outgoing leg is applied when the sweep reaches that unknown
        S x[N + 1];
        S xp = zero, xn = zero;
        T smax = T(0);
#pragma unroll
        for (int i = N + 1; i >= 1; --i) {
            const bool var = i <= N && nv[i];
            if (var) {
                x[i] = xp;
                xn = xp;
                smax = fmax(smax, fabs(sval(xp)));
            }
            if (cl[i]) xp = var ? dpS[i] - cpS[i] * xn : dpS[i];
        }
        if (!(smax == smax)) break;   // NaN
#pragma unroll
        for (int i = 1; i <= N; ++i)
            if (nv[i]) {
                s[i] = s[i] + x[i];
                step[i] = x[i];
            }
        smax_prev = smax;
        // On dual numbers one Newton step from a value within smax of the root leaves the
        // derivative part O(smax) from the implicit-function derivative whatever the start's
        // derivative was, so FP64 stops at the first step below tol (1e-10 m); FP32 with rates
        // (tol 1e-4 m) takes one more step to refine both parts.  FP32 delta numbers without rates
        // stop at once: by Newton's quadratic convergence the value is then within ~K smax^2 of the
        // root (K of the order of an inverse leg length, larger near grazing), and from the FP64
        // warm starts the first step is ~1e-6..1e-5 m (the FP32 rounding of the coordinates), so the
        // remaining error is far below that rounding.
        if (conv) break;
        if (smax < tol) {
            conv = true;
            if (sizeof(T) == 8 || std::is_same<S, de>::value) break;
        }
    }
    if (!conv) fl |= F_NOCONV;
#pragma unroll
    for (int i = 1; i <= N; ++i)
        if (nv[i]) V[i] = pr[i - 1].p + pr[i - 1].a * s[i];
}

// chains with at most one diffraction between point sources (nearly every chain)
template <int N, class S>
DRT_HD void solve_geometry_fast(const Prim<S> *pr, v3<S> *V, uint32_t &fl) {
    static_assert(N >= 0 && N <= MAXI, "chain length");
    place_tiles<N>(pr, V);
    bool has_d = false;
#pragma unroll
    for (int i = 1; i <= N; ++i) has_d = has_d || pr[i - 1].type == T_D;
    if (has_d) place_keller<N>(pr, V, fl, nullptr);
    place_reflections<N>(pr, V);
}

// any chain of N vertices: the diffractions of a segment with two or more of them by Newton (their
// start values s0 [+ ds0, rate0] indexed by vertex - 1), the others on their Keller cones
template <int N, class S, class D = double>
DRT_HD void solve_geometry_any(const Prim<S> *pr, v3<S> *V, const double *s0, uint32_t &fl,
                               const D *ds0 = nullptr, const D *rate0 = nullptr) {
    static_assert(N >= 0 && N <= MAXI, "chain length");
    place_tiles<N>(pr, V);
    // diffractions per segment: running count from the left, then each segment's total from the right
    int cf[N + 1];
    int c = 0;
#pragma unroll
    for (int i = 1; i <= N; ++i) {
        const int ty = pr[i - 1].type;
        c = ty == T_S ? 0 : c + (ty == T_D ? 1 : 0);
        cf[i] = c;
    }
    bool nv[N + 1];
    bool any_nv = false, any_single = false;
    int run = -1;
#pragma unroll
    for (int i = N; i >= 1; --i) {
        const int ty = pr[i - 1].type;
        if (ty == T_S) run = -1;
        else if (run < 0) run = cf[i];
        nv[i] = ty == T_D && run >= 2;
        any_nv = any_nv || nv[i];
        any_single = any_single || (ty == T_D && run == 1);
    }
    if constexpr (N >= 2)   // two diffractions need two vertices
        if (any_nv) newton_diffractions<N>(pr, V, nv, s0, ds0, rate0, fl);
    if (any_single) place_keller<N>(pr, V, fl, nv);
    place_reflections<N>(pr, V);
}

// MULTI: the chain may have several diffractions between point sources
template <int N, bool MULTI, class S, class D = double>
DRT_HD void solve_geometry(const Prim<S> *pr, v3<S> *V, const double *s0, uint32_t &fl,
                           const D *ds0 = nullptr, const D *rate0 = nullptr) {
    static_assert(N >= 0 && N <= MAXI, "chain length");
    if constexpr (MULTI) solve_geometry_any<N>(pr, V, s0, fl, ds0, rate0);
    else solve_geometry_fast<N>(pr, V, fl);
}

// Chain length as a template argument: N >= 0 a fixed length; LEN_ANY the length read at run time
// (one instance per length); LEN_GEN the same for the chains of the generic range (several
// diffractions in a segment, or 4 vertices), which have at least 2 vertices.
constexpr int LEN_ANY = -1, LEN_GEN = -2;

// one instance of f per chain length: f(std::integral_constant<int, N>) for N = n; lengths below
// NMIN have no instance (nothing runs for them)
static_assert(MAXI == 4, "with_length covers the lengths 0..4");
template <int NMIN = 0, class F> DRT_HD void with_length(int n, F &&f) {
    switch (n) {
    case 0: if constexpr (NMIN <= 0) f(std::integral_constant<int, 0>()); break;
    case 1: if constexpr (NMIN <= 1) f(std::integral_constant<int, 1>()); break;
    case 2: if constexpr (NMIN <= 2) f(std::integral_constant<int, 2>()); break;
    case 3: if constexpr (NMIN <= 3) f(std::integral_constant<int, 3>()); break;
    default: f(std::integral_constant<int, MAXI>()); break;
    }
}
template <int N> constexpr int len_min() { return N == LEN_GEN ? 2 : 0; }
// validity (Sec. II: the t0 multipath structure still holds): reflection points inside their
// faces with both neighbours in front, diffraction points on their edge segments with both
// neighbours in the wedge exterior, tiles lit from and seen from the front.
// In FP32 (the FP32-bulk form) the positions carry rounding errors of a few ulp of the coordinates,
// amplified a little by the image construction, so a decision whose margin (the distance of the tested
// point from the face rim, the edge end, the face plane or the wedge face) is within a bound on that
// error is not taken here: the step gets F_REDO64 and the FP64 redo decides it, which makes the flags
// of the form exact outside the 1e-9 m band of the FP64 form.  F_NEAR100 marks margins within 100x
// that bound (the FP32-bulk step uses it to keep the FP32 flags of invalid steps that moved far).
template <class T> DRT_HD T amax3(v3<T> a) { return fmax(fmax(fabs(a.x), fabs(a.y)), fabs(a.z)); }
// bound on the FP32 error of a margin computed from positions of magnitude `scale` (m): 2e-6 of the
// scale is ~17 ulp of the largest coordinate; the FP32 flags of the canyon, link and highway workloads
// were found exact outside 1e-4 m of every boundary without this test (coordinates up to ~600 m)
DRT_HD float fp32_margin_tol(float scale) { return 2e-6f * (scale + 1.f); }

// Vertex loops run over a fixed bound (MAXI) and stop at the chain length, so their array indices
// are constants after unrolling and the arrays stay in registers; N >= 0 fixes the length at compile
// time (every caller now passes a fixed N; N < 0 would take the run-time n).
// The tests at one vertex of type ty (c, nn: its point and normal or edge direction; b, cc, h1..h4 as
// in Prim) between its neighbours Pm, Pp: its flag bits, and (FP32) its smallest margin over the FP32
// error bound.  (Called out of line in the FP32 kernels it measured no faster, unlike the field
// updates, so it stays inline.)
template <class T> struct VertexCheck { uint32_t fl; T m; };
template <class T>
DRT_HD VertexCheck<T> vertex_validity_inl(int ty, v3<T> c, v3<T> nn, v3<T> b, v3<T> cc, T h1, T h2, T h3, T h4,
                                          v3<T> Pm, v3<T> Pi, v3<T> Pp) {
    constexpr bool F32 = sizeof(T) == 4;
    uint32_t fl = 0;
    T mmin = T(1e30);
    if (ty == T_R) {
        v3<T> r = Pi - c;
        T al = dot(r, b), be = dot(r, cross(b, nn));
        if (fabs(al) > h1 || fabs(be) > h2) fl |= F_FACE;
        const T dp = dot(Pm - c, nn), dn = dot(Pp - c, nn);
        if (!(dp > T(0)) || !(dn > T(0))) fl |= F_SIDE;
        if constexpr (F32) {
            const T tol = fp32_margin_tol(fmax(fmax(amax3(Pm), amax3(Pp)), fmax(amax3(Pi), amax3(c))));
            mmin = fmin(fmin(fabs(fabs(al) - h1), fabs(fabs(be) - h2)), fmin(fabs(dp), fabs(dn))) / tol;
        }
    } else if (ty == T_D) {
        const v3<T> A = c, e = nn;
        T s = dot(Pi - A, e);
        if (s < T(0) || s > h1) fl |= F_EDGE;
        T tol = T(0);
        if constexpr (F32) {
            tol = fp32_margin_tol(fmax(fmax(amax3(Pm), amax3(Pp)), fmax(amax3(Pi), amax3(A))));
            mmin = fmin(fabs(s), fabs(h1 - s)) / tol;
        }
#pragma unroll
        for (int side = -1; side <= 1; side += 2) {
            // the neighbour's direction about the edge, at angle phi from the 0-face tangent
            // towards the 0-face normal, must lie in the exterior (0, n pi), 1 <= n <= 2: phi in
            // (0, pi) when y > 0; otherwise phi in [pi, 2 pi) lies below n pi iff
            // sin(n pi - phi) > 0 (or phi = pi < n pi = 2 pi) -- no arctangent needed
            v3<T> r = (side < 0 ? Pm : Pp) - Pi;
            v3<T> rp = r - e * dot(r, e);
            const T y = dot(rp, cc), x = dot(rp, b);
            bool in = y > T(0);
            const T sn = h3 * x - h4 * y;   // r sin(n pi - phi): distance from the n-face plane
            if (!in && !(y == T(0) && x >= T(0))) {
                const T cs = h4 * x + h3 * y;   // r cos(n pi - phi)
                in = sn > T(0) || (sn == T(0) && cs < T(0));
            }
            if (!in) fl |= F_SIDE;
            if constexpr (F32) mmin = fmin(mmin, fmin(fabs(y), fabs(sn)) / tol);
        }
    } else {
        const T dp = dot(Pm - Pi, nn), dn = dot(Pp - Pi, nn);
        if (!(dp > T(0)) || !(dn > T(0))) fl |= F_SIDE;
        if constexpr (F32) {
            const T tol = fp32_margin_tol(fmax(fmax(amax3(Pm), amax3(Pp)), amax3(Pi)));
            mmin = fmin(fabs(dp), fabs(dn)) / tol;
        }
    }
    return VertexCheck<T>{fl, mmin};
}

template <int N = -1, class S>
DRT_HD uint32_t validity(const Prim<S> *pr, int n, const v3<typename ST<S>::R> *P) {
    typedef typename ST<S>::R T;
    constexpr bool F32 = sizeof(T) == 4;
    const int nv = N >= 0 ? N : n;
    uint32_t fl = 0;
    T mmin = T(1e30);    // FP32 only: the smallest margin over its bound
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 1; i <= MAXI + 1; ++i) {
        if (i > nv + 1) break;
        v3<T> d = P[i] - P[i - 1];
        if (!(dot(d, d) >= T(1e-18))) fl |= F_DEGEN;
    }
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 1; i <= MAXI; ++i) {
        if (i > nv) break;
        const Prim<S> &q = pr[i - 1];
        const VertexCheck<T> v =
            vertex_validity_inl(q.type, val(q.p), val(q.a), q.b, q.c, q.h1, q.h2, q.h3, q.h4, P[i - 1], P[i], P[i + 1]);
        fl |= v.fl;
        mmin = fmin(mmin, v.m);
    }
    if constexpr (F32) {
        if (mmin < T(1)) fl |= F_REDO64;
        if (mmin < T(100)) fl |= F_NEAR100;
    }
    return fl;
}

// ------------------------------------------------------------------------------------------------
// material and tile parameters in the working precision
template <class T> struct MatV { T eps_r, sigma, spec; bool pec; };   // spec = sqrt(1 - S^2)
template <class T> DRT_HD MatV<T> matv(const MatD &m);
template <> DRT_HD MatV<double> matv<double>(const MatD &m) { return {m.eps_r, m.sigma, m.spec, m.pec != 0.0}; }
template <> DRT_HD MatV<float> matv<float>(const MatD &m) { return {m.eps_rf, m.sigmaf, m.specf, m.pecf != 0.f}; }
template <class T> struct TileV { T area, s, cph, sph; int alpha; };   // cph + j sph = exp(j phase)
template <class T> DRT_HD TileV<T> tilev(const LinkDev &L, int idx);
template <> DRT_HD TileV<double> tilev<double>(const LinkDev &L, int idx) {
    const TileD &t = L.tiles[idx];
    return {t.area, t.s, t.cph, t.sph, (int)t.alpha};
}
template <> DRT_HD TileV<float> tilev<float>(const LinkDev &L, int idx) {
    const TileF &t = L.tilesF[idx];
    return {t.area, t.s, t.cph, t.sph, (int)t.alpha};
}

// ------------------------------------------------------------------------------------------------
// field coefficients
// Fresnel reflection coefficients for the perpendicular (TE) and parallel (TM) components;
// eps_c = eps_r - j sigma ieps with ieps = 1 / (2 pi f eps0); a perfect conductor gives -1 and +1.
template <class T>
DRT_HD void fresnel(const MatV<T> &m, T ieps, T ct, cx<T> &rte, cx<T> &rtm) {
    if (m.pec) {
        rte = C<T>(T(-1), T(0));
        rtm = C<T>(T(1), T(0));
        return;
    }
    cx<T> ec = C<T>(m.eps_r, -m.sigma * ieps);
    cx<T> sq = csqrt_(C<T>(ec.re - T(1) + ct * ct, ec.im));
    cx<T> ecct = ec * ct;
    // the two quotients a / b = a conj(b) / |b|^2 share one reciprocal: 1 / (|b1|^2 |b2|^2)
    const cx<T> a1 = C<T>(ct - sq.re, -sq.im), b1 = C<T>(ct + sq.re, sq.im), a2 = ecct - sq, b2 = ecct + sq;
    const T n1 = cabs2(b1), n2 = cabs2(b2), r = T(1) / (n1 * n2), i1 = n2 * r, i2 = n1 * r;
    rte = C<T>(fma(a1.re, b1.re, a1.im * b1.im) * i1, fma(a1.im, b1.re, -a1.re * b1.im) * i1);
    rtm = C<T>(fma(a2.re, b2.re, a2.im * b2.im) * i2, fma(a2.im, b2.re, -a2.re * b2.im) * i2);
}

// UTD transition function F(X) = 2j sqrt(X) exp(jX) int_sqrt(X)^inf exp(-j u^2) du for X >= 0,
// written as sqrt(pi X) exp(j pi/4) erfcx(exp(j pi/4) sqrt(X)) (erfcx(z) = exp(z^2) erfc(z)) and
// evaluated by the Maclaurin series of erf (small X), Laplace's continued fraction for erfc
// (middle range, evaluated bottom-up to a depth that falls with X) and the asymptotic series
// F ~ sum_m (2m-1)!! / (-2jX)^m (large X) -- Abramowitz & Stegun 7.1.5, 7.1.14, 7.1.23.
template <class T> struct TransitionCfg;
// The continued fraction's depth follows X: ceil(cf_a + cf_b / X) terms reach the working precision
// (2e-16 relative in FP64, 3e-8 in FP32, checked against 40-digit erfc on [x_ser, x_asy)); the
// asymptotic series, stopped once a term falls below asy_eps, reaches it from x_asy on (2.2e-16
// at X = 40 after 34 terms in FP64, 4.5e-9 at X = 20 after 14 terms in FP32).
template <> struct TransitionCfg<double> {
    static constexpr double x_ser = 6.0, x_asy = 40.0, cf_a = 6.0, cf_b = 370.0, asy_eps = 1e-17;
    static constexpr int n_cf = 68, n_asy = 40;
};
template <> struct TransitionCfg<float> {
    static constexpr float x_ser = 3.0f, x_asy = 20.0f, cf_a = 3.0f, cf_b = 84.0f, asy_eps = 1e-8f;
    static constexpr int n_cf = 31, n_asy = 16;
};

#ifdef __CUDA_ARCH__
// F(X) for 6 <= X < 40 in FP64: Taylor series about the nearest tabulated node X_i (|h| <= 1/4).
// With E_n = F^(n)(X_i) / n!, the equation F' = F (1/(2X) + j) - j gives E_1 = (j + c_0) E_0 - j
// and E_{n+1} = (j E_n + sum_{k<=n} c_k E_{n-k}) / (n + 1), c_k = (-1)^k / (2 X_i^(k+1)); eleven terms
// reach 1e-16 relative (against the continued fraction in 50-digit arithmetic), at a fraction of
// the continued fraction's cost at these X (up to 68 complex quotients).
__device__ inline cx<double> transition_F_nodes(double X) {
    int i = (int)rint((X - FNODE_X0) * (1.0 / FNODE_H));
    i = min(max(i, 0), FNODE_N - 1);
    const double xi = FNODE_X0 + FNODE_H * i, h = X - xi, ix = 1.0 / xi;
    constexpr int N = 10;
    double c[N];
    c[0] = 0.5 * ix;
#pragma unroll
    for (int k = 1; k < N; ++k) c[k] = -c[k - 1] * ix;
    double er[N + 1], ei[N + 1];
    er[0] = kFnode[2 * i];
    ei[0] = kFnode[2 * i + 1];
    er[1] = c[0] * er[0] - ei[0];
    ei[1] = er[0] + c[0] * ei[0] - 1.0;
#pragma unroll
    for (int n = 1; n < N; ++n) {
        double sr = -ei[n], si = er[n];   // j E_n
#pragma unroll
        for (int k = 0; k <= n; ++k) {
            sr = fma(c[k], er[n - k], sr);
            si = fma(c[k], ei[n - k], si);
        }
        er[n + 1] = sr * (1.0 / (n + 1));
        ei[n + 1] = si * (1.0 / (n + 1));
    }
    double ar = er[N], ai = ei[N];
#pragma unroll
    for (int n = N - 1; n >= 0; --n) {
        ar = fma(ar, h, er[n]);
        ai = fma(ai, h, ei[n]);
    }
    return C<double>(ar, ai);
}
#endif

// X below the asymptotic range (rare: a ray near a shadow or reflection boundary), out of line
template <class T> DRT_OUTLINE cx<T> transition_F_near(T X) {
    using Cfg = TransitionCfg<T>;
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 8)
        if (X >= T(Cfg::x_ser)) return transition_F_nodes(X);
#endif
    const T sqpi = T(1.7724538509055160273);
    const T r2 = T(0.70710678118654752440);
    T sx = sqrt(X);
    cx<T> z = C<T>(r2 * sx, r2 * sx);   // exp(j pi/4) sqrt(X)
    cx<T> pre = C<T>(sqpi * sx * r2, sqpi * sx * r2);   // sqrt(pi X) exp(j pi/4)
    if (X < T(Cfg::x_ser)) {
        // erf(z) = 2/sqrt(pi) z sum_n (-z^2)^n / (n! (2n+1)), z^2 = jX
        cx<T> term = C<T>(T(1), T(0)), acc = term;
        cx<T> mz2 = C<T>(T(0), -X);
        for (int k = 1; k < 64; ++k) {
            term = term * mz2 * (T(1) / T(k));
            cx<T> tk = term * (T(1) / T(2 * k + 1));
            acc = acc + tk;
            if (cabs2(tk) < T(1e-36) * cabs2(acc)) break;
        }
        cx<T> erf = z * acc * (T(2) / sqpi);
        cx<T> one_m = C<T>(T(1) - erf.re, -erf.im);
        return pre * cexpj(X) * one_m;
    }
    // erfcx(z) = 1 / (sqrt(pi) (z + (1/2)/(z + 1/(z + (3/2)/(z + ...)))))
    cx<T> f = z;
    const int depth = min(Cfg::n_cf, (int)ceil(T(Cfg::cf_a) + T(Cfg::cf_b) / X));
    for (int k = depth; k >= 1; --k) f = z + cdiv(C<T>(T(0.5) * T(k), T(0)), f);
    return cdiv(pre, f * sqpi);
}

template <class T> DRT_HD cx<T> transition_F(T X) {
    using Cfg = TransitionCfg<T>;
    if (!(X > T(0))) return C<T>(T(0), T(0));
    const T sqpi = T(1.7724538509055160273);
    const T r2 = T(0.70710678118654752440);
    if (X >= T(Cfg::x_asy)) {
        // 1 + sum_{m>=1} prod_{i<=m} (-(2i-1)) / (2jX) ; 1/(2jX) = -j/(2X)
        // each factor -(2m - 1) / (2jX) is purely imaginary: one real multiply per part; stop once
        // the terms fall below the working precision
        cx<T> acc = C<T>(T(1), T(0)), term = C<T>(T(1), T(0));
        const T a = T(-0.5) / X;   // 1/(2jX) = j a
        for (int mm = 1; mm <= Cfg::n_asy; ++mm) {
            const T sm = a * T(-(2 * mm - 1));   // term *= j sm
            term = C<T>(-term.im * sm, term.re * sm);
            acc = acc + term;
            if (fabs(term.re) + fabs(term.im) < T(Cfg::asy_eps)) break;
        }
        return acc;
    }
    return transition_F_near(X);
}

// one Kouyoumjian-Pathak term cot((pi +- beta)/2n) F(kL a+-(beta)) with eps = (pi +- beta) - 2 pi n N:
// cot(eps/2n) F(2 kL sin^2(eps/2)), -> n sqrt(2 pi kL) sgn(eps) exp(j pi/4) as eps -> 0
template <class T> DRT_HD cx<T> utd_term(T eps, T n, T inv2n, T kL) {
    if (fabs(eps) < T(1e-9)) {
        T m = n * sqrt(T(2 * PI) * kL) * (eps >= T(0) ? T(1) : T(-1)) * T(0.70710678118654752440);
        return C<T>(m, m);
    }
    T sh, s2, c2;
    if (n == T(1.5)) {   // right-angled wedge: eps/2 = 3u and eps/2n = 2u with u = eps/6, one sincos
        T su, cu;
        sincos(eps * T(1.0 / 6.0), &su, &cu);
        sh = su * (T(3) - T(4) * su * su);
        s2 = T(2) * su * cu;
        c2 = T(1) - T(2) * su * su;
    } else {
        sh = sin(T(0.5) * eps);
        sincos(eps * inv2n, &s2, &c2);   // cot(eps / 2n)
    }
    return transition_F(T(2) * kL * sh * sh) * (c2 / s2);
}

// the same term for a right-angled wedge (n = 3/2) from su, cu = sin, cos of eps / 6 (eps/2 = 3 eps/6,
// eps/2n = 2 eps/6)
template <class T> DRT_HD cx<T> utd_term_ra(T eps, T su, T cu, T kL) {
    if (fabs(eps) < T(1e-9)) {
        T m = T(1.5) * sqrt(T(2 * PI) * kL) * (eps >= T(0) ? T(1) : T(-1)) * T(0.70710678118654752440);
        return C<T>(m, m);
    }
    const T sh = su * (T(3) - T(4) * su * su), s2 = T(2) * su * cu, c2 = T(1) - T(2) * su * su;
    return transition_F(T(2) * kL * sh * sh) * (c2 / s2);
}
// sin, cos of x / 6 + pi / 6 - m pi / 2 from sin, cos of x / 6 (sx, cx): a turn by pi / 6, then m
// quarter turns (exact)
template <class T> DRT_HD void ra_shift(T sx, T cx, int m, T &s, T &c) {
    const T c6 = T(0.86602540378443864676), s6 = T(0.5);
    T a = sx * c6 + cx * s6, b = cx * c6 - sx * s6;   // sin, cos of x/6 + pi/6
    switch (m & 3) {   // minus m quarter turns
    case 0: s = a; c = b; break;
    case 1: s = -b; c = a; break;
    case 2: s = -a; c = -b; break;
    default: s = b; c = -a; break;
    }
}

// soft / hard wedge diffraction coefficients: Kouyoumjian-Pathak with the spherical-wave distance
// parameter L, Luebbers' face-coefficient weights for lossy wedges
// (sphip = |sin phi'|, snphi = |sin(n pi - phi)|: the incidence sines of the 0-face and n-face
// reflection coefficients, passed in from the direction components)
template <class T>
DRT_HD void utd(T n, T phi, T phip, T sphip, T snphi, T sinb0, T L, T k, T isk, const MatV<T> &m, T ieps,
                cx<T> &Ds, cx<T> &Dh) {
    // isk = 1 / sqrt(2 pi k), once per call; 1/(2n) without a division for right-angled wedges
    T kL = k * L;
    const T inv2n = n == T(1.5) ? T(1.0 / 3.0) : T(1) / (T(2) * n), itpn = inv2n * T(1 / PI);   // 1/(2n), 1/(2 pi n)
    T pref = inv2n * isk / sinb0;
    cx<T> Cc = C<T>(-pref * T(0.70710678118654752440), pref * T(0.70710678118654752440));  // -exp(-j pi/4) pref
    T bm = phi - phip, bp = phi + phip, tpn = T(2 * PI) * n;
    const T N1 = round((bm + T(PI)) * itpn), N2 = round((bm - T(PI)) * itpn);
    const T N3 = round((bp - T(PI)) * itpn), N4 = round((bp + T(PI)) * itpn);
    const T e1 = T(PI) + bm - tpn * N1, e2 = T(PI) - bm + tpn * N2;
    const T e3 = T(PI) - bp + tpn * N3, e4 = T(PI) + bp - tpn * N4;
    cx<T> t1, t2, t3, t4;
    if (n == T(1.5)) {
        // right-angled wedge: the four sin, cos of eps_i / 6 from those of phi / 6 and phi' / 6 (two
        // sincos instead of four): eps_i / 6 = pi/6 +- (phi -+ phi') / 6 -+ N_i pi / 2
        T sa, ca, sb, cb;
        sincos(phi * T(1.0 / 6.0), &sa, &ca);
        sincos(phip * T(1.0 / 6.0), &sb, &cb);
        const T sm = sa * cb - ca * sb, cm = ca * cb + sa * sb;   // (phi - phi') / 6
        const T sp = sa * cb + ca * sb, cp = ca * cb - sa * sb;   // (phi + phi') / 6
        T s, c;
        ra_shift(sm, cm, (int)N1, s, c);
        t1 = utd_term_ra(e1, s, c, kL);
        ra_shift(-sm, cm, -(int)N2, s, c);
        t2 = utd_term_ra(e2, s, c, kL);
        ra_shift(-sp, cp, -(int)N3, s, c);
        t3 = utd_term_ra(e3, s, c, kL);   // 0-face
        ra_shift(sp, cp, (int)N4, s, c);
        t4 = utd_term_ra(e4, s, c, kL);   // n-face
    } else {
        t1 = utd_term(e1, n, inv2n, kL);
        t2 = utd_term(e2, n, inv2n, kL);
        t3 = utd_term(e3, n, inv2n, kL);   // 0-face
        t4 = utd_term(e4, n, inv2n, kL);   // n-face
    }
    cx<T> r0s, r0h, rns, rnh;
    fresnel(m, ieps, sphip, r0s, r0h);
    fresnel(m, ieps, snphi, rns, rnh);
    cx<T> base = t1 + t2;
    Ds = Cc * (base + r0s * t3 + rns * t4);
    Dh = Cc * (base + r0h * t3 + rnh * t4);
}

// Effective-Roughness directive lobe normalisation for integer alpha:
// F = 2^-alpha sum_j C(alpha, j) I_j with I_j = 2 pi / (j+1) for even j and
// I_j = 2 pi / (j+1) cos(ti) sum_{w=0}^{(j-1)/2} C(2w, w) sin^{2w}(ti) / 4^w for odd j.
template <class T> DRT_HD T er_norm(int alpha, T cti) {
    T s2 = fmax(T(0), T(1) - cti * cti);
    // the sum written out for the exponents of the workloads
    if (alpha == 2) return T(2 * PI / 3) + T(PI / 2) * cti;
    if (alpha == 4) return T(2 * PI / 5) + T(PI / 16) * cti * (T(6) + s2);
    T acc = T(0), binom = T(1);   // C(alpha, j)
    T oddsum = T(0), cw = T(1), s2w = T(1);   // running sum_{w} C(2w,w) s2^w / 4^w
    int wmax = -1;
    for (int j = 0; j <= alpha; ++j) {
        T Ij;
        if ((j & 1) == 0) {
            Ij = T(2 * PI) / T(j + 1);
        } else {
            while (wmax < (j - 1) / 2) {
                ++wmax;
                if (wmax > 0) {
                    cw = cw * T(2 * (2 * wmax - 1)) / T(wmax);   // C(2w,w) from C(2w-2,w-1)
                    s2w = s2w * s2 * T(0.25);
                }
                oddsum += cw * s2w;
            }
            Ij = T(2 * PI) / T(j + 1) * cti * oddsum;
        }
        acc += binom * Ij;
        binom = binom * T(alpha - j) / T(j + 1);
    }
    return ldexp(acc, -alpha);
}

template <class T> DRT_HD v3<T> vertical_pol(v3<T> k) {
    v3<T> p = V3<T>(-k.z * k.x, -k.z * k.y, T(1) - k.z * k.z);
    if (dot(p, p) < T(1e-18)) p = V3<T>(T(1) - k.x * k.x, -k.x * k.y, -k.x * k.z);
    return unit(p);
}

// complex amplitude a_p excluding exp(-j k d): (lambda / 4 pi) x ray spreading x polarimetric chain of
// Fresnel / UTD / ER factors; TX and RX vertically polarised.  seg[1..n+1] are the segment vectors.
// Spreading and UTD distance parameters per stretch between point sources (TX, tiles, RX), after
// Kouyoumjian-Pathak: spherical from a point source; an edge-diffracted ray spreads as
// sqrt(rho_e / (s (rho_e + s))) to the next diffraction or point source at s, rho_e being the
// incident wavefront's radius of curvature in the plane of the incident ray and the edge (the distance
// from the source for a spherical wave; after a diffraction the principal radii are the distance from
// the edge along e x k_out and rho_e + distance, carried through planar reflections with mirrored
// directions, so Euler's formula gives rho_e at a second diffraction); the distance parameter is
// L = s (rho_e + s) rho1 rho2 sin^2 b0 / (rho_e (rho1 + s)(rho2 + s)), s s' sin^2 b0 / (s + s') for a
// spherical incident wave.  Loops run over the fixed bound MAXI (see validity).
// The field update at one vertex, per interaction type: E (the incident field, polarisation and
// amplitude so far) across a reflection (Fresnel, Sec. III-A), a diffraction (UTD, Sec. III-B) or a
// tile (ER, Sec. III-C), with kin / kout the unit directions of the incoming and outgoing segments.
// The FP32 kernels call them out of line (one copy each, instead of one per vertex of every unrolled
// chain length: the unrolled code otherwise outgrows the instruction cache, and the warps of an SM,
// which run different chain signatures, wait on instruction fetch); FP64 keeps them inline.
template <class T>
DRT_HD c3<T> refl_field_inl(c3<T> E, v3<T> kin, v3<T> kout, v3<T> nf, MatV<T> m, T ieps) {
    if (dot(nf, kin) > T(0)) nf = -nf;
    T ct = -dot(nf, kin);
    v3<T> ep = cross(kin, nf);
    if (dot(ep, ep) < T(1e-24)) {
        ep = cross(nf, V3<T>(T(1), T(0), T(0)));
        if (dot(ep, ep) < T(1e-12)) ep = cross(nf, V3<T>(T(0), T(1), T(0)));
    }
    ep = unit(ep);
    v3<T> epin = cross(ep, kin), epout = cross(ep, kout);
    cx<T> rte, rtm;
    fresnel(m, ieps, ct, rte, rtm);
    return cscale(ep, rte * cdot(E, ep) * m.spec) + cscale(epout, rtm * cdot(E, epin) * m.spec);
}

// e: edge direction; t0, n0: the 0-face tangent and normal; wn: wedge n; snp, cnp: sin(n pi), cos(n pi);
// Lf: the distance parameter over sin^2 b0
template <class T>
DRT_HD c3<T> diff_field_inl(c3<T> E, v3<T> kin, v3<T> kout, v3<T> e, v3<T> t0, v3<T> n0, T wn, T snp, T cnp, T Lf,
                            T k, T isk, MatV<T> m, T ieps) {
    v3<T> wi = -kin + e * dot(kin, e);
    v3<T> wo = kout - e * dot(kout, e);
    const T yi = dot(wi, n0), xi = dot(wi, t0), yo = dot(wo, n0), xo = dot(wo, t0);
    // atan2 lies in [-pi, pi]: one conditional turn maps it to [0, 2 pi) (no fmod)
    T phip = atan2(yi, xi), phi = atan2(yo, xo);
    if (phip < T(0)) phip += T(2 * PI);
    if (phi < T(0)) phi += T(2 * PI);
    T sinb0 = norm(cross(kin, e));
    const T Lp = Lf * sinb0 * sinb0;
    T sphip = T(0), snphi = T(0);
    if (!m.pec) {   // Luebbers' face coefficients: sin phi' and sin(n pi - phi) from components
        const T ri2 = xi * xi + yi * yi, ro2 = xo * xo + yo * yo;
        sphip = ri2 > T(0) ? fabs(yi) * rsqrt(ri2) : T(0);
        snphi = ro2 > T(0) ? fabs(snp * xo - cnp * yo) * rsqrt(ro2) : T(0);
    }
    cx<T> Ds, Dh;
    utd(wn, phi, phip, sphip, snphi, sinb0, Lp, k, isk, m, ieps, Ds, Dh);
    v3<T> php = -unit(cross(e, kin)), bpv = cross(php, kin);
    v3<T> ph = unit(cross(e, kout)), bv = cross(ph, kout);
    return cscale(bv, -(Ds * cdot(E, bpv))) + cscale(ph, -(Dh * cdot(E, php)));
}

template <class T>
DRT_HD c3<T> tile_field_inl(c3<T> E, v3<T> kin, v3<T> kout, v3<T> nt, TileV<T> tl) {
    if (dot(nt, kin) > T(0)) nt = -nt;
    T cti = -dot(nt, kin);
    v3<T> kspec = kin + nt * (T(2) * cti);
    T cpsi = dot(kspec, kout);
    int alpha = tl.alpha;
    T Fa = er_norm<T>(alpha, cti);
    const T hb = T(0.5) * (T(1) + cpsi);
    T lobe_h = T(1);   // ((1 + cos psi)/2)^(alpha/2): the field of the power lobe
    for (int j = 0; j < alpha / 2; ++j) lobe_h *= hb;
    if (alpha & 1) lobe_h *= sqrt(hb);
    const T qa = tl.area * cti;   // sqrt(qa / Fa) by one reciprocal square root
    T amp = tl.s * (qa > T(0) ? qa * rsqrt(qa * Fa) : sqrt(qa / Fa)) * lobe_h;
    cx<T> ph = C<T>(tl.cph, tl.sph);
    const T e2 = cabs2(E.x) + cabs2(E.y) + cabs2(E.z), nE = sqrt(e2);
    cx<T> ek = cdot(E, kout);
    c3<T> Ep = E + cscale(kout, -ek);
    const T ep2 = cabs2(Ep.x) + cabs2(Ep.y) + cabs2(Ep.z);
    if (ep2 < T(1e-24) * e2 || e2 == T(0)) Ep = cscale(vertical_pol(kout), C<T>(nE, T(0)));
    else Ep = cscale(Ep, C<T>(nE * rsqrt(ep2), T(0)));
    return cscale(Ep, ph * amp);
}

#define DRT_NOINL __host__ __device__ __noinline__
template <class T> DRT_NOINL c3<T> refl_field_out(c3<T> E, v3<T> kin, v3<T> kout, v3<T> nf, MatV<T> m, T ieps) {
    return refl_field_inl(E, kin, kout, nf, m, ieps);
}
template <class T>
DRT_NOINL c3<T> diff_field_out(c3<T> E, v3<T> kin, v3<T> kout, v3<T> e, v3<T> t0, v3<T> n0, T wn, T snp, T cnp, T Lf,
                               T k, T isk, MatV<T> m, T ieps) {
    return diff_field_inl(E, kin, kout, e, t0, n0, wn, snp, cnp, Lf, k, isk, m, ieps);
}
template <class T> DRT_NOINL c3<T> tile_field_out(c3<T> E, v3<T> kin, v3<T> kout, v3<T> nt, TileV<T> tl) {
    return tile_field_inl(E, kin, kout, nt, tl);
}

template <int N = -1, class S, class T = typename ST<S>::R>
DRT_HD cx<T> amplitude(const LinkDev &L, const Prim<S> *pr, int n, const v3<T> *seg, T fc) {
    const int nv = N >= 0 ? N : n;
    v3<T> kd[MAXI + 2];
    T len[MAXI + 2];
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 1; i <= MAXI + 1; ++i) {
        if (i > nv + 1) break;
        const T q = dot(seg[i], seg[i]), rs = rsqrt(q);   // one reciprocal square root per segment
        len[i] = q * rs;
        kd[i] = seg[i] * rs;
    }
    // distance from each diffraction to the next diffraction or point source
    T snx[MAXI + 1];
    {
        T acc = T(0);
#pragma unroll (N >= 0 ? 8 : 1)
        for (int i = MAXI; i >= 1; --i) {
            if (i > nv) continue;
            acc += len[i + 1];
            const int ty = pr[i - 1].type;
            if (ty == T_D) {
                snx[i] = acc;
                acc = T(0);
            } else if (ty == T_S) {
                acc = T(0);
            }
        }
    }
    // spreading and, per diffraction, L / sin^2 b0
    // spread^2 = sp_num / sp_den, one square root per call
    T sp_num = T(1), sp_den = T(1), Lfac[MAXI + 1];
    {
        T d = T(0), re = T(0);          // distance since the point source or latest diffraction; its rho_e
        bool after_d = false;
        v3<T> X1 = V3<T>(T(0), T(0), T(0));   // after a diffraction: direction of its caustic on the edge
#pragma unroll (N >= 0 ? 8 : 1)
        for (int i = 1; i <= MAXI + 1; ++i) {
            if (i > nv + 1) break;
            d += len[i];
            const int ty = i <= nv ? pr[i - 1].type : T_S;   // the RX ends the last stretch like a source
            if (ty == T_R) {
                if (after_d) X1 = mirror_dir(X1, val(pr[i - 1].a));
                continue;
            }
            if (!after_d) sp_den *= d * d;
            else {
                sp_num *= re;
                sp_den *= d * (re + d);
            }
            if (ty == T_S) {
                after_d = false;
                d = T(0);
                continue;
            }
            const v3<T> e = val(pr[i - 1].a);
            const T s = snx[i];
            if (!after_d) {   // spherical incident wave: rho1 = rho2 = rho_e = d
                Lfac[i] = s * d / (s + d);
                re = d;
            } else {
                const v3<T> u = e - kd[i] * dot(e, kd[i]);
                const T uu = dot(u, u), ux = dot(u, X1);
                const T cg2 = uu > T(1e-24) ? ux * ux / uu : T(0);
                const T r1 = d, r2 = re + d;
                const T rhe = T(1) / (cg2 / r1 + (T(1) - cg2) / r2);
                Lfac[i] = s * (rhe + s) * r1 * r2 / (rhe * (r1 + s) * (r2 + s));
                re = rhe;
            }
            // the caustic direction is only needed by a later diffraction of the same stretch
            bool more_d = false;
#pragma unroll (N >= 0 ? 8 : 1)
            for (int j = i + 1; j <= MAXI; ++j) {
                if (j > nv || pr[j - 1].type == T_S) break;
                more_d = more_d || pr[j - 1].type == T_D;
            }
            if (more_d) X1 = unit(cross(e, kd[i + 1]));
            after_d = true;
            d = T(0);
        }
    }
    // one division per call: the wavenumber, eps_c = eps_r - j sigma ieps and lambda / (4 pi) from 1/fc
    const T ifc = T(1) / fc;
    const T k = fc * T(2 * PI / C0), isk = rsqrt(T(2 * PI) * k);
    const T ieps = ifc * T(1 / (2 * PI * EPS0));
    c3<T> E = cscale(vertical_pol(kd[1]), C<T>(T(1), T(0)));
    v3<T> klast = kd[1];
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 1; i <= MAXI; ++i) {
        if (i > nv) break;
        const Prim<S> &q = pr[i - 1];
        const v3<T> kin = kd[i], kout = kd[i + 1];
        klast = kout;
        constexpr bool OUTL = sizeof(T) == 4;
        if (q.type == T_R) {
            const MatV<T> m = matv<T>(L.mats[q.mat]);
            if constexpr (OUTL) E = refl_field_out(E, kin, kout, val(q.a), m, ieps);
            else E = refl_field_inl(E, kin, kout, val(q.a), m, ieps);
        } else if (q.type == T_D) {
            const MatV<T> m = matv<T>(L.mats[q.mat]);
            if constexpr (OUTL)
                E = diff_field_out(E, kin, kout, val(q.a), q.b, q.c, q.h2, q.h3, q.h4, Lfac[i], k, isk, m, ieps);
            else E = diff_field_inl(E, kin, kout, val(q.a), q.b, q.c, q.h2, q.h3, q.h4, Lfac[i], k, isk, m, ieps);
        } else {
            const TileV<T> tl = tilev<T>(L, q.idx);
            if constexpr (OUTL) E = tile_field_out(E, kin, kout, val(q.a), tl);
            else E = tile_field_inl(E, kin, kout, val(q.a), tl);
        }
    }
    const T spread = sqrt(sp_num / sp_den);
    return cdot(E, vertical_pol(klast)) * (ifc * T(C0 / (4 * PI)) * spread);
}

// App. A Eq. doppler_freq: f' = f0 prod_i (c - v_i.k_i) / (c - v_{i-1}.k_i), evaluated without
// cancellation as f_D = f0 expm1( sum_i log1p(-v_i.k_i / c) - log1p(-v_{i-1}.k_i / c) )
template <int N = -1, class S, class T = typename ST<S>::R>
DRT_HD T doppler(int n, const v3<S> *V, const v3<T> *seg, T fc) {
    const int nv = N >= 0 ? N : n;
    T acc = T(0);
    const T ic = T(1) / T(C0);
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 1; i <= MAXI + 1; ++i) {
        if (i > nv + 1) break;
        v3<T> k = unit(seg[i]);
        acc += log1p(-dot(der(V[i]), k) * ic) - log1p(-dot(der(V[i - 1]), k) * ic);
    }
    return fc * expm1(acc);
}

// ------------------------------------------------------------------------------------------------
// one (path, time-step) of the FP64 form: geometry, validity, delay, Doppler, angles, amplitude;
// user outputs at [ti][perm[p]], synthesis record at [ti][p]
DRT_HD void write_outputs_fp64(const OutD &o, size_t oi, int n, const v3<double> *P, v3<double> seg_first,
                               v3<double> seg_last, double tau, cx<double> a, double fd, uint32_t fl) {
    if (o.tau) o.tau[oi] = tau;
    if (o.amp) {
        double *q = reinterpret_cast<double *>(o.amp) + 2 * oi;
        q[0] = a.re;
        q[1] = a.im;
    }
    if (o.doppler) reinterpret_cast<double *>(o.doppler)[oi] = fd;
    if (o.angles) {
        v3<double> kd = unit(seg_first), ka = -unit(seg_last);
        float *q = o.angles + 4 * oi;
        q[0] = (float)atan2(kd.y, kd.x);
        q[1] = (float)atan2(kd.z, hypot(kd.x, kd.y));
        q[2] = (float)atan2(ka.y, ka.x);
        q[3] = (float)atan2(ka.z, hypot(ka.x, ka.y));
    }
    if (o.flags) o.flags[oi] = (uint8_t)fl;
    if (o.points) {
        double *q = o.points + oi * (MAXI * 3);
        const double qn = nan("");
#pragma unroll
        for (int j = 0; j < MAXI; ++j) {
            bool in = j < n;
            q[3 * j + 0] = in ? P[j + 1].x : qn;
            q[3 * j + 1] = in ? P[j + 1].y : qn;
            q[3 * j + 2] = in ? P[j + 1].z : qn;
        }
    }
}

// record for the synthesis: amplitude (0 if the path does not exist), phase seed frac(f_0 tau) and
// per-bin step frac(df tau) split as hi (12 leading bits, so k * hi is exact in FP32) + lo
DRT_HD void write_record(const RecD &r, size_t ri, double tau, cx<double> a, uint32_t fl, double f0, double df) {
    double x = f0 * tau;
    double phi0 = x - floor(x);
    double y = df * tau;
    double st = y - floor(y);
    double hi = ldexp(rint(ldexp(st, 12)), -12);
    float4 v;
    v.x = fl ? 0.f : (float)a.re;
    v.y = fl ? 0.f : (float)a.im;
    v.z = (float)phi0;
    v.w = (float)hi;
    r.rec_a[ri] = v;
    r.rec_b[ri] = (float)(st - hi);
}

// FP64 (path, time-step) core: primitives from `load(j, type, idx)`; FP64 outputs (amp double[2],
// Doppler double) or, for the FP32-bulk form's redo, FP32 ones (float[2], float)
// Warm starts of the chains with >= 2 diffractions in a segment (paths [n_bulk, n_paths)).  The
// table holds, per chunk base c = 0..n_chunks (one past the last chunk) and multi-diffraction path,
// each diffraction vertex's edge parameter s and rate ds/dt from an FP64 dual-number solve
// ([row][path - n_bulk][2 * MAXI]).  A step at tau into chunk c starts its Newton solve from the
// cubic Hermite interpolant of (s, ds/dt) at the bases c and c + 1, which is within ~1e-10 m of the
// root on these workloads, so one Newton step converges.
DRT_HD const double *warm_row(const LinkDev &L, const double *warm, int row, int p) {
    return warm + ((size_t)row * (L.n_paths - L.n_bulk) + (p - L.n_bulk)) * (2 * MAXI);
}
struct WarmStart { double s[MAXI], ds[MAXI], rate[MAXI]; };
DRT_HD void hermite_start(const double *w0, const double *w1, double tau, double Tc, WarmStart &ws) {
    const double h = tau / Tc, h2 = h * h, h3 = h2 * h;
    const double h10 = h3 - 2.0 * h2 + h, h01 = 3.0 * h2 - 2.0 * h3, h11 = h3 - h2;
    const double g00 = 6.0 * h2 - 6.0 * h, g10 = 3.0 * h2 - 4.0 * h + 1.0, g11 = 3.0 * h2 - 2.0 * h;
    for (int j = 0; j < MAXI; ++j) {
        const double s0 = w0[j], r0 = w0[MAXI + j], s1 = w1[j], r1 = w1[MAXI + j];
        ws.s[j] = s0;
        // s(tau) - s0 = h10 Tc r0 + h01 (s1 - s0) + h11 Tc r1 (h00 + h01 = 1)
        ws.ds[j] = h10 * Tc * r0 + h01 * (s1 - s0) + h11 * Tc * r1;
        ws.rate[j] = (-g00 * (s1 - s0)) / Tc + g10 * r0 + g11 * r1;
    }
}
DRT_HD void warm_start_at(const LinkDev &L, const TimeGridD &tg, const double *warm, int p, int ti, WarmStart &ws) {
    const int c = ti / tg.chunk;
    hermite_start(warm_row(L, warm, c, p), warm_row(L, warm, c + 1, p), (ti - c * tg.chunk) * tg.dt,
                  tg.chunk * tg.dt, ws);
}
// The same interpolant for the FP32-bulk steps: the base s stays FP64 (the Newton start's base part),
// the offset and rate are FP32 (the difference s1 - s0 taken in FP64 first), which keeps the FP64 pipe
// -- 1/64 of the FP32 rate on GB300 -- out of the FP32 kernels' per-step work but for one
// subtraction and the conversions per unknown
struct WarmStart32 { double s[MAXI]; float ds[MAXI], rate[MAXI]; };
DRT_HD void warm_start_at32(const LinkDev &L, const TimeGridD &tg, const double *warm, int p, int ti,
                            WarmStart32 &ws) {
    const int c = ti / tg.chunk;
    const double *w0 = warm_row(L, warm, c, p), *w1 = warm_row(L, warm, c + 1, p);
    const float Tc = (float)tg.chunk * tg.dtf, iTc = 1.f / Tc;
    const float h = (float)(ti - c * tg.chunk) / (float)tg.chunk, h2 = h * h, h3 = h2 * h;
    const float h10 = h3 - 2.f * h2 + h, h01 = 3.f * h2 - 2.f * h3, h11 = h3 - h2;
    const float g00 = 6.f * h2 - 6.f * h, g10 = 3.f * h2 - 4.f * h + 1.f, g11 = 3.f * h2 - 2.f * h;
#pragma unroll
    for (int j = 0; j < MAXI; ++j) {
        const float d = (float)(w1[j] - w0[j]), r0 = (float)w0[MAXI + j], r1 = (float)w1[MAXI + j];
        ws.s[j] = w0[j];
        ws.ds[j] = h10 * Tc * r0 + h01 * d + h11 * Tc * r1;
        ws.rate[j] = -g00 * d * iTc + g10 * r0 + g11 * r1;
    }
}

// terminal position (and velocity on dual numbers) at time t
template <class S> DRT_HD v3<S> terminal_as(const TermD &m, double t);
template <> DRT_HD v3<dl<double>> terminal_as<dl<double>>(const TermD &m, double t) { return terminal<double>(m, t); }
template <> DRT_HD v3<double> terminal_as<double>(const TermD &m, double t) { return val(terminal<double>(m, t)); }

// S = dl<double> carries every position with its time derivative (the interaction points' sliding
// velocities, which only the Doppler shift needs); S = double runs the same geometry on values
// alone, for calls that ask for no Doppler output (H synthesis), at about half the FP64 work.
// N >= 0: chains of exactly N vertices with at most one diffraction between point sources (the
// unrolled solver; every per-vertex array in registers); N < 0: any chain, length read at run time.
// MULTI: the chain may have several diffractions in a segment (Newton, warm starts).  OUT = false
// drops the user-output code (calls that only fill synthesis records).
template <int N = -1, bool MULTI = true, bool OUT = true, class S = dl<double>, class Loader>
DRT_HD void path_step_fp64_core(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, int p, int ti,
                                const OutD &out, const RecD &rec, bool f32out, Loader load,
                                const double *warm = nullptr, double *rec64 = nullptr) {
    if constexpr (N < 0) {
        with_length<len_min<N>()>(chain_length(L, p), [&](auto NC) {
            path_step_fp64_core<decltype(NC)::value, MULTI, OUT, S>(L, tg, fg, p, ti, out, rec, f32out, load, warm,
                                                                    rec64);
        });
        return;
    } else {
    typedef double T;
    const T t = tg.t_start + ti * tg.dt;
    const uint32_t code = L.ptypes[p];
    const int4 pi = L.pprims[p];
    const int prim[MAXI] = {pi.x, pi.y, pi.z, pi.w};
    constexpr int n = N;
    Prim<S> pr[MAXI];
#pragma unroll
    for (int j = 0; j < N; ++j) pr[j] = load((code >> (8 * j)) & 0xff, prim[j]);
    v3<S> V[MAXI + 2];
    V[0] = terminal_as<S>(L.tx, t);
    V[N + 1] = terminal_as<S>(L.rx, t);
    uint32_t fl = 0;
    if (MULTI && warm && p >= L.n_bulk) {
        WarmStart ws;
        warm_start_at(L, tg, warm, p, ti, ws);
        solve_geometry<N, MULTI>(pr, V, ws.s, fl, ws.ds, ws.rate);
    } else {
        solve_geometry<N, MULTI>(pr, V, L.ps0 + (size_t)p * MAXI, fl);
    }
    v3<T> P[MAXI + 2];
    v3<T> seg[MAXI + 2];
    T d = T(0);
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 0; i <= MAXI + 1; ++i) {
        if (i > n + 1) break;
        P[i] = val(V[i]);
        if (i > 0) {
            seg[i] = P[i] - P[i - 1];
            d += norm(seg[i]);
        }
    }
    fl |= validity<N>(pr, n, P);
    T tau = d * T(1 / C0);
    // An invalid path-step contributes nothing to H (its records carry a = 0): its field coefficients
    // are computed only when the caller asked for the amplitude output, which reports them for every
    // step (a degenerate chain has none)
    const bool field = !fl || (OUT && out.amp && !(fl & F_DEGEN));
    cx<T> a = field ? amplitude<N>(L, pr, n, seg, T(fg.fc)) : C<T>(T(0), T(0));
    if constexpr (OUT) {
        if (out.tau || out.amp || out.doppler || out.angles || out.flags || out.points) {
            T fd = 0;
            if constexpr (!std::is_same<S, double>::value) fd = doppler<N>(n, V, seg, T(fg.fc));
            const size_t oi = (size_t)ti * L.n_paths + L.perm[p];
            v3<T> s_last = seg[1];
#pragma unroll (N >= 0 ? 8 : 1)
            for (int i = 2; i <= MAXI + 1; ++i)
                if (i == n + 1) s_last = seg[i];
            if (f32out) {
                OutD o2 = out;
                o2.amp = nullptr;
                o2.doppler = nullptr;
                write_outputs_fp64(o2, oi, n, P, seg[1], s_last, tau, a, fd, fl);
                if (out.amp) {
                    float *q = reinterpret_cast<float *>(out.amp) + 2 * oi;
                    q[0] = (float)a.re;
                    q[1] = (float)a.im;
                }
                if (out.doppler) reinterpret_cast<float *>(out.doppler)[oi] = (float)fd;
            } else {
                write_outputs_fp64(out, oi, n, P, seg[1], s_last, tau, a, fd, fl);
            }
        }
    }
    if (rec.rec_a) {
        const double f0 = fg.f0, df = fg.df;
        write_record(rec, (size_t)ti * L.n_paths + p, tau, a, fl, f0, df);
    }
    if (rec64) {   // (Re a, Im a, tau), a = 0 when the path does not exist
        rec64[0] = fl ? 0.0 : a.re;
        rec64[1] = fl ? 0.0 : a.im;
        rec64[2] = tau;
    }
    }
}

// an FP64 dual-number primitive without its rates
DRT_HD Prim<double> val_prim(const Prim<dl<double>> &q) {
    Prim<double> r;
    r.type = q.type;
    r.mat = q.mat;
    r.idx = q.idx;
    r.p = val(q.p);
    r.a = val(q.a);
    r.b = q.b;
    r.c = q.c;
    r.h1 = q.h1;
    r.h2 = q.h2;
    r.h3 = q.h3;
    r.h4 = q.h4;
    return r;
}

// FP32 copies (the FP32 stage of a warm-start solve)
DRT_HD v3<float> f32v(v3<double> a) { return V3<float>(a.x, a.y, a.z); }
DRT_HD Prim<float> f32_prim(const Prim<dl<double>> &q) {
    Prim<float> r;
    r.type = q.type;
    r.mat = q.mat;
    r.idx = q.idx;
    r.p = f32v(val(q.p));
    r.a = f32v(val(q.a));
    r.b = f32v(q.b);
    r.c = f32v(q.c);
    r.h1 = (float)q.h1;
    r.h2 = (float)q.h2;
    r.h3 = (float)q.h3;
    r.h4 = (float)q.h4;
    return r;
}

// One dual-number FP64 solve of a chain at time t from the edge-parameter start `sin`; writes each
// diffraction vertex's parameter and rate to sv/sd (sin and 0 where the solve failed).  N < 0: the
// chain length is read at run time and the solve runs in the instance for that length.
template <int N = -1, class Loader>
DRT_HD void solve_edge_params(const LinkDev &L, int p, double t, const double *sin, double *sv, double *sd,
                              Loader load) {
    if constexpr (N < 0) {
        with_length<len_min<N>()>(chain_length(L, p), [&](auto NC) {
            solve_edge_params<decltype(NC)::value>(L, p, t, sin, sv, sd, load);
        });
    } else {
        typedef double T;
        const uint32_t code = L.ptypes[p];
        const int4 pi = L.pprims[p];
        const int prim[MAXI] = {pi.x, pi.y, pi.z, pi.w};
        Prim<dl<T>> pr[N > 0 ? N : 1];
#pragma unroll
        for (int j = 0; j < N; ++j) pr[j] = load((code >> (8 * j)) & 0xff, prim[j]);
        v3<dl<T>> V[N + 2];
        V[0] = terminal<T>(L.tx, t);
        V[N + 1] = terminal<T>(L.rx, t);
        // Staged Newton: FP32 from the start `sin` to ~1e-4 m (FP32 runs at 64x the FP64 rate), then FP64
        // values to the FP64 tolerance (quadratic convergence: two or three steps), then one dual-number
        // step, which gives the rates (the implicit-function derivative) at the root.  A stage that does
        // not converge leaves the next one its own start.
        double s1[MAXI];
#pragma unroll
        for (int j = 0; j < MAXI; ++j) s1[j] = sin[j];
        if constexpr (N >= 2) {
            Prim<float> pf[N];
            v3<float> Vf[N + 2];
#pragma unroll
            for (int j = 0; j < N; ++j) pf[j] = f32_prim(pr[j]);
            Vf[0] = f32v(val(V[0]));
            Vf[N + 1] = f32v(val(V[N + 1]));
            uint32_t ff = 0;
            solve_geometry_any<N>(pf, Vf, s1, ff);
            if (!(ff & F_NOCONV))
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (pf[j].type == T_D) s1[j] = (double)dot(Vf[j + 1] - pf[j].p, pf[j].a);
            Prim<double> pd[N];
            v3<double> Vd[N + 2];
#pragma unroll
            for (int j = 0; j < N; ++j) pd[j] = val_prim(pr[j]);
            Vd[0] = val(V[0]);
            Vd[N + 1] = val(V[N + 1]);
            uint32_t fd = 0;
            solve_geometry_any<N>(pd, Vd, s1, fd);
            if (!(fd & F_NOCONV))
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (pd[j].type == T_D) s1[j] = dot(Vd[j + 1] - pd[j].p, pd[j].a);
        }
        uint32_t fl = 0;
        solve_geometry_any<N>(pr, V, s1, fl);
#pragma unroll
        for (int j = 0; j < MAXI; ++j) {
            sv[j] = sin[j];
            sd[j] = 0.0;
            if (j < N && pr[j].type == T_D && !(fl & F_NOCONV)) {
                dl<T> sj = dot(V[j + 1] - pr[j].p, pr[j].a);
                if (isfinite(sj.v) && isfinite(sj.d)) {
                    sv[j] = sj.v;
                    sd[j] = sj.d;
                }
            }
        }
    }
}

// one row of the warm-start table: the chunk base `row` solved from the t0 edge parameters
// edge parameters and their rates at t = 0, where the ray-tracing parameters s0 are already the
// solution (one iteration); written to out[2 * MAXI]
DRT_HD void path_t0par_fp64(const LinkDev &L, int p, double *out) {
    solve_edge_params<LEN_GEN>(L, p, 0.0, L.ps0 + (size_t)p * MAXI, out, out + MAXI,
                      [&](int ty, int idx) { return load_prim_direct<double>(L, 0.0, ty, idx); });
}

DRT_HD void path_warm_fp64(const LinkDev &L, const TimeGridD &tg, int p, int row, double *warm) {
    const double t = tg.t_start + (double)row * tg.chunk * tg.dt;
    // chunk-base solve from the linear predictor s(0) + t ds/dt(0) (solved at load: LinkDev::t0par)
    const double *q = L.t0par + (size_t)(p - L.n_bulk) * (2 * MAXI);
    double start[MAXI];
    for (int j = 0; j < MAXI; ++j) start[j] = q[j] + q[MAXI + j] * t;
    double *w = warm + ((size_t)row * (L.n_paths - L.n_bulk) + (p - L.n_bulk)) * (2 * MAXI);
    solve_edge_params<LEN_GEN>(L, p, t, start, w, w + MAXI,
                      [&](int ty, int idx) { return load_prim_direct<double>(L, t, ty, idx); });
}

// ------------------------------------------------------------------------------------------------
// FP32-bulk form.  Time steps are grouped in chunks of CHUNK consecutive steps.  Per
// (path, chunk) an FP64 base solve at the chunk's first instant t_b gives the path length d_b and
// the phase anchors frac(f_0 d_b / c), frac(df d_b / c) (k_base_fp64).  Per (path, step) the geometry
// runs in FP32 delta numbers (dd): base values at t_b, deltas since t_b, time derivatives; the
// delay is d_b + sum of the segment-length deltas, so the FP32 rounding acts on metre-scale
// deltas, not on the ~100 m path length.

// per (path, chunk) FP64 anchors
struct alignas(16) BaseRec {
    double d;                  // path length at the chunk base (m)
    float ph0, st_hi, st_lo;   // frac(f_0 d / c); frac(df d / c) = st_hi + st_lo
    float pad;
    float seg[MAXI + 1][3];    // segment vectors V_i - V_{i-1} at the chunk base, from FP64 positions
    float pad2[2];             // 96 B: read as six 16-byte words
};

// per (body, chunk) FP32 base pose: rows of R(t_b), O(t_b), v_O(t_b), a, axis k, w(t_b), wdot
struct alignas(16) PoseB { float R[9], O[3], vO[3], a[3], k[3], w, wdot, pad; };   // 96 B

// a row of 16-byte words (PoseB, BaseRec) read with 16-byte loads
template <class T> DRT_HD T ld_row(const T &src) {
    static_assert(sizeof(T) % 16 == 0 && alignof(T) >= 16, "16-byte rows");
    T r;
    const float4 *s = reinterpret_cast<const float4 *>(&src);
    float4 *d = reinterpret_cast<float4 *>(&r);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(T) / 16); ++k) d[k] = s[k];
    return r;
}

DRT_HD void body_pose_base(const BodyD &B, double tb, PoseB &q) {
    double P[POSE_W];
    body_pose_row(B, tb, P);
    for (int j = 0; j < 9; ++j) q.R[j] = (float)P[j];
    for (int j = 0; j < 3; ++j) {
        q.O[j] = (float)P[9 + j];
        q.vO[j] = (float)P[12 + j];
        q.a[j] = (float)B.a[j];
        q.k[j] = (float)B.k[j];
    }
    q.w = (float)(B.w0 + B.wdot * tb);
    q.wdot = (float)B.wdot;
    q.pad = 0.f;
}

DRT_HD void terminal_base(const TermD &m, double tb, PoseB &q) {
    for (int j = 0; j < 9; ++j) q.R[j] = (j % 4 == 0) ? 1.f : 0.f;
    for (int j = 0; j < 3; ++j) {
        q.O[j] = (float)(m.r[j] + m.v[j] * tb + 0.5 * m.a[j] * tb * tb);
        q.vO[j] = (float)(m.v[j] + m.a[j] * tb);
        q.a[j] = (float)m.a[j];
        q.k[j] = j == 2 ? 1.f : 0.f;
    }
    q.w = q.wdot = q.pad = 0.f;
}

// pose of one body tau seconds after its chunk base, as delta numbers: rotation by
// dth = w tau + wdot tau^2 / 2 about k applied to the base pose, written with sin(dth) and the
// versine 2 sin^2(dth/2) so that small rotations lose nothing.
struct PoseDD {
    v3<float> R0, R1, R2, O, dO, vO, w, k;
    float sn, vs;   // sin(dth), 1 - cos(dth)
};
DRT_HD PoseDD pose_dd(const PoseB &row, float tau) {
    const PoseB q = ld_row(row);
    PoseDD P;
    P.R0 = V3<float>(q.R[0], q.R[1], q.R[2]);
    P.R1 = V3<float>(q.R[3], q.R[4], q.R[5]);
    P.R2 = V3<float>(q.R[6], q.R[7], q.R[8]);
    P.O = V3<float>(q.O[0], q.O[1], q.O[2]);
    v3<float> a = V3<float>(q.a[0], q.a[1], q.a[2]), vb = V3<float>(q.vO[0], q.vO[1], q.vO[2]);
    P.dO = vb * tau + a * (0.5f * tau * tau);
    P.vO = vb + a * tau;
    P.k = V3<float>(q.k[0], q.k[1], q.k[2]);
    P.w = P.k * (q.w + q.wdot * tau);
    float dth = q.w * tau + 0.5f * q.wdot * tau * tau;
    float sh = sinf(0.5f * dth);
    P.sn = sinf(dth);
    P.vs = 2.f * sh * sh;
    return P;
}
DRT_HD v3<float> rotb(const PoseDD &P, const float *x) {
    v3<float> v = V3<float>(x[0], x[1], x[2]);
    return V3<float>(dot(P.R0, v), dot(P.R1, v), dot(P.R2, v));
}
// change of a base vector r under the extra rotation: sin(dth) k x r + (1 - cos(dth)) k x (k x r)
DRT_HD v3<float> drot(const PoseDD &P, v3<float> r) {
    v3<float> kr = cross(P.k, r);
    return kr * P.sn + cross(P.k, kr) * P.vs;
}
DRT_HD v3<dd> pose_point_dd(const PoseDD &P, const float *rel) {
    v3<float> rb = rotb(P, rel), dr = drot(P, rb);
    return ddv(P.O + rb, P.dO + dr, P.vO + cross(P.w, rb + dr));
}
DRT_HD v3<dd> pose_dir_dd(const PoseDD &P, const float *d0) {
    v3<float> nb = rotb(P, d0), dn = drot(P, nb);
    return ddv(nb, dn, cross(P.w, nb + dn));
}
// terminal tau seconds after its chunk base, from its base record (stored like a body pose: O = r,
// vO = v, a = a at the chunk's first instant)
DRT_HD v3<dd> terminal_dd(const PoseB &row, float tau) {
    const PoseB q = ld_row(row);
    v3<float> b = V3<float>(q.O[0], q.O[1], q.O[2]), v = V3<float>(q.vO[0], q.vO[1], q.vO[2]);
    v3<float> a = V3<float>(q.a[0], q.a[1], q.a[2]);
    return ddv(b, v * tau + a * (0.5f * tau * tau), v + a * tau);
}

// the FP32 body of primitive (type, idx)
DRT_HD int prim_body_f(const LinkDev &L, int type, int idx) {
    return type == T_R ? L.facesF[idx].body : type == T_D ? L.edgesF[idx].body : L.tilesF[idx].body;
}

// primitive posed from its body's chunk-base row
DRT_HD Prim<dd> load_prim_dd(const LinkDev &L, const PoseB &row, float tau, int type, int idx) {
    Prim<dd> q;
    q.type = type;
    q.idx = idx;
    if (L.body_fixed[prim_body_f(L, type, idx)]) {   // at rest: t0 placement, zero deltas and rates
        const v3<float> O = V3<float>(row.O[0], row.O[1], row.O[2]), z = V3<float>(0.f, 0.f, 0.f);
        auto at = [&](const float *rel) { return ddv(O + V3<float>(rel[0], rel[1], rel[2]), z, z); };
        auto dir = [&](const float *d) { return ddv(V3<float>(d[0], d[1], d[2]), z, z); };
        if (type == T_R) {
            const FaceF &f = L.facesF[idx];
            q.p = at(f.c);
            q.a = dir(f.n);
            q.b = V3<float>(f.u[0], f.u[1], f.u[2]);
            q.h1 = f.hu;
            q.h2 = f.hw;
            q.mat = f.mat;
        } else if (type == T_D) {
            const EdgeF &e = L.edgesF[idx];
            q.p = at(e.a);
            q.a = dir(e.e);
            q.b = V3<float>(e.t0[0], e.t0[1], e.t0[2]);
            q.c = V3<float>(e.n0[0], e.n0[1], e.n0[2]);
            q.h1 = e.len;
            q.h2 = e.wn;
            q.h3 = e.snp;
            q.h4 = e.cnp;
            q.mat = e.mat;
        } else {
            const TileF &tl = L.tilesF[idx];
            q.p = at(tl.c);
            q.a = dir(tl.n);
            q.mat = tl.mat;
        }
        return q;
    }
    PoseDD P = pose_dd(row, tau);
    if (type == T_R) {
        const FaceF &f = L.facesF[idx];
        q.p = pose_point_dd(P, f.c);
        q.a = pose_dir_dd(P, f.n);
        v3<float> ub = rotb(P, f.u);
        q.b = ub + drot(P, ub);
        q.h1 = f.hu;
        q.h2 = f.hw;
        q.mat = f.mat;
    } else if (type == T_D) {
        const EdgeF &e = L.edgesF[idx];
        q.p = pose_point_dd(P, e.a);
        q.a = pose_dir_dd(P, e.e);
        v3<float> tb = rotb(P, e.t0), nb = rotb(P, e.n0);
        q.b = tb + drot(P, tb);
        q.c = nb + drot(P, nb);
        q.h1 = e.len;
        q.h2 = e.wn;
        q.h3 = e.snp;
        q.h4 = e.cnp;
        q.mat = e.mat;
    } else {
        const TileF &tl = L.tilesF[idx];
        q.p = pose_point_dd(P, tl.c);
        q.a = pose_dir_dd(P, tl.n);
        q.mat = tl.mat;
    }
    return q;
}

// FP64 value-only primitive posed from its body's pose record (chunk-base solve)
DRT_HD Prim<double> load_prim_value(const LinkDev &L, const double *Pr, int type, int idx) {
    if (L.body_fixed[prim_body(L, type, idx)]) return val_prim(load_prim_fixed<double>(L, type, idx));
    Pose<double> P = load_pose<double>(Pr);
    Prim<double> q;
    q.type = type;
    q.idx = idx;
    if (type == T_R) {
        const FaceD &f = L.faces[idx];
        q.p = P.O + rot(P, f.c);
        q.a = rot(P, f.n);
        q.b = rot(P, f.u);
        q.h1 = f.hu;
        q.h2 = f.hw;
        q.mat = f.mat;
    } else if (type == T_D) {
        const EdgeD &e = L.edges[idx];
        q.p = P.O + rot(P, e.a);
        q.a = rot(P, e.e);
        q.b = rot(P, e.t0);
        q.c = rot(P, e.n0);
        q.h1 = e.len;
        q.h2 = e.wn;
        q.h3 = e.snp;
        q.h4 = e.cnp;
        q.mat = e.mat;
    } else {
        const TileD &tl = L.tiles[idx];
        q.p = P.O + rot(P, tl.c);
        q.a = rot(P, tl.n);
        q.mat = tl.mat;
    }
    return q;
}

// (path, chunk) FP64 anchors: path length and segment vectors at the chunk's first instant, phase
// seed and per-bin step.  N < 0: the chain length is read at run time (one instance per length).
template <int N = -1>
DRT_HD void path_base_fp64(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const double *pose64, int p,
                           int chunk, BaseRec *out, const double *warm = nullptr) {
    if constexpr (N < 0) {
        with_length(chain_length(L, p), [&](auto NC) {
            path_base_fp64<decltype(NC)::value>(L, tg, fg, pose64, p, chunk, out, warm);
        });
    } else {
        const double tb = tg.t_start + (double)chunk * tg.chunk * tg.dt;
        const int n_chunks = (tg.n_steps + tg.chunk - 1) / tg.chunk;
        const uint32_t code = L.ptypes[p];
        const int4 pi = L.pprims[p];
        const int prim[MAXI] = {pi.x, pi.y, pi.z, pi.w};
        Prim<double> pr[N > 0 ? N : 1];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int ty = (code >> (8 * j)) & 0xff;
            pr[j] = load_prim_value(L, pose_at(pose64, n_chunks, prim_body(L, ty, prim[j]), chunk), ty, prim[j]);
        }
        v3<double> V[N + 2];
        V[0] = val(terminal<double>(L.tx, tb));
        V[N + 1] = val(terminal<double>(L.rx, tb));
        uint32_t fl = 0;
        const double *s0 = L.ps0 + (size_t)p * MAXI;
        if (warm && p >= L.n_bulk) s0 = warm_row(L, warm, chunk, p);
        solve_geometry_any<N>(pr, V, s0, fl);
        BaseRec r;
        double d = 0.0;
#pragma unroll
        for (int i = 0; i <= MAXI; ++i) r.seg[i][0] = r.seg[i][1] = r.seg[i][2] = 0.f;
#pragma unroll
        for (int i = 1; i <= N + 1; ++i) {
            v3<double> sg = V[i] - V[i - 1];
            d += norm(sg);
            r.seg[i - 1][0] = (float)sg.x;
            r.seg[i - 1][1] = (float)sg.y;
            r.seg[i - 1][2] = (float)sg.z;
        }
        const double dc = d * (1 / C0);   // path length over c (s)
        const double x = fg.f0 * dc, y = fg.df * dc;
        double st = y - floor(y);
        double hi = ldexp(rint(ldexp(st, 12)), -12);   // 12 leading bits: k * hi exact in FP32
        r.d = d;
        r.ph0 = (float)(x - floor(x));
        r.st_hi = (float)hi;
        r.st_lo = (float)(st - hi);
        r.pad = 0.f;
        out[(size_t)chunk * L.n_paths + p] = r;
    }
}


// a delta-number primitive without its rates
DRT_HD Prim<de> strip(const Prim<dd> &q) {
    Prim<de> r;
    r.type = q.type;
    r.mat = q.mat;
    r.idx = q.idx;
    r.p = strip(q.p);
    r.a = strip(q.a);
    r.b = q.b;
    r.c = q.c;
    r.h1 = q.h1;
    r.h2 = q.h2;
    r.h3 = q.h3;
    r.h4 = q.h4;
    return r;
}
template <class S> DRT_HD Prim<S> load_prim_as(const LinkDev &L, const PoseB &row, float tau, int type, int idx) {
    if constexpr (std::is_same<S, dd>::value) return load_prim_dd(L, row, tau, type, idx);
    else return strip(load_prim_dd(L, row, tau, type, idx));
}

// Where an FP32-bulk step reads its chunk-base rows: the pose rows of its vertices' bodies and of the
// terminals (slot j < MAXI: vertex j + 1's body; MAXI: TX; MAXI + 1: RX) and its path's anchors (base;
// base2 those of a pair's second carrier, or null), chunk c at pose[slot][c - c0] and
// base[(c - c0) * bstride].  The kernels read them in global memory (c0 = 0, bstride = n_paths): the
// rows of a block's chunks are few and shared by its warps, so they stay in L1 (a copy staged in
// shared memory per block or per warp measured 16-24 % slower).
struct BulkRows {
    const PoseB *pose[MAXI + 2];
    const BaseRec *base, *base2;
    int c0, bstride;
};

// the global-memory rows of path p (base tables [chunk][path], pose table [body + 2][chunk])
DRT_HD BulkRows bulk_rows_global(const LinkDev &L, const PoseB *poseb, const BaseRec *base, const BaseRec *base2,
                                 int n_chunks, int p) {
    BulkRows R;
    const uint32_t code = L.ptypes[p];
    const int4 pi = L.pprims[p];
    const int prim[MAXI] = {pi.x, pi.y, pi.z, pi.w};
#pragma unroll
    for (int j = 0; j < MAXI; ++j) {
        const int ty = (code >> (8 * j)) & 0xff;
        R.pose[j] = poseb + (size_t)(ty == T_NONE ? 0 : prim_body_f(L, ty, prim[j])) * n_chunks;
    }
    R.pose[MAXI] = poseb + (size_t)L.n_bodies * n_chunks;
    R.pose[MAXI + 1] = poseb + (size_t)(L.n_bodies + 1) * n_chunks;
    R.base = base + p;
    R.base2 = base2 ? base2 + p : nullptr;
    R.c0 = 0;
    R.bstride = L.n_paths;
    return R;
}

template <class S> DRT_HD v3<S> terminal_as(const PoseB &q, float tau) {
    if constexpr (std::is_same<S, dd>::value) return terminal_dd(q, tau);
    else return strip(terminal_dd(q, tau));
}

template <class S>
DRT_HD void write_outputs_bulk(const OutD &o, size_t oi, int n, const v3<S> *V, v3<float> seg_first,
                               v3<float> seg_last, double tau, cx<float> a, float fd, uint32_t fl) {
    if (o.tau) o.tau[oi] = tau;
    if (o.amp) {
        float *q = reinterpret_cast<float *>(o.amp) + 2 * oi;
        q[0] = a.re;
        q[1] = a.im;
    }
    if (o.doppler) reinterpret_cast<float *>(o.doppler)[oi] = fd;
    if (o.angles) {
        v3<float> kd = unit(seg_first), ka = -unit(seg_last);
        float *q = o.angles + 4 * oi;
        q[0] = atan2f(kd.y, kd.x);
        q[1] = atan2f(kd.z, hypotf(kd.x, kd.y));
        q[2] = atan2f(ka.y, ka.x);
        q[3] = atan2f(ka.z, hypotf(ka.x, ka.y));
    }
    if (o.flags) o.flags[oi] = (uint8_t)fl;
    if (o.points) {
        double *q = o.points + oi * (MAXI * 3);
        const double qn = nan("");
#pragma unroll
        for (int j = 0; j < MAXI; ++j) {
            bool in = j < n;
            q[3 * j + 0] = in ? (double)V[j + 1].x.b + (double)V[j + 1].x.d : qn;
            q[3 * j + 1] = in ? (double)V[j + 1].y.b + (double)V[j + 1].y.d : qn;
            q[3 * j + 2] = in ? (double)V[j + 1].z.b + (double)V[j + 1].z.d : qn;
        }
    }
}

// list of (link, path, step) triples the FP32-bulk kernels hand to the FP64 redo kernel
struct RedoList { int *count; int4 *items; int cap; };

// synthesis record of one path-step: amplitude (0 if the path does not exist), phase seed and the
// per-bin phase step split hi + lo (cycles)
struct Rec5 { float ar, ai, ph, hi, lo; };

// FP32-bulk (path, time-step): geometry in delta numbers on the chunk anchors, field in FP32.
// Chains with >= 2 diffractions in a segment start their Newton solve from the FP64 chunk-base
// parameters (warm, may be null for the others).  Returns false when the step was queued for the
// FP64 redo (its record is then zero).  S = dd carries the rates the Doppler shift needs, S = de
// (calls without Doppler output) leaves them out.  N, MULTI and OUT as for path_step_fp64_core.
// A second carrier (fg2 with its anchors base2; the same time grid and chunks) shares the geometry:
// its field coefficients and phase record go to *rec2.
template <int N = -1, bool MULTI = true, bool OUT = true, class S = dd>
DRT_HD bool bulk_eval(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const BulkRows &R,
                      const double *warm, int p, int ti, const OutD &out, Rec5 &rec, const RedoList &redo, int link,
                      const FreqGridD *fg2 = nullptr, Rec5 *rec2 = nullptr) {
    if constexpr (N < 0) {
        bool ok = false;
        with_length<len_min<N>()>(chain_length(L, p), [&](auto NC) {
            ok = bulk_eval<decltype(NC)::value, MULTI, OUT, S>(L, tg, fg, R, warm, p, ti, out, rec, redo, link, fg2,
                                                               rec2);
        });
        return ok;
    } else {
    typedef float T;
    rec = Rec5{0.f, 0.f, 0.f, 0.f, 0.f};
    if (rec2) *rec2 = Rec5{0.f, 0.f, 0.f, 0.f, 0.f};
    const int chunk = ti / tg.chunk;
    const float tau_t = (float)(ti - chunk * tg.chunk) * tg.dtf;
    const uint32_t code = L.ptypes[p];
    const int4 pi = L.pprims[p];
    const int prim[MAXI] = {pi.x, pi.y, pi.z, pi.w};
    constexpr int n = N;
    Prim<S> pr[MAXI];
#pragma unroll
    for (int j = 0; j < N; ++j)
        pr[j] = load_prim_as<S>(L, R.pose[j][chunk - R.c0], tau_t, (code >> (8 * j)) & 0xff, prim[j]);
    v3<S> V[MAXI + 2];
    V[0] = terminal_as<S>(R.pose[MAXI][chunk - R.c0], tau_t);
    V[N + 1] = terminal_as<S>(R.pose[MAXI + 1][chunk - R.c0], tau_t);
    uint32_t fl = 0;
    if (MULTI && warm && p >= L.n_bulk) {
        WarmStart32 ws;
        warm_start_at32(L, tg, warm, p, ti, ws);
        solve_geometry<N, MULTI>(pr, V, ws.s, fl, ws.ds, ws.rate);
    } else {
        solve_geometry<N, MULTI>(pr, V, L.ps0 + (size_t)p * MAXI, fl);
    }
    v3<T> P[MAXI + 2];
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 0; i <= MAXI + 1; ++i) {
        if (i > n + 1) break;
        P[i] = val(V[i]);
    }
    fl |= validity<N>(pr, n, P);
    {
        // The FP32 bases carry rounding errors of ~1 ulp of the coordinates (~1e-5 m at 100 m),
        // and the delta rules multiply them by the deltas: the phase error grows with how far an
        // interaction point moved since the chunk base (~6e-4 rad per metre at 60 GHz when a
        // diffraction point slides fast near grazing).  Steps past 0.8 m at 60 GHz (scaled by
        // 1/fc) are left to the FP64 redo.
        float disp2 = 0.f;
        bool finite = true;
#pragma unroll (N >= 0 ? 8 : 1)
        for (int i = 1; i <= MAXI; ++i) {
            if (i > n) break;
            disp2 = fmaxf(disp2, V[i].x.d * V[i].x.d + V[i].y.d * V[i].y.d + V[i].z.d * V[i].z.d);
            finite = finite && isfinite(P[i].x) && isfinite(P[i].y) && isfinite(P[i].z);
        }
        const float dlim = fg2 ? fminf(fg.disp_lim, fg2->disp_lim) : fg.disp_lim;
        // A step past the displacement limit needs FP64 for its phase; an invalid step has none, and its
        // flags stand when every validity margin clears 100x the FP32 error bound (most such steps are
        // invalid: interaction points of a chain that left its faces run far and fast, and the FP32
        // decisions there have margins of metres).
        const bool invalid_clear = (fl & (F_FACE | F_EDGE | F_SIDE)) && !(fl & F_NEAR100);
        if (disp2 > dlim * dlim && !invalid_clear) fl |= F_REDO64;
        fl &= ~F_NEAR100;
        if (!finite || (fl & (F_REDO64 | F_NOCONV | F_DEGEN))) {
            // geometry FP32 cannot resolve: queue this path-step for the FP64 redo kernel (rare,
            // see F_REDO64); the list holds every path-step in the worst case
            if (redo.count) {
#ifdef __CUDA_ARCH__
                // one claim per warp: the queued steps of a warp (consecutive steps of one path)
                // stay adjacent in the list, so the redo warps run one chain signature each
                const unsigned m = __activemask();
                const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                int k0 = 0;
                if (lane == leader) k0 = atomicAdd(redo.count, __popc(m));
                const int k = __shfl_sync(m, k0, leader) + __popc(m & ((1u << lane) - 1u));
#else
                int k = (*redo.count)++;
#endif
                if (k < redo.cap) redo.items[k] = make_int4(link, p, ti, 0);
            }
            return false;
        }
    }
    const BaseRec B = ld_row(R.base[(size_t)(chunk - R.c0) * R.bstride]);
    float dd_len = 0.f;   // change of the path length since the chunk base
    v3<float> seg[MAXI + 2];
#pragma unroll (N >= 0 ? 8 : 1)
    for (int i = 1; i <= MAXI + 1; ++i) {
        if (i > n + 1) break;
        v3<S> sv = V[i] - V[i - 1];
        dd_len += norm(sv).d;
        // segment vector: FP64-accurate base + FP32 delta
        seg[i] = V3<float>(B.seg[i - 1][0] + sv.x.d, B.seg[i - 1][1] + sv.y.d, B.seg[i - 1][2] + sv.z.d);
    }
    // as in the FP64 form: an invalid step's field coefficients only for the amplitude output
    const bool field = !fl || (OUT && out.amp && !(fl & F_DEGEN));
    cx<T> a = field ? amplitude<N>(L, pr, n, seg, fg.fcf) : C<T>(T(0), T(0));
    if constexpr (OUT) {
        if (out.tau || out.amp || out.doppler || out.angles || out.flags || out.points) {
            T fd = 0.f;
            if constexpr (std::is_same<S, dd>::value) fd = doppler<N>(n, V, seg, fg.fcf);
            const size_t oi = (size_t)ti * L.n_paths + L.perm[p];
            v3<float> s_last = seg[1];
#pragma unroll (N >= 0 ? 8 : 1)
            for (int i = 2; i <= MAXI + 1; ++i)
                if (i == n + 1) s_last = seg[i];
            write_outputs_bulk(out, oi, n, V, seg[1], s_last, (B.d + (double)dd_len) / C0, a, fd, fl);
        }
    }
    auto phase_record = [&](const FreqGridD &g, const BaseRec &Bk, cx<T> ak, Rec5 &r) {
        float x = g.f0c * dd_len;
        x -= floorf(x);
        float ph = Bk.ph0 + x;
        ph -= floorf(ph);
        r.ar = fl ? 0.f : ak.re;
        r.ai = fl ? 0.f : ak.im;
        r.ph = ph;
        r.hi = Bk.st_hi;
        r.lo = fmaf(g.dfc, dd_len, Bk.st_lo);
    };
    phase_record(fg, B, a, rec);
    if (fg2) {
        const cx<T> a2 = field ? amplitude<N>(L, pr, n, seg, fg2->fcf) : C<T>(T(0), T(0));
        phase_record(*fg2, ld_row(R.base2[(size_t)(chunk - R.c0) * R.bstride]), a2, *rec2);
    }
    return true;
    }
}

template <int N = -1, bool MULTI = true, bool OUT = true, class S = dd>
DRT_HD void path_step_bulk(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const BulkRows &R,
                           const double *warm, int p, int ti, const OutD &out, const RecD &rec,
                           const RedoList &redo) {
    Rec5 r;
    bulk_eval<N, MULTI, OUT, S>(L, tg, fg, R, warm, p, ti, out, r, redo, 0);
    if (rec.rec_a) {
        size_t ri = (size_t)ti * L.n_paths + p;
        rec.rec_a[ri] = make_float4(r.ar, r.ai, r.ph, r.hi);
        rec.rec_b[ri] = r.lo;
    }
}

// FP64 redo of one queued FP32-bulk path-step (FP32 output formats); DUAL: with the rates the Doppler
// output needs (dual numbers), else values only
template <bool DUAL>
DRT_HD void path_step_redo_as(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, int p, int ti,
                              const OutD &out, const RecD &rec, const double *warm, double *rec64 = nullptr) {
    const double t = tg.t_start + ti * tg.dt;
    if constexpr (DUAL) {
        path_step_fp64_core<LEN_ANY, true, true, dl<double>>(
            L, tg, fg, p, ti, out, rec, true, [&](int ty, int idx) { return load_prim_direct<double>(L, t, ty, idx); },
            warm, rec64);
    } else {
        path_step_fp64_core<LEN_ANY, true, true, double>(
            L, tg, fg, p, ti, out, rec, true,
            [&](int ty, int idx) { return val_prim(load_prim_direct<double>(L, t, ty, idx)); }, warm, rec64);
    }
}

// one (path, step) of the FP64 form from the per-step pose table; DUAL = false when no Doppler
// output is asked for (values only); N, MULTI and OUT as for path_step_fp64_core
template <bool DUAL, int N = -1, bool MULTI = true, bool OUT = true>
DRT_HD void path_step_fp64(const LinkDev &L, const TimeGridD &tg, const FreqGridD &fg, const double *pose, int p,
                           int ti, const OutD &out, const RecD &rec, bool f32out = false,
                           const double *warm = nullptr) {
    if constexpr (DUAL) {
        path_step_fp64_core<N, MULTI, OUT, dl<double>>(
            L, tg, fg, p, ti, out, rec, f32out,
            [&](int ty, int idx) { return load_prim<double>(L, pose, tg.n_steps, ti, ty, idx); }, warm);
    } else {
        path_step_fp64_core<N, MULTI, OUT, double>(
            L, tg, fg, p, ti, out, rec, f32out,
            [&](int ty, int idx) {
                return load_prim_value(L, pose_at(pose, tg.n_steps, prim_body(L, ty, idx), ti), ty, idx);
            },
            warm);
    }
}

}  // namespace drt
