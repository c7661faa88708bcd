// drt_math.cuh -- small value types of the DRT kernels: 3-vectors, dual numbers (value + time
// derivative, carried through the geometry so interaction-point velocities fall out of it),
// complex numbers.  Header-only device code.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace drt {

#define DRT_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------------------------------------------
// dual numbers: x = v + d * eps with eps^2 = 0; d is the time derivative
template <class T> struct dl { T v, d; };
template <class T> DRT_HD dl<T> D(T v, T d) { return dl<T>{v, d}; }
template <class T> DRT_HD dl<T> operator+(dl<T> a, dl<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> DRT_HD dl<T> operator-(dl<T> a, dl<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> DRT_HD dl<T> operator-(dl<T> a) { return {-a.v, -a.d}; }
template <class T> DRT_HD dl<T> operator*(dl<T> a, dl<T> b) { return {a.v * b.v, fma(a.d, b.v, a.v * b.d)}; }
template <class T> DRT_HD dl<T> operator*(dl<T> a, T s) { return {a.v * s, a.d * s}; }
template <class T> DRT_HD dl<T> operator*(T s, dl<T> a) { return {a.v * s, a.d * s}; }
// one reciprocal per quotient and one reciprocal square root per root: division and square root
// are multi-instruction sequences on the FP64 pipe, which bounds the FP64 form
template <class T> DRT_HD dl<T> operator/(dl<T> a, dl<T> b) {
    const T inv = T(1) / b.v;
    const T q = a.v * inv;
    return {q, (a.d - q * b.d) * inv};
}
template <class T> DRT_HD dl<T> dsqrt(dl<T> a) {
    if (!(a.v > T(0))) return {sqrt(a.v), a.d / T(0)};   // zero length: value 0, rate undefined
    const T rs = rsqrt(a.v);
    return {a.v * rs, T(0.5) * a.d * rs};
}

// ------------------------------------------------------------------------------------------------
// delta numbers of the FP32-bulk form: x = b + d, where b is the value at the chunk's base instant
// (FP32, only ever multiplied by small deltas), d the change since then, carried with rules that
// never subtract two large numbers (d(xy) = b_x d_y + d_x b_y + d_x d_y, d(x/y) = (d_x - q d_y)/y,
// d(sqrt x) = d_x / (sqrt(x) + sqrt(b_x))), and v the time derivative of x (dual part).
struct dd { float b, d, v; };
DRT_HD dd DD(float b, float d, float v) { return dd{b, d, v}; }
DRT_HD dd operator+(dd a, dd c) { return {a.b + c.b, a.d + c.d, a.v + c.v}; }
DRT_HD dd operator-(dd a, dd c) { return {a.b - c.b, a.d - c.d, a.v - c.v}; }
DRT_HD dd operator-(dd a) { return {-a.b, -a.d, -a.v}; }
DRT_HD dd operator*(dd a, dd c) {
    float af = a.b + a.d, cf = c.b + c.d;
    return {a.b * c.b, fmaf(a.b, c.d, a.d * cf), fmaf(a.v, cf, af * c.v)};
}
DRT_HD dd operator*(dd a, float s) { return {a.b * s, a.d * s, a.v * s}; }
DRT_HD dd operator*(float s, dd a) { return {a.b * s, a.d * s, a.v * s}; }
DRT_HD dd operator/(dd a, dd c) {
    float q = a.b / c.b, cf = c.b + c.d;
    float d = (a.d - q * c.d) / cf;
    return {q, d, (a.v - (q + d) * c.v) / cf};
}
DRT_HD dd dsqrt(dd a) {
    float r = sqrtf(fmaxf(a.b, 0.f)), rf = sqrtf(fmaxf(a.b + a.d, 0.f));
    float den = rf + r;
    return {r, den > 0.f ? a.d / den : 0.f, rf > 0.f ? a.v / (2.f * rf) : 0.f};
}

// delta numbers without the rate part, for steps that need no Doppler shift: same rules as dd
struct de { float b, d; };
DRT_HD de operator+(de a, de c) { return {a.b + c.b, a.d + c.d}; }
DRT_HD de operator-(de a, de c) { return {a.b - c.b, a.d - c.d}; }
DRT_HD de operator-(de a) { return {-a.b, -a.d}; }
DRT_HD de operator*(de a, de c) { return {a.b * c.b, fmaf(a.b, c.d, a.d * (c.b + c.d))}; }
DRT_HD de operator*(de a, float s) { return {a.b * s, a.d * s}; }
DRT_HD de operator*(float s, de a) { return {a.b * s, a.d * s}; }
DRT_HD de operator/(de a, de c) {
    float q = a.b / c.b;
    return {q, (a.d - q * c.d) / (c.b + c.d)};
}
DRT_HD de dsqrt(de a) {
    float r = sqrtf(fmaxf(a.b, 0.f)), rf = sqrtf(fmaxf(a.b + a.d, 0.f));
    float den = rf + r;
    return {r, den > 0.f ? a.d / den : 0.f};
}
DRT_HD de strip(dd a) { return {a.b, a.d}; }

// scalar traits: real type, full value, time derivative, constants
template <class S> struct ST;
template <class T> struct ST<dl<T>> {
    typedef T R;
    static DRT_HD T val(dl<T> x) { return x.v; }
    static DRT_HD T rate(dl<T> x) { return x.d; }
    static DRT_HD dl<T> cst(T x) { return {x, T(0)}; }
};
template <> struct ST<dd> {
    typedef float R;
    static DRT_HD float val(dd x) { return x.b + x.d; }
    static DRT_HD float rate(dd x) { return x.v; }
    static DRT_HD dd cst(float x) { return {x, 0.f, 0.f}; }
};
template <> struct ST<de> {
    typedef float R;
    static DRT_HD float val(de x) { return x.b + x.d; }
    static DRT_HD float rate(de) { return 0.f; }
    static DRT_HD de cst(float x) { return {x, 0.f}; }
};
template <> struct ST<double> {   // plain values (FP64 chunk-base solve: no derivative needed)
    typedef double R;
    static DRT_HD double val(double x) { return x; }
    static DRT_HD double rate(double) { return 0.0; }
    static DRT_HD double cst(double x) { return x; }
};
template <> struct ST<float> {   // plain FP32 values (the first Newton iterations of a warm-start solve)
    typedef float R;
    static DRT_HD float val(float x) { return x; }
    static DRT_HD float rate(float) { return 0.f; }
    static DRT_HD float cst(float x) { return x; }
};
DRT_HD double dsqrt(double x) { return sqrt(x); }
template <class S> DRT_HD typename ST<S>::R sval(S x) { return ST<S>::val(x); }
template <class S> DRT_HD typename ST<S>::R srate(S x) { return ST<S>::rate(x); }
template <class S> DRT_HD S scst(typename ST<S>::R x) { return ST<S>::cst(x); }

// ------------------------------------------------------------------------------------------------
// 3-vectors over any scalar (T, dl<T> or dd)
template <class E> struct v3 { E x, y, z; };
template <class E> DRT_HD v3<E> V3(E x, E y, E z) { return v3<E>{x, y, z}; }
template <class E> DRT_HD v3<E> operator+(v3<E> a, v3<E> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class E> DRT_HD v3<E> operator-(v3<E> a, v3<E> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class E> DRT_HD v3<E> operator-(v3<E> a) { return {-a.x, -a.y, -a.z}; }
template <class E, class S> DRT_HD v3<E> operator*(v3<E> a, S s) { return {a.x * s, a.y * s, a.z * s}; }
template <class E> DRT_HD E dot(v3<E> a, v3<E> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class E> DRT_HD v3<E> cross(v3<E> a, v3<E> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// value / derivative parts of a vector of scalars, and promotion of a plain vector
template <class S> DRT_HD v3<typename ST<S>::R> val(v3<S> a) { return {sval(a.x), sval(a.y), sval(a.z)}; }
template <class S> DRT_HD v3<typename ST<S>::R> der(v3<S> a) { return {srate(a.x), srate(a.y), srate(a.z)}; }
template <class T> DRT_HD v3<dl<T>> dual(v3<T> v, v3<T> d) { return {{v.x, d.x}, {v.y, d.y}, {v.z, d.z}}; }
DRT_HD v3<dd> ddv(v3<float> b, v3<float> d, v3<float> v) { return {{b.x, d.x, v.x}, {b.y, d.y, v.y}, {b.z, d.z, v.z}}; }
DRT_HD double norm(v3<double> a) { return sqrt(dot(a, a)); }
DRT_HD float norm(v3<float> a) { return sqrtf(dot(a, a)); }
template <class T> DRT_HD dl<T> norm(v3<dl<T>> a) { return dsqrt(dot(a, a)); }
DRT_HD dd norm(v3<dd> a) { return dsqrt(dot(a, a)); }
DRT_HD de norm(v3<de> a) { return dsqrt(dot(a, a)); }
DRT_HD v3<double> unit(v3<double> a) { return a * rsqrt(dot(a, a)); }
DRT_HD v3<float> unit(v3<float> a) { return a * (1.f / norm(a)); }
// x^(-1/2) of a dual number: value rsqrt(x), rate -x'/2 x^(-3/2)
template <class T> DRT_HD v3<dl<T>> unit(v3<dl<T>> a) {
    const dl<T> q = dot(a, a);
    const T rs = rsqrt(q.v);
    const dl<T> inv = {rs, T(-0.5) * q.d * rs * rs * rs};
    return a * inv;
}
DRT_HD v3<dd> unit(v3<dd> a) { return a * (scst<dd>(1.f) / norm(a)); }
DRT_HD v3<de> unit(v3<de> a) { return a * (scst<de>(1.f) / norm(a)); }
DRT_HD v3<de> strip(v3<dd> a) { return {strip(a.x), strip(a.y), strip(a.z)}; }

// ------------------------------------------------------------------------------------------------
// complex numbers and complex 3-vectors (polarisation tracking)
template <class T> struct cx { T re, im; };
template <class T> DRT_HD cx<T> C(T re, T im) { return cx<T>{re, im}; }
template <class T> DRT_HD cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> DRT_HD cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> DRT_HD cx<T> operator-(cx<T> a) { return {-a.re, -a.im}; }
template <class T> DRT_HD cx<T> operator*(cx<T> a, cx<T> b) {
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
template <class T> DRT_HD cx<T> operator*(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <class T> DRT_HD cx<T> operator*(T s, cx<T> a) { return {a.re * s, a.im * s}; }
template <class T> DRT_HD cx<T> cdiv(cx<T> a, cx<T> b) {
    // a conj(b) / |b|^2 with one reciprocal (the magnitudes here, permittivities and continued-
    // fraction terms, are far from the exponent range where Smith's scaling would be needed)
    const T inv = T(1) / fma(b.re, b.re, b.im * b.im);
    return {fma(a.re, b.re, a.im * b.im) * inv, fma(a.im, b.re, -a.re * b.im) * inv};
}
template <class T> DRT_HD T cabs2(cx<T> a) { return a.re * a.re + a.im * a.im; }
// principal square root (Re >= 0)
template <class T> DRT_HD cx<T> csqrt_(cx<T> z) {
    T r = sqrt(z.re * z.re + z.im * z.im);   // |z| of relative permittivities: no overflow scaling
    if (r == T(0)) return {T(0), T(0)};
    // one reciprocal square root gives both t = sqrt(h) and 1/t
    if (z.re >= T(0)) {
        const T h = T(0.5) * (r + z.re), rs = rsqrt(h);
        return {h * rs, T(0.5) * z.im * rs};
    }
    const T h = T(0.5) * (r - z.re), rs = rsqrt(h);
    return {T(0.5) * fabs(z.im) * rs, copysign(h * rs, z.im)};
}
template <class T> DRT_HD cx<T> cexpj(T ph) {   // exp(j ph)
    T s, c;
    sincos(ph, &s, &c);
    return {c, s};
}

template <class T> struct c3 { cx<T> x, y, z; };
template <class T> DRT_HD c3<T> operator+(c3<T> a, c3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> DRT_HD c3<T> cscale(v3<T> e, cx<T> s) { return {s * e.x, s * e.y, s * e.z}; }
template <class T> DRT_HD c3<T> cscale(c3<T> E, cx<T> s) { return {E.x * s, E.y * s, E.z * s}; }
template <class T> DRT_HD cx<T> cdot(c3<T> E, v3<T> e) { return E.x * e.x + E.y * e.y + E.z * e.z; }
template <class T> DRT_HD T cnorm(c3<T> E) { return sqrt(cabs2(E.x) + cabs2(E.y) + cabs2(E.z)); }

// acc[j] += z w^j, j < KT, for |w| = 1 (one path's terms across a frequency tile).  Where |Im w| >= 1/4
// the three-term recurrence z_{j+1} = 2 Re(w) z_j - z_{j-1} (w + 1/w = 2 Re w on the unit circle)
// costs 2 FMA per term instead of the 4 of a complex rotation; a rounding error made at one term
// reaches a later one scaled by at most 1 / |Im w| <= 4, so the error stays below 4 j eps.  Near
// w = +-1 the rotation, whose error grows like j eps, is kept.
#ifdef __CUDACC__
template <int KT>
__device__ __forceinline__ void add_geometric(float2 (&acc)[KT], float zr, float zi, float wr, float wi) {
    if (fabsf(wi) >= 0.25f) {
        const float c2 = 2.f * wr;
        float ar = zr, ai = zi;
        float br = fmaf(zr, wr, -zi * wi), bi = fmaf(zr, wi, zi * wr);
        acc[0].x += ar;
        acc[0].y += ai;
#pragma unroll
        for (int j = 1; j < KT; ++j) {
            acc[j].x += br;
            acc[j].y += bi;
            const float cr = fmaf(c2, br, -ar), ci = fmaf(c2, bi, -ai);
            ar = br;
            ai = bi;
            br = cr;
            bi = ci;
        }
    } else {
#pragma unroll
        for (int j = 0; j < KT; ++j) {
            acc[j].x += zr;
            acc[j].y += zi;
            const float nr = fmaf(zr, wr, -zi * wi);
            zi = fmaf(zr, wi, zi * wr);
            zr = nr;
        }
    }
}
#endif

}  // namespace drt
