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
template <class T> DRT_HD dl<T> operator/(dl<T> a, dl<T> b) {
    T q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <class T> DRT_HD dl<T> dsqrt(dl<T> a) {
    T r = sqrt(a.v);
    return {r, a.d / (T(2) * r)};
}

// ------------------------------------------------------------------------------------------------
// 3-vectors over any scalar (T or dl<T>)
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

// value / derivative parts of a dual vector, and promotion of a plain vector
template <class T> DRT_HD v3<T> val(v3<dl<T>> a) { return {a.x.v, a.y.v, a.z.v}; }
template <class T> DRT_HD v3<T> der(v3<dl<T>> a) { return {a.x.d, a.y.d, a.z.d}; }
template <class T> DRT_HD v3<dl<T>> dual(v3<T> v, v3<T> d) { return {{v.x, d.x}, {v.y, d.y}, {v.z, d.z}}; }
template <class T> DRT_HD T norm(v3<T> a) { return sqrt(dot(a, a)); }
template <class T> DRT_HD dl<T> norm(v3<dl<T>> a) { return dsqrt(dot(a, a)); }
template <class T> DRT_HD v3<T> unit(v3<T> a) { return a * (T(1) / norm(a)); }

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
    // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        T r = b.im / b.re, den = b.re + b.im * r;
        return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
    }
    T r = b.re / b.im, den = b.re * r + b.im;
    return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}
template <class T> DRT_HD T cabs2(cx<T> a) { return a.re * a.re + a.im * a.im; }
// principal square root (Re >= 0)
template <class T> DRT_HD cx<T> csqrt_(cx<T> z) {
    T r = hypot(z.re, z.im);
    if (r == T(0)) return {T(0), T(0)};
    if (z.re >= T(0)) {
        T t = sqrt(T(0.5) * (r + z.re));
        return {t, z.im / (T(2) * t)};
    }
    T t = sqrt(T(0.5) * (r - z.re));
    return {fabs(z.im) / (T(2) * t), copysign(t, z.im)};
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

}  // namespace drt
