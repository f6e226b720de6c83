// pf_dual.cuh -- first-order dual numbers (value and one directional
// derivative) for the tangent-linear run of the 1D batch kernel.
//
// A model parameter theta (M_phi, A or b) enters the step through the
// parameter block; seeding its entry with derivative 1 and running the same
// step code on Dual<T> carries d(state)/d(theta) along with the state, so the
// derivative is that of the discrete step, exact up to rounding.
#pragma once
#include <cmath>
#include <cuda_runtime.h>

namespace pf {

template <typename T>
struct Dual {
    T v;   // value
    T t;   // derivative along the seeded direction
    __host__ __device__ Dual() : v(0), t(0) {}
    __host__ __device__ Dual(double x) : v(T(x)), t(0) {}   // constants carry no derivative
    __host__ __device__ Dual(T x, T dx, int) : v(x), t(dx) {}
    __host__ __device__ explicit operator double() const { return (double)v; }
};

template <typename T>
struct IsDual {
    static constexpr bool value = false;
};
template <typename T>
struct IsDual<Dual<T>> {
    static constexpr bool value = true;
};

template <typename T>
__host__ __device__ inline Dual<T> make_dual(T v, T t) {
    return Dual<T>(v, t, 0);
}

template <typename T>
__host__ __device__ inline Dual<T> operator+(Dual<T> a, Dual<T> b) {
    return make_dual(a.v + b.v, a.t + b.t);
}
template <typename T>
__host__ __device__ inline Dual<T> operator-(Dual<T> a, Dual<T> b) {
    return make_dual(a.v - b.v, a.t - b.t);
}
template <typename T>
__host__ __device__ inline Dual<T> operator-(Dual<T> a) {
    return make_dual(-a.v, -a.t);
}
template <typename T>
__host__ __device__ inline Dual<T> operator*(Dual<T> a, Dual<T> b) {
    return make_dual(a.v * b.v, a.v * b.t + a.t * b.v);
}
template <typename T>
__host__ __device__ inline Dual<T> operator/(Dual<T> a, Dual<T> b) {
    const T q = a.v / b.v;
    return make_dual(q, (a.t - q * b.t) / b.v);
}
template <typename T>
__host__ __device__ inline Dual<T>& operator+=(Dual<T>& a, Dual<T> b) {
    a = a + b;
    return a;
}
template <typename T>
__host__ __device__ inline Dual<T>& operator-=(Dual<T>& a, Dual<T> b) {
    a = a - b;
    return a;
}
template <typename T>
__host__ __device__ inline Dual<T>& operator*=(Dual<T>& a, Dual<T> b) {
    a = a * b;
    return a;
}

// natural logarithm: d ln x = dx / x
__device__ inline Dual<float> flog(Dual<float> x) { return make_dual(logf(x.v), x.t / x.v); }
__device__ inline Dual<double> flog(Dual<double> x) { return make_dual(log(x.v), x.t / x.v); }

}  // namespace pf
