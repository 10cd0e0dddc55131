// dual.cuh -- forward-mode derivative numbers for the tangent-linear step.
//
// Dual<T, N> carries a value and its derivatives along N directions; every
// arithmetic operation applies the chain rule to the derivative part.  The
// step's device functions that are templated on their arithmetic type
// (moments, equilibrium, collision, the boundary solver's right-hand side)
// evaluated on Dual numbers give the step together with its directional
// derivatives.  Comparisons look at the value only (a branch taken at the
// point of evaluation).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace lbmgb {

// the plain overloads stay visible beside the Dual ones below
using ::rsqrt;
using ::sqrt;

template <typename T, int N>
struct Dual {
    T v;
    T d[N];

    __host__ __device__ constexpr Dual() : v(0), d{} {}
    template <typename U, typename = std::enable_if_t<std::is_arithmetic<U>::value>>
    __host__ __device__ constexpr Dual(U x) : v(T(x)), d{} {}

    __host__ __device__ Dual& operator+=(const Dual& b)
    {
        v += b.v;
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] += b.d[k];
        return *this;
    }
    __host__ __device__ Dual& operator-=(const Dual& b)
    {
        v -= b.v;
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] -= b.d[k];
        return *this;
    }
    __host__ __device__ Dual& operator*=(const Dual& b)
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = d[k] * b.v + v * b.d[k];
        v *= b.v;
        return *this;
    }
};

template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator+(Dual<T, N> a, const Dual<T, N>& b)
{
    return a += b;
}
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator-(Dual<T, N> a, const Dual<T, N>& b)
{
    return a -= b;
}
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator*(Dual<T, N> a, const Dual<T, N>& b)
{
    return a *= b;
}
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator-(const Dual<T, N>& a)
{
    Dual<T, N> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b)
{
    // (a / b)' = (a' - (a / b) b') / b
    Dual<T, N> r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}

// mixed forms with plain numbers
#define LBM_DUAL_MIXED(OP)                                                                  \
    template <typename T, int N, typename U,                                                \
              typename = std::enable_if_t<std::is_arithmetic<U>::value>>                    \
    __host__ __device__ inline Dual<T, N> operator OP(const Dual<T, N>& a, U b)             \
    {                                                                                       \
        return a OP Dual<T, N>(b);                                                          \
    }                                                                                       \
    template <typename T, int N, typename U,                                                \
              typename = std::enable_if_t<std::is_arithmetic<U>::value>>                    \
    __host__ __device__ inline Dual<T, N> operator OP(U a, const Dual<T, N>& b)             \
    {                                                                                       \
        return Dual<T, N>(a) OP b;                                                          \
    }
LBM_DUAL_MIXED(+)
LBM_DUAL_MIXED(-)
LBM_DUAL_MIXED(*)
LBM_DUAL_MIXED(/)
#undef LBM_DUAL_MIXED

template <typename T, int N>
__host__ __device__ inline bool operator<(const Dual<T, N>& a, const Dual<T, N>& b)
{
    return a.v < b.v;
}
template <typename T, int N>
__host__ __device__ inline bool operator>(const Dual<T, N>& a, const Dual<T, N>& b)
{
    return a.v > b.v;
}
template <typename T, int N, typename U, typename = std::enable_if_t<std::is_arithmetic<U>::value>>
__host__ __device__ inline bool operator<(const Dual<T, N>& a, U b)
{
    return a.v < T(b);
}
template <typename T, int N, typename U, typename = std::enable_if_t<std::is_arithmetic<U>::value>>
__host__ __device__ inline bool operator>(const Dual<T, N>& a, U b)
{
    return a.v > T(b);
}

// sqrt(a)' = a' / (2 sqrt a);  rsqrt(a)' = -a' rsqrt(a) / (2 a)
template <typename T, int N>
__device__ inline Dual<T, N> sqrt(const Dual<T, N>& a)
{
    Dual<T, N> r;
    r.v = ::sqrt(a.v);
    const T h = T(0.5) / r.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
    return r;
}
template <typename T, int N>
__device__ inline Dual<T, N> rsqrt(const Dual<T, N>& a)
{
    Dual<T, N> r;
    r.v = T(1) / ::sqrt(a.v);
    const T h = T(-0.5) * r.v / a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
    return r;
}

template <typename C>
struct DualTraits {
    using Value = C;
    static constexpr int N = 0;
};
template <typename T, int N_>
struct DualTraits<Dual<T, N_>> {
    using Value = T;
    static constexpr int N = N_;
};

}  // namespace lbmgb
