// Common device types and helpers of the LB IMEX-TR kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbtr {

// Complex values are float2 / double2: .x real, .y imaginary.
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
    cplx<T> c; c.x = re; c.y = im; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// multiply by -i (sign<0) or +i (sign>0)
template <int SIGN, typename C> __device__ __forceinline__ C cmul_i(C a) {
    C c;
    if (SIGN < 0) { c.x = a.y; c.y = -a.x; } else { c.x = -a.y; c.y = a.x; }
    return c;
}

// Signed wavenumber of array index i on an M-point axis: the paper's K_M = [-M/2, M/2).
__device__ __forceinline__ int wavenum(int i, int m) { return i < (m >> 1) ? i : i - m; }

// Geometry of one problem as the kernels see it.
struct Geom {
    int dim;        // 2 or 3
    int m;          // points per axis
    int h;          // m/2: complex length of the x transform and width of the main spectrum
    int rows;       // m^(dim-1): number of x rows
    long long n;    // m^dim
    double qx, qy, qz;   // (2 pi / L_a)^2 per axis: |Bk|^2 = qx kx^2 + qy ky^2 + qz kz^2
    double xi2, tau, gamma;
};

// Lambda_k = xi^2 (1 - |Bk|^2)^2 for integer wavenumbers.
__device__ __forceinline__ double lam_of(const Geom& g, int kx, int ky, int kz) {
    double b = g.qx * (double)(kx * kx) + g.qy * (double)(ky * ky) + g.qz * (double)(kz * kz);
    double t = 1.0 - b;
    return g.xi2 * t * t;
}

}  // namespace lbtr
