// Kernels on half spectra (Lanczos vectors) and the random generator of the library.
//
// A half spectrum of length len = rows * (H + 1) holds main[rows][H] followed by
// nyq[rows] (the storage of passes.cuh).  The real inner product of two real fields
// in terms of their paper-normalised coefficients is
//     <x, y> = sum_k w_k Re(conj(x_k) y_k),  w_k = 2 for 0 < kx < M/2, else 1,
// which equals <x, y>_N by Parseval.
#pragma once
#include "common.cuh"
#include "reduce.cuh"

namespace lbtr {

struct SpecGeom {
    long long len;     // rows * (H + 1)
    int dim, m, rows;
    const void* qtab;  // [3][M] |Bk|^2 pieces (type T)
};

template <typename T>
__device__ __forceinline__ T spec_weight(const SpecGeom& g, long long i) {
    const int H = g.m >> 1;
    const long long nmain = (long long)g.rows * H;
    return (i < nmain && (i % H) != 0) ? (T)2 : (T)1;
}

template <typename T>
__device__ __forceinline__ T spec_lambda(const SpecGeom& g, long long i, T xi2) {
    const int H = g.m >> 1;
    const long long nmain = (long long)g.rows * H;
    const T* qt = static_cast<const T*>(g.qtab);
    int kx, row;
    if (i < nmain) { kx = (int)(i % H); row = (int)(i / H); } else { kx = H; row = (int)(i - nmain); }
    T bk2 = (g.dim == 3) ? qt[kx] + qt[g.m + (row % g.m)] + qt[2 * g.m + row / g.m] : qt[kx] + qt[g.m + row];
    T t = (T)1 - bk2;
    return xi2 * t * t;
}

// Elements per thread of k_spec_multidot: the warp reduction of every vector's sum is paid
// once per SPEC_MD_E loads, so a larger count amortises it (the kernel is bound by those
// reductions, not by memory, when it is small).
constexpr int SPEC_MD_E = 16;

// partials[j][block] = sum over this block's elements of w (/(Lambda + sigma) if minv)
//                      * Re(conj(Q_j) x), for j < nvec; a block covers SPEC_MD_E * blockDim.x
//                      elements
template <typename T>
__global__ void k_spec_multidot(const cplx<T>* Q, long long ldq, int nvec, const cplx<T>* x, SpecGeom g,
                                int minv, T xi2, T sigma, double* partials) {
    extern __shared__ double sred[];       // [nvec][nwarps]
    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int E = SPEC_MD_E;
    auto idx_of = [&](int e) { return ((long long)blockIdx.x * E + e) * blockDim.x + threadIdx.x; };
    cplx<T> xv[E];
    T wv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const long long i = idx_of(e);
        if (i < g.len) {
            xv[e] = x[i];
            T w = spec_weight<T>(g, i);
            if (minv) w = w / (spec_lambda<T>(g, i, xi2) + sigma);
            wv[e] = w;
        } else {
            xv[e] = mk<T>((T)0, (T)0);
            wv[e] = (T)0;
        }
    }
    for (int j = 0; j < nvec; ++j) {
        const cplx<T>* q = Q + (long long)j * ldq;
        // the loads of the E elements first (all in flight), then the products in order
        cplx<T> av[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const long long i = idx_of(e);
            av[e] = i < g.len ? q[i] : mk<T>((T)0, (T)0);
        }
        Acc<T> acc;
#pragma unroll
        for (int e = 0; e < E; ++e) acc.add(wv[e] * (av[e].x * xv[e].x + av[e].y * xv[e].y));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc.add_shfl(off);
        if (lane == 0) sred[j * nw + warp] = acc.get();
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nvec; j += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sred[j * nw + w];
        partials[(long long)j * gridDim.x + blockIdx.x] = s;
    }
}

// out[j] = sum_b partials[j][b] (fixed order), one warp per j
static __global__ void k_partials_sum(const double* partials, int nblocks, int nvec, double* out) {
    const int lane = threadIdx.x & 31;
    for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < nvec; j += gridDim.x * (blockDim.x >> 5)) {
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) s += partials[(long long)j * nblocks + b];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) out[j] = s;
    }
}

// y -= sum_j c[j] Q_j   (c in device memory, nvec <= 1024)
template <typename T>
__global__ void k_spec_multiaxpy(const cplx<T>* Q, long long ldq, int nvec, const double* c, cplx<T>* y,
                                 long long len) {
    extern __shared__ double sc[];
    for (int j = threadIdx.x; j < nvec; j += blockDim.x) sc[j] = c[j];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        cplx<T> acc = y[i];
        for (int j = 0; j < nvec; ++j) {
            const cplx<T> q = Q[(long long)j * ldq + i];
            const T cj = (T)sc[j];
            acc.x -= cj * q.x;
            acc.y -= cj * q.y;
        }
        y[i] = acc;
    }
}

// y = a * x + b * y over complex arrays (a from *a_dev / a_div when a_dev is set)
template <typename T>
__global__ void k_spec_axpby(cplx<T>* y, const cplx<T>* x, double a, double b, const double* a_dev, int a_recip,
                             long long len) {
    double av = a;
    if (a_dev) av = a_recip ? 1.0 / *a_dev : *a_dev;
    const T aa = (T)av, bb = (T)b;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        cplx<T> xv = x[i];
        cplx<T> yv = b == 0.0 ? mk<T>((T)0, (T)0) : y[i];
        y[i] = mk<T>(aa * xv.x + bb * yv.x, aa * xv.y + bb * yv.y);
    }
}

// y_spec = m^{-1/2} * x_spec  (elementwise, m = Lambda + sigma)
template <typename T>
__global__ void k_spec_msc(cplx<T>* y, const cplx<T>* x, SpecGeom g, T xi2, T sigma) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.len; i += (long long)gridDim.x * blockDim.x) {
        const T f = (T)1 / sqrt(spec_lambda<T>(g, i, xi2) + sigma);
        const cplx<T> v = x[i];
        y[i] = mk<T>(f * v.x, f * v.y);
    }
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based generator --------
struct u32x4 { unsigned x, y, z, w; };

__host__ __device__ __forceinline__ unsigned mulhi32(unsigned a, unsigned b) {
    return (unsigned)(((unsigned long long)a * (unsigned long long)b) >> 32);
}

__host__ __device__ inline u32x4 philox4x32_10(u32x4 c, unsigned k0, unsigned k1) {
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = mulhi32(M0, c.x), lo0 = M0 * c.x;
        const unsigned hi1 = mulhi32(M1, c.z), lo1 = M1 * c.z;
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// standard normal samples: element i uses counter (i/2, 0, stream, 0) and Box-Muller
template <typename T>
__global__ void k_philox_normal(T* out, long long n, unsigned long long seed, unsigned stream) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n + 1) / 2;
         i += (long long)gridDim.x * blockDim.x) {
        u32x4 r = philox4x32_10(u32x4{(unsigned)i, (unsigned)(i >> 32), stream, 0u}, (unsigned)seed,
                                (unsigned)(seed >> 32));
        const double u1 = ((double)r.x + 0.5) * (1.0 / 4294967296.0);
        const double u2 = ((double)r.y + 0.5) * (1.0 / 4294967296.0);
        const double rad = sqrt(-2.0 * log(u1));
        const double th = 6.283185307179586476925286766559 * u2;
        out[2 * i] = (T)(rad * cos(th));
        if (2 * i + 1 < n) out[2 * i + 1] = (T)(rad * sin(th));
    }
}

}  // namespace lbtr
