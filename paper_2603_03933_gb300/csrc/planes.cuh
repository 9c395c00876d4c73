// Plane kernels for 3D grids: one CTA transforms a whole z-plane along x and y.
//
// The plane sits in shared memory as P[y][kx'] (kx' = 0..M/2, row stride LD = M/2+1,
// odd, so row-parallel and column-parallel accesses are both free of bank conflicts).
// Forward: real rows -> half-length complex FFT along x -> real-spectrum fold (the
// Nyquist entry kx = M/2 lands in column M/2) -> FFT along y of the M/2+1 columns.
// The result is stored in the spectrum layout of passes.cuh (main[rows][M/2], nyq[rows]).
// Replacing the separate x and y passes saves one read and one write of the spectrum
// per direction and one launch.
#pragma once
#include "passes.cuh"

namespace lbtr {

__host__ __device__ constexpr int plane_nt(int m) { return (m / 2) * m / 8 > 1024 ? 1024 : (m / 2) * m / 8; }
__host__ __device__ constexpr int plane_ld(int m) { return m / 2 + 1; }
template <typename T> __host__ __device__ constexpr size_t plane_smem(int m) {
    return sizeof(cplx<T>) * ((size_t)m + (size_t)m * plane_ld(m)) + 128 * sizeof(double);
}

// forward x then y on the plane in shared memory
template <typename T, int M, int NT>
__device__ __forceinline__ void plane_fwd_xy(cplx<T>* P, const cplx<T>* tw) {
    constexpr int H = M / 2, LD = plane_ld(M);
    fft_lines_s<T, -1, H, M, NT, 1, LD>(P, tw, M);
    r2c_post_s<T, H, M, NT, 1, LD>(P, tw, M);
    fft_lines_s<T, -1, M, H, NT, LD, 1>(P, tw, M);        // columns kx' = 0..H-1
    fft_lines_s<T, -1, M, 1, NT, LD, 1>(P + H, tw, M);    // the Nyquist column kx' = H
}

// inverse y then x on the plane in shared memory
template <typename T, int M, int NT>
__device__ __forceinline__ void plane_inv_xy(cplx<T>* P, const cplx<T>* tw) {
    constexpr int H = M / 2, LD = plane_ld(M);
    fft_lines_s<T, +1, M, H, NT, LD, 1>(P, tw, M);
    fft_lines_s<T, +1, M, 1, NT, LD, 1>(P + H, tw, M);
    c2r_pre_s<T, H, M, NT, 1, LD>(P, tw, M);
    fft_lines_s<T, +1, H, M, NT, 1, LD>(P, tw, M);
}

// load a spectrum plane (main rows and the nyq column) into P
template <typename T, int M, int NT>
__device__ __forceinline__ void plane_load_spec(cplx<T>* P, const cplx<T>* main, const cplx<T>* nyq, int z) {
    constexpr int H = M / 2, LD = plane_ld(M), IT = (M * H + NT - 1) / NT;
    cplx<T> v[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        if (w < M * H) v[t] = main[((size_t)z * M + w / H) * H + (w % H)];
    }
    for (int y = threadIdx.x; y < M; y += NT) P[y * LD + H] = nyq[(size_t)z * M + y];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        if (w < M * H) P[(w / H) * LD + (w % H)] = v[t];
    }
}

template <typename T, int M, int NT>
__device__ __forceinline__ void plane_store_spec(const cplx<T>* P, cplx<T>* main, cplx<T>* nyq, int z) {
    constexpr int H = M / 2, LD = plane_ld(M), IT = (M * H + NT - 1) / NT;
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        if (w < M * H) main[((size_t)z * M + w / H) * H + (w % H)] = P[(w / H) * LD + (w % H)];
    }
    for (int y = threadIdx.x; y < M; y += NT) nyq[(size_t)z * M + y] = P[y * LD + H];
}

// ---- forward: real plane -> spectrum plane (modes of k_xfwd) --------------------
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(plane_nt(M)) k_plane_fwd(XfArgs<T> a) {
    constexpr int H = M / 2, NT = plane_nt(M), LD = plane_ld(M);
    constexpr int IT = (M * H + NT - 1) / NT;
    using C = cplx<T>;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* P = tw + M;
    double* red = reinterpret_cast<double*>(P + M * LD);
    const int z = blockIdx.x;
    const C zero = mk<T>((T)0, (T)0);
    C zz[IT], p[IT], gg[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const bool ok = w < M * H;
        const size_t idx = ((size_t)z * M + w / H) * H + (w % H);
        if (MODE == XF_IMEX0) {
            p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
            gg[t] = ok ? reinterpret_cast<const C*>(a.g)[idx] : zero;
            zz[t] = (ok && a.d0) ? reinterpret_cast<const C*>(a.d0)[idx] : zero;
        } else {
            zz[t] = ok ? reinterpret_cast<const C*>(a.in)[idx] : zero;
            if (MODE == XF_HVPMEAN) p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        }
    }
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];
    constexpr int NQ = (MODE == XF_ENERGY) ? 4 : 1;
    Acc<T> acc[NQ];
    T ds = (T)0;
    if (MODE == XF_IMEX0 && a.d0 == nullptr) ds = (T)(*a.dscale);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        if (w >= M * H) continue;
        C v = zz[t];
        if (MODE == XF_IMEX0) {
            C d = a.d0 ? v : mk<T>(ds * gg[t].x, ds * gg[t].y);
            v.x = d.x - a.model.eta * (gg[t].x + f2v(a.model, p[t].x) * d.x);
            v.y = d.y - a.model.eta * (gg[t].y + f2v(a.model, p[t].y) * d.y);
        } else if (MODE == XF_HVPMEAN) {
            acc[0].add(f2v(a.model, p[t].x) * v.x + f2v(a.model, p[t].y) * v.y);
        } else if (MODE == XF_ENERGY) {
            acc[0].add(f0v(a.model, v.x));
            acc[0].add(f0v(a.model, v.y));
            acc[NQ > 1 ? 1 : 0].add(f1v(a.model, v.x));
            acc[NQ > 1 ? 1 : 0].add(f1v(a.model, v.y));
            acc[NQ > 2 ? 2 : 0].add(v.x + v.y);
            acc[NQ > 3 ? 3 : 0].add(v.x * v.x + v.y * v.y);
        }
        P[(w / H) * LD + (w % H)] = v;
    }
    __syncthreads();
    plane_fwd_xy<T, M, NT>(P, tw);
    plane_store_spec<T, M, NT>(P, a.main, a.nyq, z);
    if (MODE == XF_HVPMEAN || MODE == XF_ENERGY) {
        double tot[NQ];
        block_sum<T, NQ>(acc, red, tot);
        finalize_partials(a.red, tot);
    }
}

// ---- inverse: spectrum plane -> real plane (modes of k_xinv) --------------------
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(plane_nt(M)) k_plane_inv(XiArgs<T> a) {
    constexpr int H = M / 2, NT = plane_nt(M), LD = plane_ld(M);
    constexpr int IT = (M * H + NT - 1) / NT;
    using C = cplx<T>;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* P = tw + M;
    double* red = reinterpret_cast<double*>(P + M * LD);
    const int z = blockIdx.x;
    const C zero = mk<T>((T)0, (T)0);
    C p[IT], vv[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const bool ok = w < M * H;
        const size_t idx = ((size_t)z * M + w / H) * H + (w % H);
        if (MODE != XI_PLAIN) p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        if (MODE == XI_HVP) vv[t] = ok ? reinterpret_cast<const C*>(a.v)[idx] : zero;
    }
    plane_load_spec<T, M, NT>(P, a.main, a.nyq, z);
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];
    T mean = (T)0;
    if (MODE != XI_PLAIN) mean = (T)(*a.msum * a.inv_n);
    __syncthreads();
    plane_inv_xy<T, M, NT>(P, tw);
    double mx = 0.0;
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        if (w >= M * H) continue;
        const size_t idx = ((size_t)z * M + w / H) * H + (w % H);
        C zz = P[(w / H) * LD + (w % H)];
        C o;
        if (MODE == XI_PLAIN) {
            o = mk<T>(zz.x * a.oscale, zz.y * a.oscale);
        } else if (MODE == XI_HVP) {
            o.x = zz.x + f2v(a.model, p[t].x) * vv[t].x - mean;
            o.y = zz.y + f2v(a.model, p[t].y) * vv[t].y - mean;
        } else {
            o.x = zz.x + f1v(a.model, p[t].x) - mean;
            o.y = zz.y + f1v(a.model, p[t].y) - mean;
            mx = fmax(mx, fmax(fabs((double)o.x), fabs((double)o.y)));
        }
        reinterpret_cast<C*>(a.out)[idx] = o;
    }
    if (MODE == XI_GRAD) {
        double m = block_max(mx, red);
        finalize_partials(a.red, &m);
    }
}

// ---- inverse -> pointwise -> forward on a plane (modes of k_xmid) ----------------
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(plane_nt(M)) k_plane_mid(XmArgs<T> a) {
    constexpr int H = M / 2, NT = plane_nt(M), LD = plane_ld(M);
    constexpr int IT = (M * H + NT - 1) / NT;
    using C = cplx<T>;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* P = tw + M;
    const int z = blockIdx.x;
    const C zero = mk<T>((T)0, (T)0);
    C p[IT], gg[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const bool ok = w < M * H;
        const size_t idx = ((size_t)z * M + w / H) * H + (w % H);
        p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        if (MODE == XM_IMEX) gg[t] = ok ? reinterpret_cast<const C*>(a.g)[idx] : zero;
    }
    plane_load_spec<T, M, NT>(P, a.main, a.nyq, z);
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];
    __syncthreads();
    plane_inv_xy<T, M, NT>(P, tw);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        if (w >= M * H) continue;
        const int e = (w / H) * LD + (w % H);
        C zz = P[e];
        T dx = zz.x * a.scale, dy = zz.y * a.scale;
        C o;
        if (MODE == XM_IMEX) {
            o.x = dx - a.model.eta * (gg[t].x + f2v(a.model, p[t].x) * dx);
            o.y = dy - a.model.eta * (gg[t].y + f2v(a.model, p[t].y) * dy);
        } else {
            o.x = f2v(a.model, p[t].x) * dx;
            o.y = f2v(a.model, p[t].y) * dy;
        }
        P[e] = o;
    }
    __syncthreads();
    plane_fwd_xy<T, M, NT>(P, tw);
    plane_store_spec<T, M, NT>(P, a.main, a.nyq, z);
}

}  // namespace lbtr
