// x-row passes (2D grids, and 3D grids not handled by the plane kernels) as register-resident
// four-step transforms.
//
// A CTA owns NR consecutive rows.  A real row of M samples is transformed as H = M/2 complex
// pairs z[n] = x[2n] + i x[2n+1] (the half-length real method of fft_core.cuh): L2 threads
// per row, thread j holding z[j + L2 m] (m < L1), a DFT of length L1 in registers, the
// twiddle W_H^{ja}, one padded transpose through shared memory and a DFT of length L2.  The
// row spectrum then goes to a padded row buffer, from which the real-spectrum fold reads
// mirror pairs X[k], X[H - k] and stores X[0..H-1] to the main spectrum and X[H] to the
// Nyquist column, coalesced.  The inverse runs the same steps backwards; the pointwise work
// of each mode (F''(phi) v, F'(phi), sum F, the IMEX b) is fused as in the plane kernels.
#pragma once
#include "passes.cuh"
#include "planes.cuh"

namespace lbtr {

template <int M> struct RowGeo {
    static constexpr int H = M / 2;
    static constexpr int L1 = fs_l1(H), L2 = fs_l2(H), RR = L1 / L2;
    static constexpr int NR = 128 / L2;                 // rows per CTA
    static constexpr int NT = NR * L2;                  // 128 threads
    static constexpr int PX = L2 + 1;
    static constexpr int RSX = ((L1 * PX / L2) % 2) ? L1 * PX : L1 * PX + L2;
    static constexpr int RS2 = H + L2;
};

__host__ __device__ constexpr int rows_nt(int) { return 128; }
template <typename T> __host__ __device__ constexpr size_t rows_smem_t(int nr, int rsx, int rs2) {
    return ((size_t)nr * rsx + (size_t)nr * rs2) * 2 * sizeof(T) + 128 * sizeof(double);
}
template <typename T, int M> __host__ __device__ constexpr size_t rows_smem() {
    return rows_smem_t<T>(RowGeo<M>::NR, RowGeo<M>::RSX, RowGeo<M>::RS2);
}

template <typename T, int M> struct RowSmem {
    cplx<T>* S;     // transpose, NR x RSX
    cplx<T>* B;     // row spectra, NR x RS2 (slot H of a row holds X[H] on the inverse)
    double* red;
    __device__ __forceinline__ RowSmem(unsigned char* raw) {
        using G = RowGeo<M>;
        S = reinterpret_cast<cplx<T>*>(raw);
        B = S + G::NR * G::RSX;
        red = reinterpret_cast<double*>(B + G::NR * G::RS2);
    }
};

// forward: u[m] = z[j + L2 m] of local row y -> unfolded row spectrum in B[y][k]
template <typename T, int M>
__device__ __forceinline__ void rows_fwd(cplx<T> (&u)[RowGeo<M>::L1], const RowSmem<T, M>& sm, const cplx<T>* __restrict__ tw) {
    using G = RowGeo<M>;
    constexpr int L1 = G::L1, L2 = G::L2, RR = G::RR;
    const int j = threadIdx.x % L2, y = threadIdx.x / L2;
    dft_r<-1, L1, T>(u);
#pragma unroll
    for (int a = 1; a < L1; ++a) u[a] = cmul(u[a], __ldg(&tw[2 * j * a]));      // W_H^{ja}
#pragma unroll
    for (int a = 0; a < L1; ++a) sm.S[y * G::RSX + a * G::PX + j] = u[a];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < RR; ++s) {
        const int a = j + L2 * s;
#pragma unroll
        for (int jj = 0; jj < L2; ++jj) u[s * L2 + jj] = sm.S[y * G::RSX + a * G::PX + jj];
        dft_r<-1, L2, T>(&u[s * L2]);
    }
#pragma unroll
    for (int s = 0; s < RR; ++s)
#pragma unroll
        for (int b = 0; b < L2; ++b) sm.B[y * G::RS2 + j + L2 * s + L1 * b] = u[s * L2 + b];
    __syncthreads();
}

// fold B[y][.] into the real spectrum X[0..H] of row row0 + y and store it
template <typename T, int M>
__device__ __forceinline__ void rows_fold_store(const RowSmem<T, M>& sm, cplx<T>* main, cplx<T>* nyq, long long row0,
                                                int rows, const cplx<T>* __restrict__ tw) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1, L2 = G::L2;
    const int j = threadIdx.x % L2, y = threadIdx.x / L2;
    const long long row = row0 + y;
    if (row >= rows) return;
    const T hf = (T)0.5;
#pragma unroll
    for (int t = 0; t < L1; ++t) {
        const int k = j + L2 * t;
        C out;
        if (k == 0) {
            const C z0 = sm.B[y * G::RS2];
            out = mk<T>(z0.x + z0.y, (T)0);
            nyq[row] = mk<T>(z0.x - z0.y, (T)0);
        } else {
            const C zk = sm.B[y * G::RS2 + k], zm = sm.B[y * G::RS2 + H - k];
            const C e = mk<T>(hf * (zk.x + zm.x), hf * (zk.y - zm.y));
            const C o = mk<T>(hf * (zk.y + zm.y), -hf * (zk.x - zm.x));
            out = cadd(e, cmul(__ldg(&tw[k]), o));
        }
        main[row * H + k] = out;
    }
}

// load the spectrum of row row0 + y into B[y][0..H] (slot H: the Nyquist entry)
template <typename T, int M>
__device__ __forceinline__ void rows_load_spec(const RowSmem<T, M>& sm, const cplx<T>* __restrict__ main,
                                               const cplx<T>* __restrict__ nyq, long long row0, int rows) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1, L2 = G::L2;
    const int j = threadIdx.x % L2, y = threadIdx.x / L2;
    const long long row = row0 + y;
    const bool ok = row < rows;
    const C zero = mk<T>((T)0, (T)0);
    C v[L1];
#pragma unroll
    for (int t = 0; t < L1; ++t) v[t] = ok ? main[row * H + j + L2 * t] : zero;
    const C vn = (ok && j == 0) ? nyq[row] : zero;
#pragma unroll
    for (int t = 0; t < L1; ++t) sm.B[y * G::RS2 + j + L2 * t] = v[t];
    if (j == 0) sm.B[y * G::RS2 + H] = vn;
    __syncthreads();
}

// inverse: B[y][0..H] -> u[d] = z[j + L2 d] (unscaled)
template <typename T, int M>
__device__ __forceinline__ void rows_inv(cplx<T> (&u)[RowGeo<M>::L1], const RowSmem<T, M>& sm, const cplx<T>* __restrict__ tw) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1, L2 = G::L2, RR = G::RR;
    const int j = threadIdx.x % L2, y = threadIdx.x / L2;
#pragma unroll
    for (int s = 0; s < RR; ++s) {
#pragma unroll
        for (int b = 0; b < L2; ++b) {
            const int k = j + L2 * s + L1 * b;
            C val;
            if (s == 0 && b == 0 && j == 0) {
                const T x0 = sm.B[y * G::RS2].x, xh = sm.B[y * G::RS2 + H].x;
                val = mk<T>(x0 + xh, x0 - xh);
            } else {
                const C xk = sm.B[y * G::RS2 + k], xm = sm.B[y * G::RS2 + H - k];
                const C e = mk<T>(xk.x + xm.x, xk.y - xm.y);
                const C d = mk<T>(xk.x - xm.x, xk.y + xm.y);
                const C o = cmul(d, cconj(__ldg(&tw[k])));
                val = mk<T>(e.x - o.y, e.y + o.x);
            }
            u[s * L2 + b] = val;
        }
        const int a = j + L2 * s;
        dft_r<+1, L2, T>(&u[s * L2]);
#pragma unroll
        for (int c = 1; c < L2; ++c) u[s * L2 + c] = cmul(u[s * L2 + c], cconj(__ldg(&tw[2 * c * a])));
    }
#pragma unroll
    for (int s = 0; s < RR; ++s)
#pragma unroll
        for (int c = 0; c < L2; ++c) sm.S[y * G::RSX + (j + L2 * s) * G::PX + c] = u[s * L2 + c];
    __syncthreads();
#pragma unroll
    for (int a = 0; a < L1; ++a) u[a] = sm.S[y * G::RSX + a * G::PX + j];
    dft_r<+1, L1, T>(u);
}

template <int M> __device__ __forceinline__ long long rows_idx(long long row0, int m) {
    using G = RowGeo<M>;
    const int j = threadIdx.x % G::L2, y = threadIdx.x / G::L2;
    return (row0 + y) * G::H + j + G::L2 * m;
}

template <typename T, int M, int MODE>
__device__ __forceinline__ void rows_fwd_body(const XfArgs<T>& a) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int L1 = G::L1;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RowSmem<T, M> sm(smem_raw);
    const long long row0 = (long long)blockIdx.x * G::NR;
    const bool ok = row0 + threadIdx.x / G::L2 < a.rows;
    const C zero = mk<T>((T)0, (T)0);
    C u[L1];
    constexpr int NQ = (MODE == XF_ENERGY) ? 4 : 1;
    Acc<T> acc[NQ];
    if (MODE == XF_IMEX0) {
        C p[L1], gg[L1];
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const long long idx = rows_idx<M>(row0, m);
            p[m] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
            gg[m] = ok ? reinterpret_cast<const C*>(a.g)[idx] : zero;
            u[m] = (ok && a.d0) ? reinterpret_cast<const C*>(a.d0)[idx] : zero;
        }
        const T ds = a.d0 ? (T)0 : (T)(*a.dscale);
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const C d = a.d0 ? u[m] : mk<T>(ds * gg[m].x, ds * gg[m].y);
            u[m].x = d.x - a.model.eta * (gg[m].x + f2v(a.model, p[m].x) * d.x);
            u[m].y = d.y - a.model.eta * (gg[m].y + f2v(a.model, p[m].y) * d.y);
        }
    } else {
        C p[L1];
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const long long idx = rows_idx<M>(row0, m);
            u[m] = ok ? reinterpret_cast<const C*>(a.in)[idx] : zero;
            if (MODE == XF_HVPMEAN) p[m] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        }
        if (ok) {
#pragma unroll
            for (int m = 0; m < L1; ++m) {
                const C v = u[m];
                if (MODE == XF_HVPMEAN) {
                    acc[0].add(f2v(a.model, p[m].x) * v.x + f2v(a.model, p[m].y) * v.y);
                } else if (MODE == XF_ENERGY) {
                    acc[0].add(f0v(a.model, v.x));
                    acc[0].add(f0v(a.model, v.y));
                    acc[NQ > 1 ? 1 : 0].add(f1v(a.model, v.x));
                    acc[NQ > 1 ? 1 : 0].add(f1v(a.model, v.y));
                    acc[NQ > 2 ? 2 : 0].add(v.x + v.y);
                    acc[NQ > 3 ? 3 : 0].add(v.x * v.x + v.y * v.y);
                }
            }
        }
    }
    rows_fwd<T, M>(u, sm, a.tw);
    rows_fold_store<T, M>(sm, a.main, a.nyq, row0, a.rows, a.tw);
    if (MODE == XF_HVPMEAN || MODE == XF_ENERGY) {
        double tot[NQ];
        block_sum<T, NQ>(acc, sm.red, tot);
        finalize_partials(a.red, tot);
    }
}

template <typename T, int M, int MODE>
__device__ __forceinline__ void rows_inv_body(const XiArgs<T>& a) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int L1 = G::L1;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RowSmem<T, M> sm(smem_raw);
    const long long row0 = (long long)blockIdx.x * G::NR;
    const bool ok = row0 + threadIdx.x / G::L2 < a.rows;
    const C zero = mk<T>((T)0, (T)0);
    C p[L1], vv[L1];
    if (MODE != XI_PLAIN) {
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const long long idx = rows_idx<M>(row0, m);
            p[m] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
            if (MODE == XI_HVP) vv[m] = ok ? reinterpret_cast<const C*>(a.v)[idx] : zero;
        }
    }
    rows_load_spec<T, M>(sm, a.main, a.nyq, row0, a.rows);
    C u[L1];
    rows_inv<T, M>(u, sm, a.tw);
    T mean = (T)0;
    if (MODE != XI_PLAIN) mean = (T)(*a.msum * a.inv_n);
    double mx = 0.0;
    if (ok) {
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const C zz = u[m];
            C o;
            if (MODE == XI_PLAIN) {
                o = mk<T>(zz.x * a.oscale, zz.y * a.oscale);
            } else if (MODE == XI_HVP) {
                o.x = zz.x + f2v(a.model, p[m].x) * vv[m].x - mean;
                o.y = zz.y + f2v(a.model, p[m].y) * vv[m].y - mean;
            } else {
                o.x = zz.x + f1v(a.model, p[m].x) - mean;
                o.y = zz.y + f1v(a.model, p[m].y) - mean;
                mx = fmax(mx, fmax(fabs((double)o.x), fabs((double)o.y)));
            }
            reinterpret_cast<C*>(a.out)[rows_idx<M>(row0, m)] = o;
        }
    }
    if (MODE == XI_GRAD) {
        double mm = block_max(mx, sm.red);
        finalize_partials(a.red, &mm);
    }
}

// one problem per launch
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(128) k_rows_fwd(XfArgs<T> a) { rows_fwd_body<T, M, MODE>(a); }
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(128) k_rows_inv(XiArgs<T> a) { rows_inv_body<T, M, MODE>(a); }
// many problems of the same size per launch: blockIdx.y selects the problem's arguments
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(128) k_rows_fwd_b(const XfArgs<T>* __restrict__ args) {
    rows_fwd_body<T, M, MODE>(args[blockIdx.y]);
}
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(128) k_rows_inv_b(const XiArgs<T>* __restrict__ args) {
    rows_inv_body<T, M, MODE>(args[blockIdx.y]);
}

template <typename T, int M, int MODE>
__global__ void __launch_bounds__(128) k_rows_mid(XmArgs<T> a) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int L1 = G::L1;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RowSmem<T, M> sm(smem_raw);
    const long long row0 = (long long)blockIdx.x * G::NR;
    const bool ok = row0 + threadIdx.x / G::L2 < a.rows;
    const C zero = mk<T>((T)0, (T)0);
    C p[L1], gg[L1];
#pragma unroll
    for (int m = 0; m < L1; ++m) {
        const long long idx = rows_idx<M>(row0, m);
        p[m] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        if (MODE == XM_IMEX) gg[m] = ok ? reinterpret_cast<const C*>(a.g)[idx] : zero;
    }
    rows_load_spec<T, M>(sm, a.main, a.nyq, row0, a.rows);
    C u[L1];
    rows_inv<T, M>(u, sm, a.tw);
#pragma unroll
    for (int m = 0; m < L1; ++m) {
        const T dx = u[m].x * a.scale, dy = u[m].y * a.scale;
        if (MODE == XM_IMEX) {
            u[m].x = dx - a.model.eta * (gg[m].x + f2v(a.model, p[m].x) * dx);
            u[m].y = dy - a.model.eta * (gg[m].y + f2v(a.model, p[m].y) * dy);
        } else {
            u[m].x = f2v(a.model, p[m].x) * dx;
            u[m].y = f2v(a.model, p[m].y) * dy;
        }
    }
    __syncthreads();    // the inverse's last reads of S precede the forward's first writes
    rows_fwd<T, M>(u, sm, a.tw);
    rows_fold_store<T, M>(sm, a.main, a.nyq, row0, a.rows, a.tw);
}

}  // namespace lbtr
