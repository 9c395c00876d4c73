// Plane kernels for 3D grids of 32^3..128^3: one CTA transforms a whole z-plane along x and y.
//
// Each line transform is a register-resident four-step factorisation.  A line of length
// L = L1 * L2 is held by L2 threads, thread j owning the L1 samples x[j + L2 m]:
//   forward:  DFT_L1 over m in registers, twiddle W_L^{j a}, one transpose through shared
//             memory, DFT_L2 over j in registers; thread j' ends with X[a + L1 b] for
//             a = j' + L2 s (s < L1 / L2), b < L2;
//   inverse:  the mirror image (DFT_L2 over b, twiddle W_L^{-c a}, transpose, DFT_L1 over a),
//             from that layout back to the first one.
// The x transform is the half-length real method of fft_core.cuh (H = M/2 complex samples
// z[n] = x[2n] + i x[2n+1] per row); its real-spectrum fold is done while the y transform
// reads its input, each thread reading the two mirror columns kx and H - kx it needs.
// The two real columns kx = 0 and kx = M/2 (Nyquist) travel through the y transform
// packed as one complex column X(0, y) + i X(M/2, y); the forward unpacks them with
// X(0, k) = (Z_k + conj Z_-k) / 2, X(M/2, k) = (Z_k - conj Z_-k) / 2i, the inverse packs the
// Hermitian parts of both columns, so that each inverse column transform is real as the
// real-to-complex inverse assumes.
// Per plane and direction this is three transposes through shared memory and three or
// four barriers; spectra are stored in the layout of passes.cuh (main[rows][M/2], nyq[rows]).
#pragma once
#include "passes.cuh"

namespace lbtr {

// four-step factors of a line of length L: L1 registers, L2 threads
__host__ __device__ constexpr int fs_l1(int L) { return L <= 16 ? 4 : L <= 64 ? 8 : 16; }
__host__ __device__ constexpr int fs_l2(int L) { return L / fs_l1(L); }

template <int M> struct PlaneGeo {
    static constexpr int H = M / 2;
    static constexpr int L1x = fs_l1(H), L2x = fs_l2(H), L1y = fs_l1(M), L2y = fs_l2(M);
    static constexpr int NT = H * L2y;                 // threads: one per (column, y-thread)
    static constexpr int RX = M * L2x / NT;            // rows per thread in the x transform
    static constexpr int PX = L2x + 1;                 // x transpose: slot a * PX + j within a row
    // row stride of the x transpose: a multiple of L2x, odd in units of L2x, so that the
    // rows of a half-warp fall on disjoint banks
    static constexpr int RSX = ((L1x * PX / L2x) % 2) ? L1x * PX : L1x * PX + L2x;
    static constexpr int RS2 = H + L2x;                // row stride of the x <-> y hand-off
    static constexpr int TS = M + 1;                   // column stride of the y transpose
    static constexpr int SA = (M * RSX > H * TS) ? M * RSX : H * TS;
    static constexpr int SB = M * RS2;
};

__host__ __device__ constexpr int plane_nt(int m) { return (m / 2) * fs_l2(m); }

// Two buffers (transpose and hand-off) when they fit, else one buffer and extra barriers.
template <typename T, int M> __host__ __device__ constexpr bool plane_onebuf() {
    using G = PlaneGeo<M>;
    return (size_t)(G::SA + G::SB + M) * 2 * sizeof(T) + 256 * sizeof(double) > 200 * 1024;
}
template <typename T, int M> __host__ __device__ constexpr size_t plane_smem_t() {
    using G = PlaneGeo<M>;
    const size_t nb = plane_onebuf<T, M>() ? (G::SA > G::SB ? G::SA : G::SB) : (size_t)(G::SA + G::SB);
    return (nb + M) * 2 * sizeof(T) + 256 * sizeof(double);
}
template <typename T> __host__ __device__ constexpr size_t plane_smem(int m) {
    return m == 32 ? plane_smem_t<T, 32>() : m == 64 ? plane_smem_t<T, 64>() : plane_smem_t<T, 128>();
}

template <typename T, int M> struct PlaneSmem {
    cplx<T>* A;    // x or y transpose
    cplx<T>* B;    // hand-off between the x and y transforms (aliases A in one-buffer mode)
    cplx<T>* Z0;   // the packed kx = 0 column of the forward output
    double* red;
    __device__ __forceinline__ PlaneSmem(unsigned char* raw) {
        using G = PlaneGeo<M>;
        A = reinterpret_cast<cplx<T>*>(raw);
        B = plane_onebuf<T, M>() ? A : A + G::SA;
        const int nb = plane_onebuf<T, M>() ? (G::SA > G::SB ? G::SA : G::SB) : G::SA + G::SB;
        Z0 = A + nb;
        red = reinterpret_cast<double*>(Z0 + M);
    }
};

// ---- forward x: rows in registers (thread j: z[j + L2x m]) -> hand-off buffer B[y][kx] ----
template <typename T, int M>
__device__ __forceinline__ void p4_fwd_x(cplx<T> (&u)[PlaneGeo<M>::RX][PlaneGeo<M>::L1x], const PlaneSmem<T, M>& sm,
                                         const cplx<T>* __restrict__ tw) {
    using G = PlaneGeo<M>;
    constexpr int L1 = G::L1x, L2 = G::L2x, RR = L1 / L2;
    const int j = threadIdx.x % L2, y0 = threadIdx.x / L2;
#pragma unroll
    for (int r = 0; r < G::RX; ++r) {
        const int y = y0 + r * (G::NT / L2);
        dft_r<-1, L1, T>(u[r]);
#pragma unroll
        for (int a = 1; a < L1; ++a) u[r][a] = cmul(u[r][a], __ldg(&tw[2 * j * a]));   // W_H^{ja}
#pragma unroll
        for (int a = 0; a < L1; ++a) sm.A[y * G::RSX + a * G::PX + j] = u[r][a];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < G::RX; ++r) {
        const int y = y0 + r * (G::NT / L2);
#pragma unroll
        for (int s = 0; s < RR; ++s) {
            const int a = j + L2 * s;
#pragma unroll
            for (int jj = 0; jj < L2; ++jj) u[r][s * L2 + jj] = sm.A[y * G::RSX + a * G::PX + jj];
            dft_r<-1, L2, T>(&u[r][s * L2]);
        }
    }
    if (plane_onebuf<T, M>()) __syncthreads();
#pragma unroll
    for (int r = 0; r < G::RX; ++r) {
        const int y = y0 + r * (G::NT / L2);
#pragma unroll
        for (int s = 0; s < RR; ++s)
#pragma unroll
            for (int b = 0; b < L2; ++b) sm.B[y * G::RS2 + j + L2 * s + L1 * b] = u[r][s * L2 + b];
    }
    __syncthreads();
}

// ---- forward y: B (with the real-spectrum fold) -> registers, thread (kx, i) holding
//      Y[ky = i + L2y s + L1y b][kx] at w[s L2y + b]; kx = 0 is the packed column ----
template <typename T, int M>
__device__ __forceinline__ void p4_fwd_y(cplx<T> (&w)[PlaneGeo<M>::L1y], const PlaneSmem<T, M>& sm,
                                         const cplx<T>* __restrict__ tw) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1y, L2 = G::L2y, RR = L1 / L2;
    const int kx = threadIdx.x % H, i = threadIdx.x / H;
    const C wk = __ldg(&tw[kx]);
    const T hf = (T)0.5;
#pragma unroll
    for (int m = 0; m < L1; ++m) {
        const int y = i + L2 * m;
        if (kx == 0) {
            const C z0 = sm.B[y * G::RS2];
            w[m] = mk<T>(z0.x + z0.y, z0.x - z0.y);      // X(0) + i X(H), both real
        } else {
            const C zk = sm.B[y * G::RS2 + kx], zm = sm.B[y * G::RS2 + H - kx];
            const C e = mk<T>(hf * (zk.x + zm.x), hf * (zk.y - zm.y));
            const C o = mk<T>(hf * (zk.y + zm.y), -hf * (zk.x - zm.x));
            w[m] = cadd(e, cmul(wk, o));
        }
    }
    dft_r<-1, L1, T>(w);
#pragma unroll
    for (int a = 1; a < L1; ++a) w[a] = cmul(w[a], __ldg(&tw[i * a]));       // W_M^{ia}
    if (plane_onebuf<T, M>()) __syncthreads();
#pragma unroll
    for (int a = 0; a < L1; ++a) sm.A[kx * G::TS + a * L2 + i] = w[a];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < RR; ++s) {
        const int a = i + L2 * s;
#pragma unroll
        for (int jj = 0; jj < L2; ++jj) w[s * L2 + jj] = sm.A[kx * G::TS + a * L2 + jj];
        dft_r<-1, L2, T>(&w[s * L2]);
    }
}

// store the forward output of plane z; the packed column is unpacked through Z0
template <typename T, int M>
__device__ __forceinline__ void p4_store_spec(const cplx<T> (&w)[PlaneGeo<M>::L1y], const PlaneSmem<T, M>& sm,
                                              cplx<T>* main, cplx<T>* nyq, int z) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1y, L2 = G::L2y, RR = L1 / L2;
    const int kx = threadIdx.x % H, i = threadIdx.x / H;
    const size_t row0 = (size_t)z * M;
#pragma unroll
    for (int s = 0; s < RR; ++s)
#pragma unroll
        for (int b = 0; b < L2; ++b) {
            const int ky = i + L2 * s + L1 * b;
            if (kx) main[(row0 + ky) * H + kx] = w[s * L2 + b];
            else sm.Z0[ky] = w[s * L2 + b];
        }
    __syncthreads();
    const T hf = (T)0.5;
    for (int ky = threadIdx.x; ky < M; ky += G::NT) {
        const C zk = sm.Z0[ky], zm = sm.Z0[(M - ky) & (M - 1)];
        main[(row0 + ky) * H] = mk<T>(hf * (zk.x + zm.x), hf * (zk.y - zm.y));
        nyq[row0 + ky] = mk<T>(hf * (zk.y + zm.y), -hf * (zk.x - zm.x));
    }
}

// load plane z of a spectrum into the forward-output layout; kx = 0 packs the Hermitian
// parts of the kx = 0 and Nyquist columns
template <typename T, int M>
__device__ __forceinline__ void p4_load_spec(cplx<T> (&w)[PlaneGeo<M>::L1y], const cplx<T>* __restrict__ main,
                                             const cplx<T>* __restrict__ nyq, int z) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1y, L2 = G::L2y, RR = L1 / L2;
    const int kx = threadIdx.x % H, i = threadIdx.x / H;
    const size_t row0 = (size_t)z * M;
    const T hf = (T)0.5;
#pragma unroll
    for (int s = 0; s < RR; ++s)
#pragma unroll
        for (int b = 0; b < L2; ++b) {
            const int ky = i + L2 * s + L1 * b;
            if (kx) {
                w[s * L2 + b] = main[(row0 + ky) * H + kx];
            } else {
                const int km = (M - ky) & (M - 1);
                const C x0 = main[(row0 + ky) * H], x0m = main[(row0 + km) * H];
                const C xh = nyq[row0 + ky], xhm = nyq[row0 + km];
                const C e = mk<T>(hf * (x0.x + x0m.x), hf * (x0.y - x0m.y));
                const C f = mk<T>(hf * (xh.x + xhm.x), hf * (xh.y - xhm.y));
                w[s * L2 + b] = mk<T>(e.x - f.y, e.y + f.x);
            }
        }
}

// ---- inverse y: registers in the forward-output layout -> B[y][kx] (time domain in y) ----
template <typename T, int M>
__device__ __forceinline__ void p4_inv_y(cplx<T> (&w)[PlaneGeo<M>::L1y], const PlaneSmem<T, M>& sm,
                                         const cplx<T>* __restrict__ tw) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1y, L2 = G::L2y, RR = L1 / L2;
    const int kx = threadIdx.x % H, i = threadIdx.x / H;
#pragma unroll
    for (int s = 0; s < RR; ++s) {
        const int a = i + L2 * s;
        dft_r<+1, L2, T>(&w[s * L2]);
#pragma unroll
        for (int c = 1; c < L2; ++c) w[s * L2 + c] = cmul(w[s * L2 + c], cconj(__ldg(&tw[c * a])));   // W_M^{-ca}
#pragma unroll
        for (int c = 0; c < L2; ++c) sm.A[kx * G::TS + a * L2 + c] = w[s * L2 + c];
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < L1; ++a) w[a] = sm.A[kx * G::TS + a * L2 + i];
    dft_r<+1, L1, T>(w);
    if (plane_onebuf<T, M>()) __syncthreads();
#pragma unroll
    for (int d = 0; d < L1; ++d) sm.B[(i + L2 * d) * G::RS2 + kx] = w[d];
    __syncthreads();
}

// ---- inverse x: B (with the complex-to-real pre-step) -> rows in registers,
//      thread j holding z[j + L2x d] (unscaled) ----
template <typename T, int M>
__device__ __forceinline__ void p4_inv_x(cplx<T> (&u)[PlaneGeo<M>::RX][PlaneGeo<M>::L1x], const PlaneSmem<T, M>& sm,
                                         const cplx<T>* __restrict__ tw) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int H = G::H, L1 = G::L1x, L2 = G::L2x, RR = L1 / L2;
    const int j = threadIdx.x % L2, y0 = threadIdx.x / L2;
#pragma unroll
    for (int r = 0; r < G::RX; ++r) {
        const int y = y0 + r * (G::NT / L2);
#pragma unroll
        for (int s = 0; s < RR; ++s) {
#pragma unroll
            for (int b = 0; b < L2; ++b) {
                const int kx = j + L2 * s + L1 * b;
                C val;
                if (s == 0 && b == 0 && j == 0) {
                    const C wv = sm.B[y * G::RS2];                // x0 + i xh, both real
                    val = mk<T>(wv.x + wv.y, wv.x - wv.y);
                } else {
                    const C xk = sm.B[y * G::RS2 + kx], xm = sm.B[y * G::RS2 + H - kx];
                    const C e = mk<T>(xk.x + xm.x, xk.y - xm.y);
                    const C d = mk<T>(xk.x - xm.x, xk.y + xm.y);
                    const C o = cmul(d, cconj(__ldg(&tw[kx])));
                    val = mk<T>(e.x - o.y, e.y + o.x);
                }
                u[r][s * L2 + b] = val;
            }
            const int a = j + L2 * s;
            dft_r<+1, L2, T>(&u[r][s * L2]);
#pragma unroll
            for (int c = 1; c < L2; ++c) u[r][s * L2 + c] = cmul(u[r][s * L2 + c], cconj(__ldg(&tw[2 * c * a])));
        }
    }
    if (plane_onebuf<T, M>()) __syncthreads();
#pragma unroll
    for (int r = 0; r < G::RX; ++r) {
        const int y = y0 + r * (G::NT / L2);
#pragma unroll
        for (int s = 0; s < RR; ++s)
#pragma unroll
            for (int c = 0; c < L2; ++c) sm.A[y * G::RSX + (j + L2 * s) * G::PX + c] = u[r][s * L2 + c];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < G::RX; ++r) {
        const int y = y0 + r * (G::NT / L2);
#pragma unroll
        for (int a = 0; a < L1; ++a) u[r][a] = sm.A[y * G::RSX + a * G::PX + j];
        dft_r<+1, L1, T>(u[r]);
    }
}

// complex-pair index of sample (y, j + L2x m) of plane z
template <int M> __device__ __forceinline__ size_t p4_idx(int z, int r, int m) {
    using G = PlaneGeo<M>;
    const int j = threadIdx.x % G::L2x, y = threadIdx.x / G::L2x + r * (G::NT / G::L2x);
    return ((size_t)z * M + y) * G::H + j + G::L2x * m;
}

// ---- forward: real plane -> spectrum plane (modes of k_xfwd) --------------------
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(plane_nt(M)) k_plane_fwd(XfArgs<T> a) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int RX = G::RX, L1 = G::L1x;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PlaneSmem<T, M> sm(smem_raw);
    const int z = blockIdx.x;
    C u[RX][L1];
    constexpr int NQ = (MODE == XF_ENERGY) ? 4 : 1;
    Acc<T> acc[NQ];
    if (MODE == XF_IMEX0) {
        const T ds = a.d0 ? (T)0 : (T)(*a.dscale);
#pragma unroll
        for (int r = 0; r < RX; ++r) {
            C p[L1], gg[L1];
#pragma unroll
            for (int m = 0; m < L1; ++m) {
                const size_t idx = p4_idx<M>(z, r, m);
                p[m] = reinterpret_cast<const C*>(a.phi)[idx];
                gg[m] = reinterpret_cast<const C*>(a.g)[idx];
                if (a.d0) u[r][m] = reinterpret_cast<const C*>(a.d0)[idx];
            }
#pragma unroll
            for (int m = 0; m < L1; ++m) {
                const C d = a.d0 ? u[r][m] : mk<T>(ds * gg[m].x, ds * gg[m].y);
                u[r][m].x = d.x - a.model.eta * (gg[m].x + f2v(a.model, p[m].x) * d.x);
                u[r][m].y = d.y - a.model.eta * (gg[m].y + f2v(a.model, p[m].y) * d.y);
            }
        }
    } else {
        C p[RX][L1];
#pragma unroll
        for (int r = 0; r < RX; ++r)
#pragma unroll
            for (int m = 0; m < L1; ++m) {
                const size_t idx = p4_idx<M>(z, r, m);
                u[r][m] = reinterpret_cast<const C*>(a.in)[idx];
                if (MODE == XF_HVPMEAN) p[r][m] = reinterpret_cast<const C*>(a.phi)[idx];
            }
#pragma unroll
        for (int r = 0; r < RX; ++r)
#pragma unroll
            for (int m = 0; m < L1; ++m) {
                const C v = u[r][m];
                if (MODE == XF_HVPMEAN) {
                    acc[0].add(f2v(a.model, p[r][m].x) * v.x + f2v(a.model, p[r][m].y) * v.y);
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
    p4_fwd_x<T, M>(u, sm, a.tw);
    C w[G::L1y];
    p4_fwd_y<T, M>(w, sm, a.tw);
    p4_store_spec<T, M>(w, sm, a.main, a.nyq, z);
    if (MODE == XF_HVPMEAN || MODE == XF_ENERGY) {
        double tot[NQ];
        block_sum<T, NQ>(acc, sm.red, tot);
        finalize_partials(a.red, tot);
    }
}

// ---- inverse: spectrum plane -> real plane (modes of k_xinv) --------------------
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(plane_nt(M)) k_plane_inv(XiArgs<T> a) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int RX = G::RX, L1 = G::L1x;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PlaneSmem<T, M> sm(smem_raw);
    const int z = blockIdx.x;
    C w[G::L1y];
    p4_load_spec<T, M>(w, a.main, a.nyq, z);
    p4_inv_y<T, M>(w, sm, a.tw);
    // the pointwise operands are fetched before the x transform (in flight during it) when
    // registers allow, i.e. in single precision
    constexpr bool EARLY = sizeof(T) == 4;
    C p[RX][L1], vv[RX][L1];
    auto fetch = [&]() {
        if (MODE != XI_PLAIN) {
#pragma unroll
            for (int r = 0; r < RX; ++r)
#pragma unroll
                for (int m = 0; m < L1; ++m) {
                    const size_t idx = p4_idx<M>(z, r, m);
                    p[r][m] = reinterpret_cast<const C*>(a.phi)[idx];
                    if (MODE == XI_HVP) vv[r][m] = reinterpret_cast<const C*>(a.v)[idx];
                }
        }
    };
    if (EARLY) fetch();
    C u[RX][L1];
    p4_inv_x<T, M>(u, sm, a.tw);
    if (!EARLY) fetch();
    T mean = (T)0;
    if (MODE != XI_PLAIN) mean = (T)(*a.msum * a.inv_n);
    double mx = 0.0;
#pragma unroll
    for (int r = 0; r < RX; ++r)
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const C zz = u[r][m];
            C o;
            if (MODE == XI_PLAIN) {
                o = mk<T>(zz.x * a.oscale, zz.y * a.oscale);
            } else if (MODE == XI_HVP) {
                o.x = zz.x + f2v(a.model, p[r][m].x) * vv[r][m].x - mean;
                o.y = zz.y + f2v(a.model, p[r][m].y) * vv[r][m].y - mean;
            } else {
                o.x = zz.x + f1v(a.model, p[r][m].x) - mean;
                o.y = zz.y + f1v(a.model, p[r][m].y) - mean;
                mx = fmax(mx, fmax(fabs((double)o.x), fabs((double)o.y)));
            }
            reinterpret_cast<C*>(a.out)[p4_idx<M>(z, r, m)] = o;
        }
    if (MODE == XI_GRAD) {
        double mm = block_max(mx, sm.red);
        finalize_partials(a.red, &mm);
    }
}

// ---- inverse -> pointwise -> forward on a plane (modes of k_xmid) ----------------
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(plane_nt(M)) k_plane_mid(XmArgs<T> a) {
    using G = PlaneGeo<M>;
    using C = cplx<T>;
    constexpr int RX = G::RX, L1 = G::L1x;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PlaneSmem<T, M> sm(smem_raw);
    const int z = blockIdx.x;
    C w[G::L1y];
    p4_load_spec<T, M>(w, a.main, a.nyq, z);
    p4_inv_y<T, M>(w, sm, a.tw);
    constexpr bool EARLY = sizeof(T) == 4;
    C p[RX][L1], gg[RX][L1];
    auto fetch = [&]() {
#pragma unroll
        for (int r = 0; r < RX; ++r)
#pragma unroll
            for (int m = 0; m < L1; ++m) {
                const size_t idx = p4_idx<M>(z, r, m);
                p[r][m] = reinterpret_cast<const C*>(a.phi)[idx];
                if (MODE == XM_IMEX) gg[r][m] = reinterpret_cast<const C*>(a.g)[idx];
            }
    };
    if (EARLY) fetch();
    C u[RX][L1];
    p4_inv_x<T, M>(u, sm, a.tw);
    if (!EARLY) fetch();
#pragma unroll
    for (int r = 0; r < RX; ++r)
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const T dx = u[r][m].x * a.scale, dy = u[r][m].y * a.scale;
            if (MODE == XM_IMEX) {
                u[r][m].x = dx - a.model.eta * (gg[r][m].x + f2v(a.model, p[r][m].x) * dx);
                u[r][m].y = dy - a.model.eta * (gg[r][m].y + f2v(a.model, p[r][m].y) * dy);
            } else {
                u[r][m].x = f2v(a.model, p[r][m].x) * dx;
                u[r][m].y = f2v(a.model, p[r][m].y) * dy;
            }
        }
    __syncthreads();    // the inverse's last reads of A precede the forward's first writes
    p4_fwd_x<T, M>(u, sm, a.tw);
    p4_fwd_y<T, M>(w, sm, a.tw);
    p4_store_spec<T, M>(w, sm, a.main, a.nyq, z);
}

}  // namespace lbtr
