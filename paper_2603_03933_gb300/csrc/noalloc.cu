// lb_hessvec_noalloc: the Hessian-vector product without any device allocation.
//
// Some callers cannot call cudaMalloc: plug-ins hosted by a framework whose caching
// allocator owns all device memory and forbids side allocations, and latency-critical
// loops that must not pay the implicit device synchronisation of cudaMalloc/cudaFree.
// This entry point serves them: it needs no lb_ctx, and its scratch (one half
// spectrum, the reduction partials, the twiddle and wavenumber tables) lives in a
// file-scope __device__ array of fixed size.  The caller passes only the problem, the
// input fields and the output field.  Every call writes its tables into that array with
// a small kernel on the caller's stream, so after the first call on a device (which
// resolves the array's address) a call only enqueues kernels.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/lbtr.h"
#include "planes.cuh"

namespace lbtr {
namespace {

constexpr size_t kScratchBytes = 3u << 20;     // 3 MiB per device, held until process exit
constexpr long long kMaxPoints = 1LL << 18;     // N <= 2^18: up to 64^3 or 512^2
constexpr int kMaxDevices = 64;

// The scratch itself.  Host code must never dereference or pass this symbol: on the
// host it is a stand-in, not a device address; its device address comes from
// cudaGetSymbolAddress in device_setup below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DevState {
    bool ready = false;
    unsigned char* base = nullptr;             // device address of g_noalloc_scratch
};
DevState g_dev[kMaxDevices];
std::mutex g_mu;

#define NA_SWITCH_M(mval, ...)                                      \
    switch (mval) {                                                 \
        case 8: { constexpr int M = 8; __VA_ARGS__; } break;        \
        case 16: { constexpr int M = 16; __VA_ARGS__; } break;      \
        case 32: { constexpr int M = 32; __VA_ARGS__; } break;      \
        case 64: { constexpr int M = 64; __VA_ARGS__; } break;      \
        case 128: { constexpr int M = 128; __VA_ARGS__; } break;    \
        case 256: { constexpr int M = 256; __VA_ARGS__; } break;    \
        case 512: { constexpr int M = 512; __VA_ARGS__; } break;    \
        default: break;                                             \
    }

template <typename T, int M> cudaError_t set_attrs() {
    cudaError_t e = cudaSuccess, r;
    r = cudaFuncSetAttribute((const void*)k_xfwd<T, M, XF_HVPMEAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)x_smem<T>(M));
    if (r != cudaSuccess) e = r;
    r = cudaFuncSetAttribute((const void*)k_xinv<T, M, XI_HVP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)x_smem<T>(M));
    if (r != cudaSuccess) e = r;
    for (const void* f : {(const void*)k_cols<T, M, C_FWD>, (const void*)k_cols<T, M, C_INV>,
                          (const void*)k_cols<T, M, C_LAM>}) {
        r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem<T>(M));
        if (r != cudaSuccess) e = r;
    }
    if constexpr (M >= 32 && M <= 128) {
        r = cudaFuncSetAttribute((const void*)k_plane_fwd<T, M, XF_HVPMEAN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem<T>(M));
        if (r != cudaSuccess) e = r;
        r = cudaFuncSetAttribute((const void*)k_plane_inv<T, M, XI_HVP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem<T>(M));
        if (r != cudaSuccess) e = r;
    }
    return e;
}

// Once per device, with that device current: resolve the scratch address and set the
// shared-memory limits of the kernels used below.  Neither step allocates memory.
cudaError_t device_setup(int dev, unsigned char** base) {
    std::lock_guard<std::mutex> lk(g_mu);
    DevState& d = g_dev[dev];
    if (d.ready) { *base = d.base; return cudaSuccess; }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    for (int m = 8; m <= 512; m *= 2) {
        cudaError_t r = cudaSuccess;
        NA_SWITCH_M(m, r = set_attrs<double, M>(); if (r == cudaSuccess) r = set_attrs<float, M>());
        if (r != cudaSuccess) return r;
    }
    d.base = static_cast<unsigned char*>(p);
    d.ready = true;
    *base = d.base;
    return cudaSuccess;
}

// The twiddles W_M^j = exp(-2 pi i j / M) and the per-axis |Bk|^2 terms (2 pi k / L_a)^2
// (signed wavenumber k of index i) of one problem, evaluated in double and rounded to T;
// also resets the reduction ticket.  One block; m <= 512.
template <typename T>
__global__ void k_noalloc_tables(cplx<T>* tw, T* qt, unsigned* ticket, int m, int dim, double lx, double ly,
                                 double lz) {
    const double two_pi = 6.283185307179586476925286766559;
    const double len[3] = {lx, ly, lz};
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)j / (double)m, &sn, &cs);
        tw[j] = mk<T>((T)cs, (T)sn);
    }
    for (int i = threadIdx.x; i < 3 * m; i += blockDim.x) {
        const int ax = i / m, idx = i % m;
        const int k = idx < m / 2 ? idx : idx - m;
        double q = 0.0;
        if (ax < dim) {
            const double c = two_pi / len[ax];
            q = c * c * (double)k * (double)k;
        }
        qt[i] = (T)q;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

struct Layout {
    size_t spec, tw, qtab, partials, result, ticket, total;
};

template <typename T> Layout layout(long long spec_len, int m, int max_blocks) {
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    Layout L{};
    size_t off = 0;
    L.spec = off; off += up(sizeof(cplx<T>) * (size_t)spec_len);
    L.tw = off; off += up(sizeof(cplx<T>) * (size_t)m);
    L.qtab = off; off += up(sizeof(T) * 3 * (size_t)m);
    L.partials = off; off += up(sizeof(double) * (size_t)max_blocks);
    L.result = off; off += up(sizeof(double) * 4);
    L.ticket = off; off += up(sizeof(unsigned));
    L.total = off;
    return L;
}

template <typename T>
lb_status run(const lb_problem& pr, const T* phi, const T* v, T* hv, cudaStream_t s, unsigned char* base) {
    using C = cplx<T>;
    const int m = pr.n, h = m / 2, dim = pr.dim;
    const int rows = dim == 3 ? m * m : m;
    const long long n = (long long)rows * m;
    const long long slen = (long long)rows * (h + 1);
    const bool planes = (dim == 3 && m >= 32 && m <= 128);
    const int gx = planes ? m : (rows + x_nl(m) - 1) / x_nl(m);
    const Layout L = layout<T>(slen, m, gx);
    if (L.total > kScratchBytes) return LB_ERR_UNSUPPORTED;
    C* spec = reinterpret_cast<C*>(base + L.spec);
    C* tw = reinterpret_cast<C*>(base + L.tw);
    T* qt = reinterpret_cast<T*>(base + L.qtab);
    double* partials = reinterpret_cast<double*>(base + L.partials);
    double* result = reinterpret_cast<double*>(base + L.result);
    unsigned* ticket = reinterpret_cast<unsigned*>(base + L.ticket);

    // tables of this problem and the reduction ticket, written on the device in stream
    // order (the shared array keeps the last call's contents, so the ticket must be reset)
    k_noalloc_tables<T><<<1, 512, 0, s>>>(tw, qt, ticket, m, dim, pr.box[0], pr.box[1], dim == 3 ? pr.box[2] : 1.0);
    if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;

    Model<T> model;
    model.tau = (T)pr.tau; model.gamma = (T)pr.gamma; model.eta = (T)0.1;
    RedSlot rs;
    rs.partials = partials; rs.result = result; rs.ticket = ticket; rs.nq = 1; rs.max_mask = 0u;

    XfArgs<T> xf{};
    xf.in = v; xf.phi = phi; xf.main = spec; xf.nyq = spec + (size_t)rows * h;
    xf.tw = tw; xf.rows = rows; xf.model = model; xf.red = rs; xf.done = nullptr;
    XiArgs<T> xi{};
    xi.main = spec; xi.nyq = spec + (size_t)rows * h; xi.out = hv; xi.phi = phi; xi.v = v;
    xi.msum = result; xi.inv_n = 1.0 / (double)n; xi.oscale = (T)1; xi.tw = tw; xi.rows = rows;
    xi.model = model; xi.red = rs; xi.done = nullptr;

    auto lg = [](long long val) { int k = 0; while ((1LL << k) < val) ++k; return k; };
    auto colargs = [&](int axis) {
        ColArgs<T> a{};
        const long long M = m, H = h;
        a.main = spec; a.nyq = spec + (size_t)rows * h;
        a.tw = tw; a.qtab = qt;
        if (dim == 3 && axis == 1) {
            a.seg[0] = ColSeg{(int)(M * H), lg(H), M * H, 1, H, 0, -1};
            a.seg[1] = ColSeg{(int)M, 0, M, 0, 1, 1, (int)H};
        } else if (dim == 3) {
            a.seg[0] = ColSeg{(int)(M * H), lg(M * H), 0, 1, M * H, 0, -1};
            a.seg[1] = ColSeg{(int)M, lg(M), 0, 1, M, 0, (int)H};
        } else {
            a.seg[0] = ColSeg{(int)H, lg(H), 0, 1, H, 0, -1};
            a.seg[1] = ColSeg{1, 0, 0, 0, 1, 1, (int)H};
        }
        a.nb_main = (a.seg[0].nlines + COL_NL - 1) / COL_NL;
        a.dim = dim; a.xi2 = (T)(pr.xi * pr.xi); a.kscale = (T)(1.0 / (double)n); a.eta = (T)0.1;
        return a;
    };
    auto colgrid = [&](const ColArgs<T>& a) { return a.nb_main + (a.seg[1].nlines + COL_NL - 1) / COL_NL; };

    NA_SWITCH_M(m, {
        if (planes) {
            if constexpr (M >= 32 && M <= 128) {
                k_plane_fwd<T, M, XF_HVPMEAN><<<M, plane_nt(M), plane_smem<T>(M), s>>>(xf);
                ColArgs<T> az = colargs(2);
                k_cols<T, M, C_LAM><<<colgrid(az), col_nt(M), col_smem<T>(M), s>>>(az);
                k_plane_inv<T, M, XI_HVP><<<M, plane_nt(M), plane_smem<T>(M), s>>>(xi);
            }
        } else {
            k_xfwd<T, M, XF_HVPMEAN><<<gx, x_nt(M), x_smem<T>(M), s>>>(xf);
            if (dim == 3) {
                ColArgs<T> ay = colargs(1);
                k_cols<T, M, C_FWD><<<colgrid(ay), col_nt(M), col_smem<T>(M), s>>>(ay);
                ColArgs<T> az = colargs(2);
                k_cols<T, M, C_LAM><<<colgrid(az), col_nt(M), col_smem<T>(M), s>>>(az);
                k_cols<T, M, C_INV><<<colgrid(ay), col_nt(M), col_smem<T>(M), s>>>(ay);
            } else {
                ColArgs<T> ay = colargs(1);
                k_cols<T, M, C_LAM><<<colgrid(ay), col_nt(M), col_smem<T>(M), s>>>(ay);
            }
            k_xinv<T, M, XI_HVP><<<gx, x_nt(M), x_smem<T>(M), s>>>(xi);
        }
    });
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace
}  // namespace lbtr

extern "C" lb_status lb_hessvec_noalloc(const lb_problem* prob, lb_precision prec, const void* phi, const void* v,
                                        void* hv, lb_stream stream) {
    using namespace lbtr;
    if (!prob || !phi || !v || !hv) return LB_ERR_INVALID_ARG;
    if (prob->dim != 2 && prob->dim != 3) return LB_ERR_UNSUPPORTED;
    if (!pow2(prob->n) || prob->n < 8 || prob->n > 512) return LB_ERR_UNSUPPORTED;
    long long npts = 1;
    for (int a = 0; a < prob->dim; ++a) npts *= prob->n;
    if (npts > kMaxPoints) return LB_ERR_UNSUPPORTED;   // beyond the fixed scratch
    for (int a = 0; a < prob->dim; ++a)
        if (!(prob->box[a] > 0.0) || !std::isfinite(prob->box[a])) return LB_ERR_INVALID_ARG;
    if (prec != LB_FP64 && prec != LB_MIXED) return LB_ERR_INVALID_ARG;
    if ((((uintptr_t)phi | (uintptr_t)v | (uintptr_t)hv) & 15u) != 0) return LB_ERR_INVALID_ARG;
    if (hv == phi || hv == v) return LB_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LB_ERR_CUDA;
    unsigned char* base = nullptr;
    if (device_setup(dev, &base) != cudaSuccess) return LB_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == LB_FP64)
        return run<double>(*prob, (const double*)phi, (const double*)v, (double*)hv, s, base);
    return run<float>(*prob, (const float*)phi, (const float*)v, (float*)hv, s, base);
}
