// Method definitions of Plan<T>; included by the per-precision translation units.
#pragma once
#include <cmath>
#include <cstring>

#include "plan.cuh"
#include "planes.cuh"
#include "lines.cuh"
#include "rows.cuh"
#include "imex_fused.cuh"
#include "imex3d.cuh"
#include "hvp3d.cuh"

namespace lbtr {

#define LB_CK(call)                                                              \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) { err = std::string(#call) + ": " + cudaGetErrorString(e_); return 6; } \
    } while (0)

// Dispatch a compile-time grid size M over the supported powers of two.
#define LB_SWITCH_M(mval, ...)                                      \
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

// x rows: the four-step row kernels for M >= 16, the shared-memory Stockham kernels for M = 8
template <typename T, int M> int rows_grid(int rows) { return (rows + RowGeo<M>::NR - 1) / RowGeo<M>::NR; }
template <typename T, int M, int MODE> void launch_xfwd(const XfArgs<T>& a, int grid, cudaStream_t s) {
    if constexpr (M >= 16) k_rows_fwd<T, M, MODE><<<rows_grid<T, M>(a.rows), 128, rows_smem<T, M>(), s>>>(a);
    else k_xfwd<T, M, MODE><<<grid, x_nt(M), x_smem<T>(M), s>>>(a);
}
template <typename T, int M, int MODE> void launch_xinv(const XiArgs<T>& a, int grid, cudaStream_t s) {
    if constexpr (M >= 16) k_rows_inv<T, M, MODE><<<rows_grid<T, M>(a.rows), 128, rows_smem<T, M>(), s>>>(a);
    else k_xinv<T, M, MODE><<<grid, x_nt(M), x_smem<T>(M), s>>>(a);
}
template <typename T, int M, int MODE> void launch_xmid(const XmArgs<T>& a, int grid, cudaStream_t s) {
    if constexpr (M >= 16) k_rows_mid<T, M, MODE><<<rows_grid<T, M>(a.rows), 128, rows_smem<T, M>(), s>>>(a);
    else k_xmid<T, M, MODE><<<grid, x_nt(M), x_smem<T>(M), s>>>(a);
}
template <typename T, int M, int MODE> void launch_cols(const ColArgs<T>& a, int grid, cudaStream_t s) {
    k_cols<T, M, MODE><<<grid, col_nt(M), col_smem<T>(M), s>>>(a);
}

template <typename T, int M, int MODE> void launch_pfwd(const XfArgs<T>& a, cudaStream_t s) {
    if constexpr (M >= 32 && M <= 128) k_plane_fwd<T, M, MODE><<<M, plane_nt(M), plane_smem<T>(M), s>>>(a);
}
template <typename T, int M, int MODE> void launch_pinv(const XiArgs<T>& a, cudaStream_t s) {
    if constexpr (M >= 32 && M <= 128) k_plane_inv<T, M, MODE><<<M, plane_nt(M), plane_smem<T>(M), s>>>(a);
}
template <typename T, int M, int MODE> void launch_pmid(const XmArgs<T>& a, cudaStream_t s) {
    if constexpr (M >= 32 && M <= 128) k_plane_mid<T, M, MODE><<<M, plane_nt(M), plane_smem<T>(M), s>>>(a);
}

template <typename T, int M, int MODE> void launch_lines(const ColArgs<T>& a, int ntiles, int grid, cudaStream_t s) {
    if constexpr (M >= 16 && M <= 256 && ln_mode_ok(MODE)) k_lines<T, M, MODE><<<grid, ln_nt(M), ln_smem<T>(M), s>>>(a, ntiles);
}

// Shared-memory attributes of the pipelined column passes; *per = CTAs per SM of the C_LAM pass.
template <typename T, int M> cudaError_t set_lines_attrs(int* per) {
    cudaError_t e = cudaSuccess;
    *per = 0;
    if constexpr (M >= 16 && M <= 256) {
        auto setl = [&](const void* f) {
            cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ln_smem<T>(M));
            if (r != cudaSuccess) e = r;
        };
        setl((const void*)k_lines<T, M, C_FWD>);
        setl((const void*)k_lines<T, M, C_INV>);
        setl((const void*)k_lines<T, M, C_LAM>);
        setl((const void*)k_lines<T, M, C_LAM_E>);
        setl((const void*)k_lines<T, M, C_SOLVE>);
        setl((const void*)k_lines_b<T, M, C_LAM>);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_lines<T, M, C_LAM>, ln_nt(M), ln_smem<T>(M));
    }
    return e;
}

template <typename T, int M> cudaError_t set_plane_attrs() {
    cudaError_t e = cudaSuccess;
    if constexpr (M >= 32 && M <= 128) {
        auto setp = [&](const void* f) {
            cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem<T>(M));
            if (r != cudaSuccess) e = r;
        };
        setp((const void*)k_plane_fwd<T, M, XF_PLAIN>);
        setp((const void*)k_plane_fwd<T, M, XF_HVPMEAN>);
        setp((const void*)k_plane_fwd<T, M, XF_ENERGY>);
        setp((const void*)k_plane_fwd<T, M, XF_IMEX0>);
        setp((const void*)k_plane_inv<T, M, XI_PLAIN>);
        setp((const void*)k_plane_inv<T, M, XI_HVP>);
        setp((const void*)k_plane_inv<T, M, XI_GRAD>);
        setp((const void*)k_plane_mid<T, M, XM_IMEX>);
        setp((const void*)k_plane_mid<T, M, XM_TOP>);
    }
    return e;
}

template <typename T, int M, int TPC> const void* zl_kernel() {
    if constexpr (M >= 16 && M <= 256) return (const void*)k_imex_lines<T, M, TPC>;
    return nullptr;
}

template <typename T, int M, int TPC> const void* zf_kernel() {
    if constexpr (M >= 16) return (const void*)k_imex_zfused<T, M, TPC>;
    return nullptr;
}

template <typename T, int M> cudaError_t set_smem_attrs() {
    cudaError_t e = cudaSuccess;
    auto setx = [&](const void* f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)x_smem<T>(M));
        if (r != cudaSuccess) e = r;
    };
    auto setc = [&](const void* f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)col_smem<T>(M));
        if (r != cudaSuccess) e = r;
    };
    setx((const void*)k_xfwd<T, M, XF_PLAIN>);
    setx((const void*)k_xfwd<T, M, XF_HVPMEAN>);
    setx((const void*)k_xfwd<T, M, XF_ENERGY>);
    setx((const void*)k_xfwd<T, M, XF_IMEX0>);
    setx((const void*)k_xinv<T, M, XI_PLAIN>);
    setx((const void*)k_xinv<T, M, XI_HVP>);
    setx((const void*)k_xinv<T, M, XI_GRAD>);
    setx((const void*)k_xmid<T, M, XM_IMEX>);
    setx((const void*)k_xmid<T, M, XM_TOP>);
    if constexpr (M >= 16) {
        auto setr = [&](const void* f) {
            cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem<T, M>());
            if (r != cudaSuccess) e = r;
        };
        setr((const void*)k_rows_fwd<T, M, XF_PLAIN>);
        setr((const void*)k_rows_fwd<T, M, XF_HVPMEAN>);
        setr((const void*)k_rows_fwd<T, M, XF_ENERGY>);
        setr((const void*)k_rows_fwd<T, M, XF_IMEX0>);
        setr((const void*)k_rows_inv<T, M, XI_PLAIN>);
        setr((const void*)k_rows_inv<T, M, XI_HVP>);
        setr((const void*)k_rows_inv<T, M, XI_GRAD>);
        setr((const void*)k_rows_mid<T, M, XM_IMEX>);
        setr((const void*)k_rows_mid<T, M, XM_TOP>);
        setr((const void*)k_rows_fwd_b<T, M, XF_HVPMEAN>);
        setr((const void*)k_rows_inv_b<T, M, XI_HVP>);
    }
    setc((const void*)k_cols<T, M, C_FWD>);
    setc((const void*)k_cols<T, M, C_INV>);
    setc((const void*)k_cols<T, M, C_LAM>);
    setc((const void*)k_cols<T, M, C_LAM_E>);
    setc((const void*)k_cols<T, M, C_QUAD_E>);
    setc((const void*)k_cols<T, M, C_IMEX_IN>);
    setc((const void*)k_cols<T, M, C_IMEX_OUT>);
    setc((const void*)k_cols<T, M, C_TOP_OUT>);
    setc((const void*)k_cols<T, M, C_MSCALE_IN>);
    setc((const void*)k_cols<T, M, C_SOLVE>);
    setc((const void*)k_cols<T, M, C_DBOX>);
    return e;
}

template <typename T> Plan<T>::~Plan() {
    if (d_base_) cudaFree(d_base_);
}

template <typename T>
int Plan<T>::init(int dim, int m, const double box[3], double xi, double tau, double gamma, std::string& err) {
    dim_ = dim; m_ = m; h_ = m / 2;
    rows_ = dim == 3 ? m * m : m;
    n_ = (long long)rows_ * m;
    for (int i = 0; i < 3; ++i) box_[i] = box[i];
    set_params(xi, tau, gamma);

    int dev = 0, nsm = 0;
    LB_CK(cudaGetDevice(&dev));
    LB_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    cudaError_t ea = cudaSuccess;
    LB_SWITCH_M(m_, ea = set_smem_attrs<T, M>());
    if (ea != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea); return 6; }
    use_planes_ = (dim_ == 3 && m_ >= 32 && m_ <= 128);
    hvp3_ = (sizeof(T) == 4 && dim_ == 3 && m_ == H3::M);
    if (hvp3_) {
        ea = cudaFuncSetAttribute((const void*)k_hvp_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)H3::FSMEM);
        if (ea != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea); return 6; }
        // the fused kernel needs every CTA resident at once (cooperative launch); without
        // that, products take the plane kernels below
        int per = 0;
        ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hvp_fused<T>, H3::NT, H3::FSMEM);
        if (ea != cudaSuccess) { err = std::string("cudaOccupancyMaxActiveBlocksPerMultiprocessor: ") + cudaGetErrorString(ea); return 6; }
        int coop = 0;
        LB_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        hvp3_grid_ = (coop && per > 0) ? nsm * per : 0;
        if constexpr (sizeof(T) == 4) {
            // the persistent subproblem kernel (k_imex3)
            const size_t sm3 = I3_SMEM;
            ea = cudaFuncSetAttribute((const void*)k_imex3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
            if (ea != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea); return 6; }
            int per3 = 0;
            ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per3, k_imex3<T>, H3::NT, sm3);
            if (ea != cudaSuccess) { err = std::string("cudaOccupancyMaxActiveBlocksPerMultiprocessor: ") + cudaGetErrorString(ea); return 6; }
            const int g3 = nsm * per3;
            // every warp owns at most one z-line task, and task warps are at most half of the
            // CTA (each parks its lines in the scratch of a warp without a task)
            imex3_grid_ = (coop && per3 > 0 && 2 * i3_task_warps(g3) <= 32 && g3 <= I3_MAXG) ? g3 : 0;
            imex3_smem_ = sm3;
        }
    }
    if (use_planes_) {
        LB_SWITCH_M(m_, ea = set_plane_attrs<T, M>());
        if (ea != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea); return 6; }
    }

    {
        int per = 0;
        LB_SWITCH_M(m_, ea = set_lines_attrs<T, M>(&per));
        if (ea != cudaSuccess) { err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ea); return 6; }
        ln_grid_cap_ = per > 0 ? nsm * per : 0;
    }
    if (dim_ == 3 && !use_planes_ && ln_grid_cap_ > 0) {
        // the three line passes of a 3D product as one cooperative launch (k_lines3)
        int per = 0, coop = 0;
        LB_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        LB_SWITCH_M(m_, {
            if constexpr (M >= 16 && M <= 256) {
                ea = cudaFuncSetAttribute((const void*)k_lines3<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)ln_smem<T>(M));
                if (ea == cudaSuccess)
                    ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lines3<T, M>, ln_nt(M), ln_smem<T>(M));
            }
        });
        if (ea != cudaSuccess) { err = std::string("k_lines3 attributes: ") + cudaGetErrorString(ea); return 6; }
        // at most 512 CTAs: k_lines3 adds its per-CTA shares with one load round of 16 per lane
        ln3_grid_ = (coop && per > 0 && nsm * per <= 512) ? nsm * per : 0;
    }

    int occ = 0;
    LB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_secular<T>, 256, 3 * m_ * sizeof(T)));
    if (occ < 1) occ = 1;
    coop_blocks_ = nsm * occ;
    if (coop_blocks_ > 4 * nsm) coop_blocks_ = 4 * nsm;

    // fused reciprocal-space IMEX kernel: smallest tiles-per-CTA whose cooperative grid
    // fits on the device with the columns resident in shared memory
    {
        const int nb_main_i = (int)(((long long)(dim_ == 3 ? m_ * h_ : h_) + COL_NL - 1) / COL_NL);
        const int nb_nyq_i = ((dim_ == 3 ? m_ : 1) + COL_NL - 1) / COL_NL;
        zf_ntiles_ = nb_main_i + nb_nyq_i;
        zf_nbmain_ = nb_main_i;
        zf_tpc_ = 0;
        zf_lines_ = false;
        // register-resident columns, every tile on the device at once: the first of
        // 1, 2, 4 tiles per CTA whose cooperative grid fits without spilling registers
        for (int tpc = 1; tpc <= 4 && m_ >= 16 && m_ <= 256; tpc *= 2) {
            const size_t sm = sizeof(T) == 8 ? zl_smem<double>(m_, tpc) : zl_smem<float>(m_, tpc);
            if (sm > 227 * 1024) continue;
            const void* f = nullptr;
            LB_SWITCH_M(m_, {
                if (tpc == 1) f = zl_kernel<T, M, 1>();
                else if (tpc == 2) f = zl_kernel<T, M, 2>();
                else f = zl_kernel<T, M, 4>();
            });
            if (!f) continue;
            cudaFuncAttributes fa;
            LB_CK(cudaFuncGetAttributes(&fa, f));
            if (fa.localSizeBytes > 64) continue;     // a variant that spills more than a few registers is not taken
            LB_CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            int per = 0;
            LB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, zl_nt(m_, tpc), sm));
            const int grid = (zf_ntiles_ + tpc - 1) / tpc;
            if (per >= 1 && grid <= per * nsm && grid <= 2048) {     // 2048: the reducing barrier's tree
                zf_lines_ = true; zf_tpc_ = tpc; zf_grid_ = grid; zf_smem_ = sm;
                break;
            }
        }
        for (int tpc = 1; tpc <= 4 && m_ >= 16 && !zf_lines_; tpc *= 2) {
            const size_t sm = sizeof(T) == 8 ? zf_smem<double>(m_, tpc) : zf_smem<float>(m_, tpc);
            if (sm > 227 * 1024) break;
            const void* f = nullptr;
            LB_SWITCH_M(m_, {
                if (tpc == 1) f = zf_kernel<T, M, 1>();
                else if (tpc == 2) f = zf_kernel<T, M, 2>();
                else f = zf_kernel<T, M, 4>();
            });
            if (!f) break;
            LB_CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            int per = 0;
            LB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, zf_nt(m_, tpc), sm));
            const int grid = (zf_ntiles_ + tpc - 1) / tpc;
            if (per >= 1 && grid <= per * nsm) { zf_tpc_ = tpc; zf_grid_ = grid; zf_smem_ = sm; break; }
        }
    }
    int gx = (rows_ + x_nl(m_) - 1) / x_nl(m_);
    int gc = (int)((((long long)rows_ * h_) + COL_NL - 1) / COL_NL + (rows_ + COL_NL - 1) / COL_NL);
    max_blocks_ = std::max(std::max(gx, gc), std::max(coop_blocks_, 8 * nsm));

    const long long sl = spec_len();
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    size_t o_tw = take(sizeof(C) * m_);
    size_t o_q = take(sizeof(T) * 3 * m_);
    size_t o_w = take(sizeof(C) * sl);
    size_t o_w2 = take(sizeof(C) * sl);
    size_t o_b0 = take(sizeof(C) * sl);
    size_t o_b1 = take(sizeof(C) * sl);
    size_t o_p = take(sizeof(double) * S_COUNT * SLOT_Q * (size_t)max_blocks_);
    size_t o_r = take(sizeof(double) * S_COUNT * SLOT_Q);
    size_t o_t = take(sizeof(unsigned) * S_COUNT);
    size_t o_sp = take(sizeof(double) * (2 * 5 * (size_t)std::max(std::max(coop_blocks_, zf_grid_), imex3_grid_) +
                                         5 * 64 + 8));
    size_t o_bar = take(sizeof(unsigned) * BAR_WORDS);
    size_t o_err = take(sizeof(int));
    size_t o_st = take(sizeof(ImexState));
    bytes_ = off;
    cudaError_t ma = cudaMalloc(&d_base_, bytes_);
    if (ma != cudaSuccess) { err = "cudaMalloc of the plan workspace failed"; d_base_ = nullptr; return 7; }
    char* b = static_cast<char*>(d_base_);
    d_tw_ = reinterpret_cast<C*>(b + o_tw);
    d_qtab_ = reinterpret_cast<T*>(b + o_q);
    d_work_ = reinterpret_cast<C*>(b + o_w);
    d_work2_ = reinterpret_cast<C*>(b + o_w2);
    d_b_[0] = reinterpret_cast<C*>(b + o_b0);
    d_b_[1] = reinterpret_cast<C*>(b + o_b1);
    d_partials_ = reinterpret_cast<double*>(b + o_p);
    d_result_ = reinterpret_cast<double*>(b + o_r);
    d_ticket_ = reinterpret_cast<unsigned*>(b + o_t);
    d_secpart_ = reinterpret_cast<double*>(b + o_sp);
    d_bar_ = reinterpret_cast<unsigned*>(b + o_bar);
    d_err_ = reinterpret_cast<int*>(b + o_err);
    d_state_ = reinterpret_cast<ImexState*>(b + o_st);
    LB_CK(cudaMemset(d_base_, 0, bytes_));

    // twiddles W_M^j = exp(-2 pi i j / M), evaluated in long double on the host
    std::vector<C> tw(m_);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int j = 0; j < m_; ++j) {
        long double ang = -2.0L * pi * (long double)j / (long double)m_;
        tw[j] = mk<T>((T)cosl(ang), (T)sinl(ang));
    }
    // |Bk|^2 per axis: (2 pi / L_a)^2 k^2 with the signed wavenumber of each index
    std::vector<T> q(3 * m_, (T)0);
    for (int a = 0; a < 3; ++a) {
        if (a >= dim_) break;
        long double c = 2.0L * pi / (long double)box_[a];
        for (int i = 0; i < m_; ++i) {
            int k = i < m_ / 2 ? i : i - m_;
            q[a * m_ + i] = (T)(c * c * (long double)k * (long double)k);
        }
    }
    LB_CK(cudaMemcpy(d_tw_, tw.data(), sizeof(C) * m_, cudaMemcpyHostToDevice));
    LB_CK(cudaMemcpy(d_qtab_, q.data(), sizeof(T) * 3 * m_, cudaMemcpyHostToDevice));
    return 0;
}

template <typename T> void Plan<T>::set_params(double xi, double tau, double gamma) {
    xi2_ = xi * xi; tau_ = tau; gamma_ = gamma;
    model_.tau = (T)tau; model_.gamma = (T)gamma; model_.eta = (T)eta;
}

template <typename T> RedSlot Plan<T>::redslot(int slot, int nq, unsigned max_mask) {
    RedSlot r;
    r.partials = d_partials_ + (size_t)slot * SLOT_Q * max_blocks_;
    r.result = d_result_ + slot * SLOT_Q;
    r.ticket = d_ticket_ + slot;
    r.nq = nq;
    r.max_mask = max_mask;
    return r;
}

template <typename T>
void Plan<T>::xfwd(int mode, const T* in, const T* phi, const T* g, const T* d0, const double* dscale,
                   C* spec, int slot, cudaStream_t s, const int* done, bool partials_only) {
    XfArgs<T> a;
    a.in = in; a.phi = phi; a.g = g; a.d0 = d0; a.dscale = dscale;
    a.main = spec; a.nyq = spec + (size_t)rows_ * h_;
    a.tw = d_tw_; a.rows = rows_; a.model = model_; a.model.eta = (T)eta;
    a.red = redslot(slot, mode == XF_ENERGY ? 4 : 1, 0u);
    if (partials_only) a.red.ticket = nullptr;
    a.done = done;
    int grid = (rows_ + x_nl(m_) - 1) / x_nl(m_);
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    LB_SWITCH_M(m_, {
        if (mode == XF_PLAIN) launch_xfwd<T, M, XF_PLAIN>(a, grid, s);
        else if (mode == XF_HVPMEAN) launch_xfwd<T, M, XF_HVPMEAN>(a, grid, s);
        else if (mode == XF_ENERGY) launch_xfwd<T, M, XF_ENERGY>(a, grid, s);
        else launch_xfwd<T, M, XF_IMEX0>(a, grid, s);
    });
    if (prof_) {
        double nf = mode == XF_HVPMEAN ? 2 : mode == XF_IMEX0 ? (d0 ? 3 : 2) : 1;
        prof_->end(K_XFWD, e0, s, nf * fb() + sb());
    }
}

template <typename T>
void Plan<T>::xinv(int mode, const C* spec, T* out, const T* phi, const T* v, const double* msum, T oscale,
                   int slot, cudaStream_t s, const int* done) {
    XiArgs<T> a;
    a.main = spec; a.nyq = spec + (size_t)rows_ * h_;
    a.out = out; a.phi = phi; a.v = v; a.msum = msum; a.inv_n = 1.0 / (double)n_; a.oscale = oscale;
    a.tw = d_tw_; a.rows = rows_; a.model = model_;
    a.red = redslot(slot, 1, 1u);
    a.done = done;
    int grid = (rows_ + x_nl(m_) - 1) / x_nl(m_);
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    LB_SWITCH_M(m_, {
        if (mode == XI_PLAIN) launch_xinv<T, M, XI_PLAIN>(a, grid, s);
        else if (mode == XI_HVP) launch_xinv<T, M, XI_HVP>(a, grid, s);
        else launch_xinv<T, M, XI_GRAD>(a, grid, s);
    });
    if (prof_) prof_->end(K_XINV, e0, s, sb() + (mode == XI_HVP ? 3 : mode == XI_GRAD ? 2 : 1) * fb());
}

template <typename T>
void Plan<T>::xmid(int mode, C* spec, const T* phi, const T* g, T scale, cudaStream_t s, const int* done) {
    XmArgs<T> a;
    a.main = spec; a.nyq = spec + (size_t)rows_ * h_;
    a.phi = phi; a.g = g; a.tw = d_tw_; a.rows = rows_; a.scale = scale;
    a.model = model_; a.model.eta = (T)eta;
    a.done = done;
    int grid = (rows_ + x_nl(m_) - 1) / x_nl(m_);
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    LB_SWITCH_M(m_, {
        if (mode == XM_IMEX) launch_xmid<T, M, XM_IMEX>(a, grid, s);
        else launch_xmid<T, M, XM_TOP>(a, grid, s);
    });
    if (prof_) prof_->end(K_XMID, e0, s, 2 * sb() + (mode == XM_IMEX ? 2 : 1) * fb());
}

// axis: 1 = Y, 2 = Z
template <typename T>
int Plan<T>::col_args(int axis, int mode, C* spec, C* dst, const C* src, T kscale, double escale, double sigma,
                      const double* lam, int slot, const int* done, ColArgs<T>& a) const {
    const long long M = m_, H = h_;
    a.main = spec; a.nyq = spec ? spec + (size_t)rows_ * h_ : nullptr;
    a.dst_main = dst; a.dst_nyq = dst ? dst + (size_t)rows_ * h_ : nullptr;
    a.src_main = src; a.src_nyq = src ? src + (size_t)rows_ * h_ : nullptr;
    a.tw = d_tw_; a.qtab = d_qtab_;
    ColSeg s0{}, s1{};
    auto lg = [](long long v) { int k = 0; while ((1LL << k) < v) ++k; return k; };
    if (dim_ == 3 && axis == 1) {
        s0 = ColSeg{(int)(M * H), lg(H), M * H, 1, H, 0, -1};
        s1 = ColSeg{(int)M, 0, M, 0, 1, 1, (int)H};
    } else if (dim_ == 3) {
        s0 = ColSeg{(int)(M * H), lg(M * H), 0, 1, M * H, 0, -1};
        s1 = ColSeg{(int)M, lg(M), 0, 1, M, 0, (int)H};
    } else {
        s0 = ColSeg{(int)H, lg(H), 0, 1, H, 0, -1};
        s1 = ColSeg{1, 0, 0, 0, 1, 1, (int)H};
    }
    a.seg[0] = s0; a.seg[1] = s1;
    a.nb_main = (s0.nlines + COL_NL - 1) / COL_NL;
    int grid = a.nb_main + (s1.nlines + COL_NL - 1) / COL_NL;
    a.dim = dim_; a.xi2 = (T)xi2_; a.kscale = kscale; a.escale = escale; a.eta = (T)eta;
    a.sigma = (T)sigma; a.lam = lam;
    a.red = const_cast<Plan<T>*>(this)->redslot(slot, mode == C_IMEX_OUT ? 2 : mode == C_DBOX ? 3 : 1, 0u);
    a.done = done;
    return grid;
}

template <typename T>
void Plan<T>::cols(int axis, int mode, C* spec, C* dst, const C* src, T kscale, double escale, double sigma,
                   const double* lam, int slot, cudaStream_t s, const int* done) {
    ColArgs<T> a;
    const int grid = col_args(axis, mode, spec, dst, src, kscale, escale, sigma, lam, slot, done, a);
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    const bool lines = ln_grid_cap_ > 0 && ln_mode_ok(mode) && dst == nullptr && src == nullptr;
    if (lines) {
        const int lg_grid = std::min(grid, ln_grid_cap_);
        LB_SWITCH_M(m_, {
            switch (mode) {
                case C_FWD: launch_lines<T, M, C_FWD>(a, grid, lg_grid, s); break;
                case C_INV: launch_lines<T, M, C_INV>(a, grid, lg_grid, s); break;
                case C_LAM: launch_lines<T, M, C_LAM>(a, grid, lg_grid, s); break;
                case C_LAM_E: launch_lines<T, M, C_LAM_E>(a, grid, lg_grid, s); break;
                default: launch_lines<T, M, C_SOLVE>(a, grid, lg_grid, s); break;
            }
        });
    } else LB_SWITCH_M(m_, {
        switch (mode) {
            case C_FWD: launch_cols<T, M, C_FWD>(a, grid, s); break;
            case C_INV: launch_cols<T, M, C_INV>(a, grid, s); break;
            case C_LAM: launch_cols<T, M, C_LAM>(a, grid, s); break;
            case C_LAM_E: launch_cols<T, M, C_LAM_E>(a, grid, s); break;
            case C_QUAD_E: launch_cols<T, M, C_QUAD_E>(a, grid, s); break;
            case C_IMEX_IN: launch_cols<T, M, C_IMEX_IN>(a, grid, s); break;
            case C_IMEX_OUT: launch_cols<T, M, C_IMEX_OUT>(a, grid, s); break;
            case C_TOP_OUT: launch_cols<T, M, C_TOP_OUT>(a, grid, s); break;
            case C_SOLVE: launch_cols<T, M, C_SOLVE>(a, grid, s); break;
            case C_DBOX: launch_cols<T, M, C_DBOX>(a, grid, s); break;
            default: launch_cols<T, M, C_MSCALE_IN>(a, grid, s); break;
        }
    });
    if (prof_) {
        const bool innermost = (dim_ == 3) ? axis == 2 : axis == 1;
        double ns = mode == C_QUAD_E ? 1 : (mode == C_IMEX_OUT || mode == C_TOP_OUT) ? 3 : 2;
        prof_->end(innermost ? K_COLI : K_COLY, e0, s, ns * sb());
    }
}

// All transforms except the innermost axis, forward (x pass, plus y in 3D).
template <typename T>
void Plan<T>::fwd_outer(int mode, const T* in, const T* phi, const T* g, const T* d0, const double* dscale,
                        C* spec, int slot, cudaStream_t s, const int* done) {
    if (!use_planes_) {
        xfwd(mode, in, phi, g, d0, dscale, spec, slot, s, done);
        if (dim_ == 3) cols(1, C_FWD, spec, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, s, done);
        return;
    }
    XfArgs<T> a;
    a.in = in; a.phi = phi; a.g = g; a.d0 = d0; a.dscale = dscale;
    a.main = spec; a.nyq = spec + (size_t)rows_ * h_;
    a.tw = d_tw_; a.rows = rows_; a.model = model_; a.model.eta = (T)eta;
    a.red = redslot(slot, mode == XF_ENERGY ? 4 : 1, 0u);
    a.done = done;
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    LB_SWITCH_M(m_, {
        if (mode == XF_PLAIN) launch_pfwd<T, M, XF_PLAIN>(a, s);
        else if (mode == XF_HVPMEAN) launch_pfwd<T, M, XF_HVPMEAN>(a, s);
        else if (mode == XF_ENERGY) launch_pfwd<T, M, XF_ENERGY>(a, s);
        else launch_pfwd<T, M, XF_IMEX0>(a, s);
    });
    if (prof_) {
        double nf = mode == XF_HVPMEAN ? 2 : mode == XF_IMEX0 ? (d0 ? 3 : 2) : 1;
        prof_->end(K_XFWD, e0, s, nf * fb() + sb());
    }
}

// All transforms except the innermost axis, inverse, with the x-pass epilogue.
template <typename T>
void Plan<T>::inv_outer(int mode, C* spec, T* out, const T* phi, const T* v, const double* msum, T oscale,
                        int slot, cudaStream_t s, const int* done) {
    if (!use_planes_) {
        if (dim_ == 3) cols(1, C_INV, spec, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, s, done);
        xinv(mode, spec, out, phi, v, msum, oscale, slot, s, done);
        return;
    }
    XiArgs<T> a;
    a.main = spec; a.nyq = spec + (size_t)rows_ * h_;
    a.out = out; a.phi = phi; a.v = v; a.msum = msum; a.inv_n = 1.0 / (double)n_; a.oscale = oscale;
    a.tw = d_tw_; a.rows = rows_; a.model = model_;
    a.red = redslot(slot, 1, 1u);
    a.done = done;
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    LB_SWITCH_M(m_, {
        if (mode == XI_PLAIN) launch_pinv<T, M, XI_PLAIN>(a, s);
        else if (mode == XI_HVP) launch_pinv<T, M, XI_HVP>(a, s);
        else launch_pinv<T, M, XI_GRAD>(a, s);
    });
    if (prof_) prof_->end(K_XINV, e0, s, sb() + (mode == XI_HVP ? 3 : mode == XI_GRAD ? 2 : 1) * fb());
}

// Inverse outer transforms -> pointwise -> forward outer transforms.
template <typename T>
void Plan<T>::mid_outer(int mode, C* spec, const T* phi, const T* g, T scale, cudaStream_t s, const int* done) {
    if (!use_planes_) {
        if (dim_ == 3) cols(1, C_INV, spec, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, s, done);
        xmid(mode, spec, phi, g, scale, s, done);
        if (dim_ == 3) cols(1, C_FWD, spec, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, s, done);
        return;
    }
    XmArgs<T> a;
    a.main = spec; a.nyq = spec + (size_t)rows_ * h_;
    a.phi = phi; a.g = g; a.tw = d_tw_; a.rows = rows_; a.scale = scale;
    a.model = model_; a.model.eta = (T)eta;
    a.done = done;
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    LB_SWITCH_M(m_, {
        if (mode == XM_IMEX) launch_pmid<T, M, XM_IMEX>(a, s);
        else launch_pmid<T, M, XM_TOP>(a, s);
    });
    if (prof_) prof_->end(K_XMID, e0, s, 2 * sb() + (mode == XM_IMEX ? 2 : 1) * fb());
}

template <typename T> void Plan<T>::hessvec(const T* phi, const T* v, T* hv, cudaStream_t s) {
    if (hvp3_grid_ > 0) {
        Hvp3Args<T> a;
        a.v = v; a.phi = phi; a.hv = hv; a.spec = d_work_; a.tw = d_tw_; a.qtab = d_qtab_;
        a.model = model_;
        a.partials = d_partials_;
        a.bar.count = d_bar_; a.bar.gen = d_bar_ + 32; a.bar.err = d_err_; a.bar.budget = budget_; a.bar.tree = d_bar_ + 64;
        a.inv_n = 1.0 / (double)n_;
        a.xi2 = (T)xi2_;
        a.kscale = (T)(1.0 / (double)n_);
        {
            void* args[] = {&a};
            cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
            cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_hvp_fused<T>, dim3(hvp3_grid_), dim3(H3::NT),
                                                        args, H3::FSMEM, s);
            if (e != cudaSuccess && launch_err_ == cudaSuccess) launch_err_ = e;
            if (prof_) prof_->end(K_XFWD, e0, s, 3 * fb());
            return;
        }
    }
    if (ln3_grid_ > 0) {
        // 3D on the x-row path: x rows forward, the three line passes in one launch, x rows inverse
        // the row kernel leaves its sums of F''(phi) v per block; k_lines3 combines them
        xfwd(XF_HVPMEAN, v, phi, nullptr, nullptr, nullptr, d_work_, S_HVP, s, nullptr, true);
        int nrp = 0;
        LB_SWITCH_M(m_, { if constexpr (M >= 16) nrp = rows_grid<T, M>(rows_); });
        const double* rpart = d_partials_ + (size_t)S_HVP * SLOT_Q * max_blocks_;
        double* l2 = d_secpart_;
        double* msum = slot_mut(S_HVP);
        ColArgs<T> yf, zl, yi;
        const int ty = col_args(1, C_FWD, d_work_, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, nullptr, yf);
        const int tz = col_args(2, C_LAM, d_work_, nullptr, nullptr, (T)(1.0 / (double)n_), 0.0, 0.0, nullptr, S_RED0,
                                nullptr, zl);
        col_args(1, C_INV, d_work_, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, nullptr, yi);
        GridBar bar;
        bar.count = d_bar_; bar.gen = d_bar_ + 32; bar.err = d_err_; bar.budget = budget_; bar.tree = d_bar_ + 64;
        int ty_ = ty, tz_ = tz;
        void* args[] = {&yf, &zl, &yi, &ty_, &tz_, &bar, &rpart, &nrp, &l2, &msum};
        const void* f = nullptr;
        LB_SWITCH_M(m_, { if constexpr (M >= 16 && M <= 256) f = (const void*)k_lines3<T, M>; });
        cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
        cudaError_t e = f ? cudaLaunchCooperativeKernel(f, dim3(ln3_grid_), dim3(ln_nt(m_)), args, ln_smem<T>(m_), s)
                          : cudaErrorInvalidValue;
        if (e != cudaSuccess && launch_err_ == cudaSuccess) launch_err_ = e;
        if (prof_) prof_->end(K_COLI, e0, s, 6 * sb());
        xinv(XI_HVP, d_work_, hv, phi, v, slot(S_HVP), (T)1, S_RED0, s);
        return;
    }
    const int inner = dim_ == 3 ? 2 : 1;
    fwd_outer(XF_HVPMEAN, v, phi, nullptr, nullptr, nullptr, d_work_, S_HVP, s);
    cols(inner, C_LAM, d_work_, nullptr, nullptr, (T)(1.0 / (double)n_), 0.0, 0.0, nullptr, S_RED0, s);
    inv_outer(XI_HVP, d_work_, hv, phi, v, slot(S_HVP), (T)1, S_RED0, s);
}

// The three argument structs of hessvec on the 2D x-row path, for batched launches of many
// problems of the same size; false on other paths.
template <typename T>
bool Plan<T>::hvp_args(const T* phi, const T* v, T* hv, XfArgs<T>& xf, ColArgs<T>& ca, int& col_grid,
                       int& col_tiles, XiArgs<T>& xi, bool any_lines) const {
    // 2D only: a 3D grid on the x-row path also has its y passes, which the batched
    // launches (rows forward, innermost lines, rows inverse) do not make
    if (dim_ != 2 || m_ < 16 || (ln_grid_cap_ <= 0 && !any_lines)) return false;
    Plan<T>* self = const_cast<Plan<T>*>(this);
    xf.in = v; xf.phi = phi; xf.g = nullptr; xf.d0 = nullptr; xf.dscale = nullptr;
    xf.main = d_work_; xf.nyq = d_work_ + (size_t)rows_ * h_;
    xf.tw = d_tw_; xf.rows = rows_; xf.model = model_; xf.model.eta = (T)eta;
    xf.red = self->redslot(S_HVP, 1, 0u);
    xf.done = nullptr;
    const int inner = dim_ == 3 ? 2 : 1;
    col_tiles = col_args(inner, C_LAM, d_work_, nullptr, nullptr, (T)(1.0 / (double)n_), 0.0, 0.0, nullptr, S_RED0,
                         nullptr, ca);
    col_grid = ln_grid_cap_ > 0 ? std::min(col_tiles, ln_grid_cap_) : col_tiles;
    xi.main = d_work_; xi.nyq = d_work_ + (size_t)rows_ * h_;
    xi.out = hv; xi.phi = phi; xi.v = v; xi.msum = self->slot(S_HVP); xi.inv_n = 1.0 / (double)n_;
    xi.oscale = (T)1; xi.tw = d_tw_; xi.rows = rows_; xi.model = model_; xi.model.eta = (T)eta;
    xi.red = self->redslot(S_RED0, 1, 1u);
    xi.done = nullptr;
    return true;
}

// hessvec of `count` problems of grid size m at once (device argument arrays from hvp_args)
template <typename T>
cudaError_t launch_hvp_batch(int m, int rows, int count, const XfArgs<T>* xf, const ColArgs<T>* ca, int col_grid,
                             int col_tiles, const XiArgs<T>* xi, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    LB_SWITCH_M(m, {
        if constexpr (M >= 16) {
            const dim3 gx((unsigned)rows_grid<T, M>(rows), (unsigned)count);
            k_rows_fwd_b<T, M, XF_HVPMEAN><<<gx, 128, rows_smem<T, M>(), s>>>(xf);
            if constexpr (M <= 256) {
                k_lines_b<T, M, C_LAM><<<dim3((unsigned)col_grid, (unsigned)count), ln_nt(M), ln_smem<T>(M), s>>>(ca, col_tiles);
            } else {
                e = cudaErrorInvalidValue;
            }
            k_rows_inv_b<T, M, XI_HVP><<<gx, 128, rows_smem<T, M>(), s>>>(xi);
        } else {
            e = cudaErrorInvalidValue;
        }
    });
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

template <typename T> void Plan<T>::energy_grad(const T* phi, T* grad, cudaStream_t s) {
    const int inner = dim_ == 3 ? 2 : 1;
    const double inv_n = 1.0 / (double)n_;
    fwd_outer(XF_ENERGY, phi, phi, nullptr, nullptr, nullptr, d_work_, S_EF, s);
    if (grad) {
        cols(inner, C_LAM_E, d_work_, nullptr, nullptr, (T)inv_n, inv_n * inv_n, 0.0, nullptr, S_EG, s);
        inv_outer(XI_GRAD, d_work_, grad, phi, nullptr, slot(S_EF) + 1, (T)1, S_GMAX, s);
    } else {
        cols(inner, C_QUAD_E, d_work_, nullptr, nullptr, (T)1, inv_n * inv_n, 0.0, nullptr, S_EG, s);
    }
}

template <typename T> void Plan<T>::box_derivs(const T* x, cudaStream_t s) {
    const int inner = dim_ == 3 ? 2 : 1;
    const double inv_n = 1.0 / (double)n_;
    fwd_outer(XF_PLAIN, x, nullptr, nullptr, nullptr, nullptr, d_work_, S_RED0, s);
    cols(inner, C_DBOX, d_work_, nullptr, nullptr, (T)1, inv_n * inv_n, 0.0, nullptr, S_DBOX, s);
}

template <typename T> void Plan<T>::quad_energy(const T* x, cudaStream_t s) {
    const int inner = dim_ == 3 ? 2 : 1;
    const double inv_n = 1.0 / (double)n_;
    fwd_outer(XF_PLAIN, x, nullptr, nullptr, nullptr, nullptr, d_work_, S_RED0, s);
    cols(inner, C_QUAD_E, d_work_, nullptr, nullptr, (T)1, inv_n * inv_n, 0.0, nullptr, S_QUAD, s);
}

template <typename T> void Plan<T>::phys_reduce(int op, const T* x, const T* y, int slot, cudaStream_t s) {
    PhysRedArgs<T> a;
    a.x = x; a.y = y; a.n = n_;
    int grid = (int)std::min<long long>(max_blocks_, (n_ + 255) / 256);
    if (grid < 1) grid = 1;
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    if (op == R_DOT) {
        a.red = redslot(slot, 1, 0u);
        k_physred<T, R_DOT><<<grid, 256, 0, s>>>(a);
    } else if (op == R_SUMSQ_MAX) {
        a.red = redslot(slot, 2, 2u);
        k_physred<T, R_SUMSQ_MAX><<<grid, 256, 0, s>>>(a);
    } else if (op == R_POW23) {
        a.red = redslot(slot, 2, 0u);
        k_physred<T, R_POW23><<<grid, 256, 0, s>>>(a);
    } else {
        a.red = redslot(slot, 2, 0u);
        k_physred<T, R_SUM_SUMSQ><<<grid, 256, 0, s>>>(a);
    }
    if (prof_) prof_->end(K_REDUCE, e0, s, (op == R_DOT ? 2 : 1) * fb());
}

template <typename T> void Plan<T>::secular(const C* b, int check, int j, cudaStream_t s) {
    SecArgs<T> a;
    a.bmain = b; a.bnyq = b + (size_t)rows_ * h_;
    a.qtab = d_qtab_;
    a.res = slot(S_IMEX);
    a.st = d_state_;
    a.partials = d_secpart_;
    a.bar.count = d_bar_; a.bar.gen = d_bar_ + 32; a.bar.err = d_err_; a.bar.budget = budget_; a.bar.tree = d_bar_ + 64;
    a.dim = dim_; a.m = m_; a.rows = rows_;
    a.inv_n2 = 1.0 / ((double)n_ * (double)n_);
    a.eta = eta; a.r = r_; a.rtol = rtol_; a.steptol = steptol_;
    a.eps_abs = eps_abs_; a.eps_rel_abs = eps_rel_abs_; a.stall = stall_k();
    a.check = check; a.max_iter = max_iter_;
    a.xi2 = (T)xi2_;
    void* args[] = {&a};
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_secular<T>, dim3(coop_blocks_), dim3(256), args,
                                                3 * m_ * sizeof(T), s);
    if (e != cudaSuccess && launch_err_ == cudaSuccess) launch_err_ = e;
    if (prof_) prof_->end(K_SECULAR, e0, s, sb());
}

template <typename T> void Plan<T>::zfused(const C* bold, C* bnew, int check, cudaStream_t s) {
    ZfArgs<T> a;
    a.work = d_work_; a.bold = bold; a.bnew = bnew;
    a.tw = d_tw_; a.qtab = d_qtab_;
    const long long M = m_, H = h_;
    auto lg = [](long long v) { int k = 0; while ((1LL << k) < v) ++k; return k; };
    if (dim_ == 3) {
        a.seg[0] = ColSeg{(int)(M * H), lg(M * H), 0, 1, M * H, 0, -1};
        a.seg[1] = ColSeg{(int)M, lg(M), 0, 1, M, 0, (int)H};
    } else {
        a.seg[0] = ColSeg{(int)H, lg(H), 0, 1, H, 0, -1};
        a.seg[1] = ColSeg{1, 0, 0, 0, 1, 1, (int)H};
    }
    a.nb_main = zf_nbmain_; a.ntiles = zf_ntiles_;
    a.dim = dim_; a.m = m_;
    a.st = d_state_;
    a.partials = d_secpart_;
    a.bar.count = d_bar_; a.bar.gen = d_bar_ + 32; a.bar.err = d_err_; a.bar.budget = budget_; a.bar.tree = d_bar_ + 64;
    a.xi2 = (T)xi2_; a.eta = (T)eta;
    a.inv_n = 1.0 / (double)n_; a.inv_n2 = 1.0 / ((double)n_ * (double)n_);
    a.r = r_; a.rtol = rtol_; a.steptol = steptol_; a.eps_abs = eps_abs_; a.eps_rel_abs = eps_rel_abs_;
    a.stall = stall_k();
    a.check = check; a.max_iter = max_iter_;
    a.spec_half = (long long)rows_ * h_;
    a.t_thr_abs2 = (T)(eps_abs_ * eta * eps_abs_ * eta);
    a.t_thr_rel2 = (T)(eps_rel_abs_ * eta * eps_rel_abs_ * eta);
    a.t_r2 = (T)(r_ * r_);
    a.t_rtol_r2 = (T)(rtol_ * r_ * r_);
    a.t_inv_n2 = (T)a.inv_n2;
    void* args[] = {&a};
    const void* f = nullptr;
    LB_SWITCH_M(m_, {
        if (zf_lines_) {
            if (zf_tpc_ == 1) f = zl_kernel<T, M, 1>();
            else if (zf_tpc_ == 2) f = zl_kernel<T, M, 2>();
            else f = zl_kernel<T, M, 4>();
        } else {
            if (zf_tpc_ == 1) f = zf_kernel<T, M, 1>();
            else if (zf_tpc_ == 2) f = zf_kernel<T, M, 2>();
            else f = zf_kernel<T, M, 4>();
        }
    });
    const int nt = zf_lines_ ? zl_nt(m_, zf_tpc_) : zf_nt(m_, zf_tpc_);
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    cudaError_t e = cudaLaunchCooperativeKernel(f, dim3(zf_grid_), dim3(nt), args, zf_smem_, s);
    if (e != cudaSuccess && launch_err_ == cudaSuccess) launch_err_ = e;
    if (prof_) prof_->end(K_COLI, e0, s, 4 * sb());
}

template <typename T>
int Plan<T>::imex_init(const T* phi, const T* g, const T* d0, const double* dscale_dev, double r,
                       double eps_abs, double eps_rel_abs, int max_iter, cudaStream_t s) {
    r_ = r; eps_abs_ = eps_abs; eps_rel_abs_ = eps_rel_abs; max_iter_ = max_iter;
    rtol_ = sizeof(T) == 8 ? 1e-13 : 2e-6;
    steptol_ = sizeof(T) == 8 ? 1e-15 : 1e-8;
    model_.eta = (T)eta;
    const int inner = dim_ == 3 ? 2 : 1;
    cudaMemsetAsync(d_state_, 0, sizeof(ImexState), s);
    cudaMemsetAsync(d_b_[1], 0, sizeof(C) * spec_len(), s);
    fwd_outer(XF_IMEX0, nullptr, phi, g, d0, dscale_dev, d_work_, S_RED0, s);
    if (zf_tpc_ > 0) {
        zfused(d_b_[1], d_b_[0], 0, s);
        return 0;
    }
    const double inv_n = 1.0 / (double)n_;
    cols(inner, C_IMEX_OUT, d_work_, d_b_[0], d_b_[1], (T)1, inv_n * inv_n, 0.0, nullptr, S_IMEX, s);
    secular(d_b_[0], 0, 0, s);
    return 0;
}

template <typename T> int Plan<T>::imex_iterate(const T* phi, const T* g, int j0, int count, cudaStream_t s) {
    const int inner = dim_ == 3 ? 2 : 1;
    const double inv_n = 1.0 / (double)n_;
    const int* done = &d_state_->done;
    if (zf_tpc_ > 0) {
        // d_work_ holds d_j after the inner inverse; x/y pass builds b_j; the fused kernel
        // does the rest of the iteration
        for (int j = j0; j < j0 + count; ++j) {
            mid_outer(XM_IMEX, d_work_, phi, g, (T)1, s, done);
            zfused(d_b_[(j - 1) & 1], d_b_[j & 1], 1, s);
        }
        return 0;
    }
    for (int j = j0; j < j0 + count; ++j) {
        C* src = d_b_[(j - 1) & 1];
        C* dst = d_b_[j & 1];
        cols(inner, C_IMEX_IN, nullptr, d_work_, src, (T)inv_n, 0.0, 0.0, &d_state_->lam, S_RED0, s, done);
        mid_outer(XM_IMEX, d_work_, phi, g, (T)1, s, done);
        cols(inner, C_IMEX_OUT, d_work_, dst, src, (T)1, inv_n * inv_n, 0.0, nullptr, S_IMEX, s, done);
        secular(dst, 1, j, s);
    }
    return 0;
}

template <typename T>
int Plan<T>::imex_persistent(const T* phi, const T* g, const T* d0, const double* dscale_dev, T* d, double r,
                             double eps_abs, double eps_rel_abs, int max_iter, cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        return -1;
    } else {
        if (imex3_grid_ <= 0) return -1;
        r_ = r; eps_abs_ = eps_abs; eps_rel_abs_ = eps_rel_abs; max_iter_ = max_iter;
        rtol_ = 2e-6;
        steptol_ = 1e-8;
        model_.eta = (T)eta;
        cudaMemsetAsync(d_state_, 0, sizeof(ImexState), s);
        Imex3Args<T> a;
        a.phi = phi; a.g = g; a.d0 = d0; a.dscale = dscale_dev; a.d = d;
        a.spec = d_work_; a.b0 = d_b_[0]; a.b1 = d_b_[1];
        a.tw = d_tw_; a.qtab = d_qtab_;
        a.model = model_;
        a.st = d_state_;
        a.partials = reinterpret_cast<Part<T>*>(d_secpart_);
        a.bar.count = d_bar_; a.bar.gen = d_bar_ + 32; a.bar.err = d_err_; a.bar.budget = budget_; a.bar.tree = d_bar_ + 64;
        a.xi2 = (T)xi2_; a.eta = (T)eta; a.kscale = (T)(1.0 / (double)n_);
        a.r = r_; a.rtol = rtol_; a.steptol = steptol_;
        a.stall = stall_k(); a.max_iter = max_iter_;
        const double inv_n2 = 1.0 / ((double)n_ * (double)n_);
        a.t_thr_abs2 = (T)(eps_abs_ * eta * eps_abs_ * eta);
        a.t_thr_rel2 = (T)(eps_rel_abs_ * eta * eps_rel_abs_ * eta);
        a.t_r2 = (T)(r_ * r_);
        a.t_rtol_r2 = (T)(rtol_ * r_ * r_);
        a.t_inv_n2 = (T)inv_n2;
        void* args[] = {&a};
        cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_imex3<T>, dim3(imex3_grid_), dim3(H3::NT), args,
                                                    imex3_smem_, s);
        if (e != cudaSuccess && launch_err_ == cudaSuccess) launch_err_ = e;
        if (prof_) prof_->end(K_COLI, e0, s, 0.0);
        return 0;
    }
}

template <typename T> void Plan<T>::imex_final(T* d, cudaStream_t s) {
    // caller has synchronised and knows final_src via the state
    ImexState st;
    cudaMemcpyAsync(&st, d_state_, sizeof(ImexState), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    const int inner = dim_ == 3 ? 2 : 1;
    const double inv_n = 1.0 / (double)n_;
    cols(inner, C_IMEX_IN, nullptr, d_work_, d_b_[st.final_src & 1], (T)inv_n, 0.0, 0.0, &d_state_->final_lam,
         S_RED0, s);
    inv_outer(XI_PLAIN, d_work_, d, nullptr, nullptr, nullptr, (T)1, S_RED0, s);
}

template <typename T> void Plan<T>::to_spectrum(const T* x, C* out, cudaStream_t s) {
    // paper-normalised coefficients: DFT / N
    const int inner = dim_ == 3 ? 2 : 1;
    fwd_outer(XF_PLAIN, x, nullptr, nullptr, nullptr, nullptr, out, S_RED0, s);
    cols(inner, C_FWD, out, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, s);
    long long len = spec_len() * 2;
    k_axpby<T><<<(int)std::min<long long>(4096, (len + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<T*>(out), reinterpret_cast<const T*>(out), 1.0 / (double)n_, 0.0, nullptr, 0.0, len);
}

template <typename T> void Plan<T>::from_spectrum(const C* q, T* x, bool msc, double sigma, cudaStream_t s) {
    const int inner = dim_ == 3 ? 2 : 1;
    if (msc) {
        cols(inner, C_MSCALE_IN, nullptr, d_work2_, q, (T)1, 0.0, sigma, nullptr, S_RED0, s);
    } else {
        cudaMemcpyAsync(d_work2_, q, sizeof(C) * spec_len(), cudaMemcpyDeviceToDevice, s);
        cols(inner, C_INV, d_work2_, nullptr, nullptr, (T)1, 0.0, 0.0, nullptr, S_RED0, s);
    }
    inv_outer(XI_PLAIN, d_work2_, x, nullptr, nullptr, nullptr, (T)1, S_RED0, s);
}

template <typename T> void Plan<T>::kop(const T* phi, const C* q, C* out, double sigma, cudaStream_t s) {
    const int inner = dim_ == 3 ? 2 : 1;
    cols(inner, C_MSCALE_IN, nullptr, d_work2_, q, (T)1, 0.0, sigma, nullptr, S_RED0, s);
    mid_outer(XM_TOP, d_work2_, phi, nullptr, (T)1, s);
    cols(inner, C_TOP_OUT, d_work2_, out, q, (T)(1.0 / (double)n_), 0.0, sigma, nullptr, S_RED0, s);
}

template <typename T> void Plan<T>::precond(const T* x, T* out, double shift, cudaStream_t s) {
    const int inner = dim_ == 3 ? 2 : 1;
    fwd_outer(XF_PLAIN, x, nullptr, nullptr, nullptr, nullptr, d_work2_, S_RED0, s);
    cols(inner, C_SOLVE, d_work2_, nullptr, nullptr, (T)(1.0 / (double)n_), 0.0, shift, nullptr, S_RED0, s);
    inv_outer(XI_PLAIN, d_work2_, out, nullptr, nullptr, nullptr, (T)1, S_RED0, s);
}

template <typename T> void Plan<T>::taylor_rem(const T* v, const T* sd, int slot, cudaStream_t s) {
    int grid = (int)std::min<long long>(max_blocks_, (n_ + 255) / 256);
    if (grid < 1) grid = 1;
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    k_taylor_rem<T><<<grid, 256, 0, s>>>(v, sd, n_, model_, redslot(slot, 1, 0u));
    if (prof_) prof_->end(K_REDUCE, e0, s, 2 * fb());
}

template <typename T> void Plan<T>::axpby(T* y, const T* x, double a, double b, cudaStream_t s) {
    int grid = (int)std::min<long long>(4 * max_blocks_, (n_ + 255) / 256);
    if (grid < 1) grid = 1;
    cudaEvent_t e0 = prof_ ? prof_->begin(s) : nullptr;
    k_axpby<T><<<grid, 256, 0, s>>>(y, x, a, b, nullptr, 0.0, n_);
    if (prof_) prof_->end(K_REDUCE, e0, s, (b == 0.0 ? 2 : 3) * fb());
}

template <typename T> void Plan<T>::sub_scalar(T* y, const double* c, double scale, cudaStream_t s) {
    int grid = (int)std::min<long long>(4 * max_blocks_, (n_ + 255) / 256);
    k_sub_scalar<T><<<grid, 256, 0, s>>>(y, c, scale, n_);
}

template <typename T> void Plan<T>::random_normal(T* out, unsigned long long seed, unsigned stream, cudaStream_t s) {
    int grid = (int)std::min<long long>(4 * max_blocks_, (n_ / 2 + 255) / 256 + 1);
    k_philox_normal<T><<<grid, 256, 0, s>>>(out, n_, seed, stream);
}

template <typename T> int Plan<T>::read_error(cudaStream_t s) {
    int e = 0;
    cudaMemcpyAsync(&e, d_err_, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (e) reset_barrier(s);
    return e;
}

template <typename T> void Plan<T>::reset_barrier(cudaStream_t s) {
    cudaMemsetAsync(d_bar_, 0, BAR_WORDS * sizeof(unsigned), s);
    cudaMemsetAsync(d_err_, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
}

}  // namespace lbtr
