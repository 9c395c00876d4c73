// Host-side plan of the FFT-based LB operators for one grid and precision.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "aux_kernels.cuh"
#include "passes.cuh"
#include "prof.cuh"
#include "spec_kernels.cuh"

namespace lbtr {

// Result slots of the reductions (each launch that reduces owns one slot).
enum Slot {
    S_HVP = 0,     // sum F''(phi) v
    S_EF = 1,      // [0] sum F, [1] sum F', [2] sum phi, [3] sum phi^2
    S_EG = 2,      // G (Parseval sum)
    S_GMAX = 3,    // max |g|
    S_IMEX = 4,    // [0] sum w |db|^2 / N^2, [1] sum w |b|^2 / N^2
    S_RED0 = 5,    // generic physical reductions
    S_RED1 = 6,
    S_QUAD = 7,    // G(s) of the ratio test
    S_DBOX = 8,    // sum_k 1/2 |phi_hat|^2 dLambda/dL_a * L_a, a = x, y, z
    S_COUNT = 9
};
constexpr int SLOT_Q = 4;           // quantities per slot

struct Status {
    int code = 0;
    std::string msg;
};

template <typename T>
class Plan {
public:
    using C = cplx<T>;
    // The IMEX residual is ||b_{j-1} - b_j|| / eta; in float it stops falling at the rounding
    // level of b, which can lie above the requested tolerance.  The float path therefore
    // also ends, reported as stalled (not converged), after 512 checked iterations without
    // progress (stall_update); 0 in double: the paper's tests alone.
    static int stall_k() { return sizeof(T) == 4 ? 512 : 0; }
    Plan() = default;
    ~Plan();
    int init(int dim, int m, const double box[3], double xi, double tau, double gamma, std::string& err);
    void set_params(double xi, double tau, double gamma);

    // --- operators (all enqueue on `s`) ---
    // Hv = P[F^{-1} Lambda F v + F''(phi) v]
    void hessvec(const T* phi, const T* v, T* hv, cudaStream_t s);
    // energy pieces into slots S_EF (sum F, sum F', sum phi, sum phi^2) and S_EG (G);
    // gradient into grad (if non-null) and max |g| into S_GMAX
    void energy_grad(const T* phi, T* grad, cudaStream_t s);
    // sum_k 1/2 |x_hat_k|^2 4 xi^2 (1 - |Bk|^2) (Bk)_a^2 (a = x, y, z) into S_DBOX
    void box_derivs(const T* x, cudaStream_t s);
    // G(s) = 1/2 sum_k Lambda_k |s_hat_k|^2 into S_QUAD
    void quad_energy(const T* x, cudaStream_t s);
    // physical reductions into slot (R_DOT: sum x y; R_SUMSQ_MAX; R_SUM_SUMSQ)
    void phys_reduce(int op, const T* x, const T* y, int slot, cudaStream_t s);

    // --- subproblem (Algorithm 3) ---
    // Set up b_0 from d0 (or dscale * g) and the first multiplier.
    int imex_init(const T* phi, const T* g, const T* d0, const double* dscale_dev, double r,
                  double eps_abs, double eps_rel_abs, int max_iter, cudaStream_t s);
    // Enqueue iterations j0 .. j0+count-1 (device-side early exit once done).
    int imex_iterate(const T* phi, const T* g, int j0, int count, cudaStream_t s);
    // d = F^{-1}(B[final_src] / (1 + eta (Lambda + final_lam)))
    void imex_final(T* d, cudaStream_t s);
    // The whole solve (init, iterations, the returned iterate d) as one cooperative launch
    // (k_imex3, 3D 128^3 float grids); available() is false elsewhere or when switched off.
    bool imex_persistent_available() const { return imex3_grid_ > 0 && imex3_on_; }
    void set_imex_persistent(bool on) { imex3_on_ = on; }
    int imex_persistent(const T* phi, const T* g, const T* d0, const double* dscale_dev, T* d, double r,
                        double eps_abs, double eps_rel_abs, int max_iter, cudaStream_t s);

    // --- spectral operators used by Lanczos ---
    // out = K q with K = M^{-1/2} H M^{-1/2} (q, out paper-normalised half spectra)
    void kop(const T* phi, const C* q, C* out, double sigma, cudaStream_t s);
    // x (physical) -> paper-normalised half spectrum
    void to_spectrum(const T* x, C* out, cudaStream_t s);
    // paper-normalised half spectrum -> physical; with msc: apply M^{-1/2} first
    void from_spectrum(const C* q, T* x, bool msc, double sigma, cudaStream_t s);

    // out = F^{-1}[(Lambda + shift)^{-1} F x] with the k = 0 mode removed (PCG preconditioner)
    void precond(const T* x, T* out, double shift, cudaStream_t s);
    // sum_x s^2 (F''(v)/2 + F'''(v) s/6 + s^2/24) into slot
    void taylor_rem(const T* v, const T* sd, int slot, cudaStream_t s);
    // y = a x + b y on physical fields
    void axpby(T* y, const T* x, double a, double b, cudaStream_t s);
    // y -= (*c) * scale
    void sub_scalar(T* y, const double* c, double scale, cudaStream_t s);
    // i.i.d. N(0,1) samples from Philox4x32-10 (seed, stream)
    void random_normal(T* out, unsigned long long seed, unsigned stream, cudaStream_t s);
    int max_blocks() const { return max_blocks_; }

    // barrier / error bookkeeping
    void set_barrier_budget(long long cycles) { budget_ = cycles > 0 ? cycles : kDefaultBudget; }
    int read_error(cudaStream_t s);     // returns and clears the device error flag (sync)
    // first error returned by a cooperative launch since the last call (then cleared)
    cudaError_t take_launch_error() { cudaError_t e = launch_err_; launch_err_ = cudaSuccess; return e; }
    void reset_barrier(cudaStream_t s);
    void set_prof(Prof* p) { prof_ = p; }

    // accessors
    const double* slot(int k) const { return d_result_ + k * SLOT_Q; }
    double* slot_mut(int k) { return d_result_ + k * SLOT_Q; }
    ImexState* imex_state() { return d_state_; }
    long long n() const { return n_; }
    long long spec_len() const { return (long long)rows_ * (h_ + 1); }
    int m() const { return m_; }
    int dim() const { return dim_; }
    int rows() const { return rows_; }
    size_t bytes() const { return bytes_; }
    double eta = 0.1;
    int coop_blocks() const { return coop_blocks_; }
    const T* qtab() const { return d_qtab_; }
    T xi2() const { return (T)xi2_; }

    static constexpr long long kDefaultBudget = 4000000000LL;   // ~2 s at 2 GHz

    // the argument structs of one hessvec on the 2D x-row path (for batched launches); false elsewhere.
    // any_lines: also on grids whose line pass has no persistent k_lines variant (the
    // batched sweep kernel brings its own line tiles)
    bool hvp_args(const T* phi, const T* v, T* hv, XfArgs<T>& xf, ColArgs<T>& ca, int& col_grid, int& col_tiles,
                  XiArgs<T>& xi, bool any_lines = false) const;
    int col_args(int axis, int mode, C* spec, C* dst, const C* src, T kscale, double escale, double sigma,
                 const double* lam, int slot, const int* done, ColArgs<T>& a) const;

private:
    // partials_only: the block sums stay per block (for a later kernel to combine)
    void xfwd(int mode, const T* in, const T* phi, const T* g, const T* d0, const double* dscale,
              C* spec, int slot, cudaStream_t s, const int* done = nullptr, bool partials_only = false);
    void xinv(int mode, const C* spec, T* out, const T* phi, const T* v, const double* msum, T oscale,
              int slot, cudaStream_t s, const int* done = nullptr);
    void xmid(int mode, C* spec, const T* phi, const T* g, T scale, cudaStream_t s, const int* done = nullptr);
    void cols(int axis, int mode, C* spec, C* dst, const C* src, T kscale, double escale, double sigma,
              const double* lam, int slot, cudaStream_t s, const int* done = nullptr);
    void fwd_outer(int mode, const T* in, const T* phi, const T* g, const T* d0, const double* dscale, C* spec,
                   int slot, cudaStream_t s, const int* done = nullptr);
    void inv_outer(int mode, C* spec, T* out, const T* phi, const T* v, const double* msum, T oscale, int slot,
                   cudaStream_t s, const int* done = nullptr);
    void mid_outer(int mode, C* spec, const T* phi, const T* g, T scale, cudaStream_t s, const int* done = nullptr);
    RedSlot redslot(int slot, int nq, unsigned max_mask);
    void secular(const C* b, int check, int j, cudaStream_t s);
    void zfused(const C* bold, C* bnew, int check, cudaStream_t s);

    int dim_ = 0, m_ = 0, h_ = 0, rows_ = 0;
    long long n_ = 0;
    double box_[3] = {0, 0, 0};
    double xi2_ = 1, tau_ = 0, gamma_ = 0;
    Model<T> model_{};
    size_t bytes_ = 0;
    int coop_blocks_ = 0;
    long long budget_ = kDefaultBudget;
    // imex parameters of the current solve
    double r_ = 0, eps_abs_ = 0, eps_rel_abs_ = 0, rtol_ = 0, steptol_ = 0;

    int max_iter_ = 0;

    // device memory
    void* d_base_ = nullptr;
    C* d_tw_ = nullptr;        // W_M
    T* d_qtab_ = nullptr;      // [3][M]
    C* d_work_ = nullptr;      // work spectrum (rows*(H+1))
    C* d_work2_ = nullptr;     // second work spectrum
    C* d_b_[2] = {nullptr, nullptr};
    double* d_partials_ = nullptr;   // per-slot partial sums [S_COUNT][SLOT_Q][max_blocks]
    double* d_result_ = nullptr;     // [S_COUNT][SLOT_Q]
    unsigned* d_ticket_ = nullptr;   // [S_COUNT]
    double* d_secpart_ = nullptr;    // [2][3][coop_blocks]
    // barrier words, one 128-byte line each: [0] count, [32] generation, [64] groups done,
    // [64 + 32 (1 + g)] arrivals of group g (g < 64)
    static constexpr int BAR_WORDS = 64 + 32 * 65;
    unsigned* d_bar_ = nullptr;
    int* d_err_ = nullptr;
    ImexState* d_state_ = nullptr;
    int max_blocks_ = 0;
    cudaError_t launch_err_ = cudaSuccess;
    Prof* prof_ = nullptr;
    bool use_planes_ = false;
    bool hvp3_ = false;       // 3D 128^3 float products take the kernels of hvp3d.cuh
    int hvp3_grid_ = 0;       // CTAs of the fused cooperative product (0: three kernels)
    int imex3_grid_ = 0;      // CTAs of the persistent subproblem kernel (0: not available)
    bool imex3_on_ = true;
    size_t imex3_smem_ = 0;   // its dynamic shared memory
    int ln_grid_cap_ = 0;     // persistent grid of the pipelined column passes (0: not used)
    int ln3_grid_ = 0;        // cooperative grid of k_lines3 (3D x-row path products; 0: not used)
    int zf_tpc_ = 0, zf_grid_ = 0, zf_ntiles_ = 0, zf_nbmain_ = 0;
    size_t zf_smem_ = 0;
    bool zf_lines_ = false;   // the fused iteration runs as k_imex_lines (else k_imex_zfused)
    double fb() const { return (double)n_ * sizeof(T); }
    double sb() const { return (double)spec_len() * sizeof(C); }
};

// hessvec of `count` problems of grid size m on the x-row path in one launch per pass;
// xf, ca, xi: device arrays of `count` argument structs from Plan<T>::hvp_args
template <typename T>
cudaError_t launch_hvp_batch(int m, int rows, int count, const XfArgs<T>* xf, const ColArgs<T>* ca, int col_grid,
                             int col_tiles, const XiArgs<T>* xi, cudaStream_t s);

}  // namespace lbtr
