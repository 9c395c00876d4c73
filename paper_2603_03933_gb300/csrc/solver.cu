// Outer IMEX-TR loop (Algorithms 1 and 2) and the Lanczos lambda_min driver.
#include "ctx.cuh"

template <typename T>
lb_status lb_ctx::lambda_min(lbtr::Plan<T>& p, const T* phi, const lb_eig_opts& o, T* vec, lb_eig_info* info,
                             cudaStream_t s) {
    (void)p; (void)phi; (void)o; (void)vec; (void)info; (void)s;
    err = "lb_lambda_min: not built yet";
    return LB_ERR_UNSUPPORTED;
}
template lb_status lb_ctx::lambda_min<float>(lbtr::Plan<float>&, const float*, const lb_eig_opts&, float*,
                                             lb_eig_info*, cudaStream_t);
template lb_status lb_ctx::lambda_min<double>(lbtr::Plan<double>&, const double*, const lb_eig_opts&, double*,
                                              lb_eig_info*, cudaStream_t);

lb_status lb_ctx::tr_solve(double* phi, const lb_tr_opts& o, lb_tr_info* info, cudaStream_t s) {
    (void)phi; (void)o; (void)info; (void)s;
    err = "lb_imex_tr_solve: not built yet";
    return LB_ERR_UNSUPPORTED;
}
