// double instantiation of the LB operator plan.
#include "plan_impl.cuh"
namespace lbtr {
template class Plan<double>;
template cudaError_t launch_hvp_batch<double>(int, int, int, const XfArgs<double>*, const ColArgs<double>*, int, int,
                                          const XiArgs<double>*, cudaStream_t);
}
