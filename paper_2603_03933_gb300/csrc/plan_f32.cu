// float instantiation of the LB operator plan (the mixed-precision working type).
#include "plan_impl.cuh"
namespace lbtr {
template class Plan<float>;
template cudaError_t launch_hvp_batch<float>(int, int, int, const XfArgs<float>*, const ColArgs<float>*, int, int,
                                          const XiArgs<float>*, cudaStream_t);
}
