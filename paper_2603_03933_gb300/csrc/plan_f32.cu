// float instantiation of the LB operator plan (the mixed-precision working type).
#include "plan_impl.cuh"
namespace lbtr { template class Plan<float>; }
