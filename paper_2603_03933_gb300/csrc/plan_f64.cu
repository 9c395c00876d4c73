// double instantiation of the LB operator plan.
#include "plan_impl.cuh"
namespace lbtr { template class Plan<double>; }
