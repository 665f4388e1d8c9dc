// FP64 instantiation (the build checked against the FP64 oracle).
#include "lbm_launch_impl.cuh"
template struct lbm::Ops<double>;
