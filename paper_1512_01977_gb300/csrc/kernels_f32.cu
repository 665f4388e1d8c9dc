// FP32 instantiation: populations stored as deviations f_i - w_i rho_ref.
#include "lbm_launch_impl.cuh"
template struct lbm::Ops<float>;
