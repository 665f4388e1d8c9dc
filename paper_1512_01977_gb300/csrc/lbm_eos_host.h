// Host EOS helpers of the library (eos_host.cu).
#pragma once

#include "lbm_axi.h"

namespace lbm {
bool critical_point(const lbm_eos& e, double* Tc, double* rho_c);
bool coexistence(const lbm_eos& e, double T, double* rho_v, double* rho_l);
double absolute_temperature(const lbm_eos& e);
void eos_pressure(const lbm_eos& e, double T, double rho, double* p, double* dp);
}  // namespace lbm
