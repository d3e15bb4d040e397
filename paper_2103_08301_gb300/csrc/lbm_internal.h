// Declarations shared by the host translation units of the solver library.
#pragma once

#include <cstdint>

namespace lbm {

// Carnahan-Starling parameters at absolute temperature T.
struct Thermo {
    double a, b, R, T;
};

double cs_pressure(const Thermo &t, double rho);
double cs_dpressure(const Thermo &t, double rho);
void cs_critical(double a, double b, double R, double *Tc, double *rhoc);
// Maxwell coexistence below Tc; returns nonzero at or above Tc.
int maxwell(const Thermo &t, double *rho_g, double *rho_l, double *p_sat);
// Gas-branch density with p0(rho) = p; nonzero if p is outside the branch.
int gas_density(const Thermo &t, double p, double *rho);
// Liquid-branch density with p0(rho) = p below Tc; nonzero otherwise.
int liquid_density(const Thermo &t, double p, double *rho);
double node_noise(uint64_t seed, uint64_t node, double amp);

} // namespace lbm
