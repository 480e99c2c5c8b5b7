// thermo.h -- host FP64 thermodynamics and parameter derivation (Sec. 3, App. B).
#pragma once

namespace lbm_host {

struct CS {  // Carnahan-Starling EOS, Eq. (28)
    double a, b, R;
    double p(double rho, double T) const;
    double dp(double rho, double T) const;   // d p / d rho
    double mu(double rho, double T) const;   // Eq. (29)
};

// Critical point: dp/drho = d2p/drho2 = 0.  Returns 0 or a negative LBM_ERR code.
int critical(const CS& eos, double* rho_c, double* T_c, double* p_c);
// Maxwell coexistence at temperature T: equal pressure and chemical potential.
int maxwell(const CS& eos, double T, double* rho_v, double* rho_l, double* p0);
// Appendix B: eps with F(eps) = 0 (Eq. S13), Newton from eps = 2, Simpson quadrature.
int li_epsilon(const CS& eos, double T, double rho_v, double rho_l, double p0, double* eps);
// Continuum planar profile of the free-energy model (Eq. 26): width and surface tension.
int fe_theory(const CS& eos, double T, double rho_v, double rho_l, double p0, double kappa,
              double* width, double* gamma);
// Continuum planar profile of the pseudopotential model (Eq. S44, S46).
int pp_theory(const CS& eos, double T, double rho_v, double rho_l, double p0, double eps,
              double kappa_P, double kappa_Li, double* width, double* gamma);
// Consistent densities of a 2-D droplet: equal chemical potential, p(rho_l) - p(rho_v) =
// gamma / radius (Laplace), Newton from (rho_v, rho_l).
int kelvin_2d(const CS& eos, double T, double gamma, double radius, double* rho_v, double* rho_l);

}  // namespace lbm_host
