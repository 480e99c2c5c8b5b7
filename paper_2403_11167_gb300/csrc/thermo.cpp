// thermo.cpp -- host FP64 thermodynamics and the theoretical parameter procedure.
//
// Carnahan-Starling EOS (Eq. 28) and chemical potential (Eq. 29) with eta = b rho/4;
// critical point from dp/drho = d2p/drho2 = 0 (reduced to one equation in eta);
// Maxwell densities (equal p and mu_b, Eq. S12); Li's epsilon by the Newton /
// Simpson procedure of Appendix B (Eqs. S13, S14); continuum planar profiles of
// both models (Eq. 26, Eq. S44) for the interface width and surface tension
// (Eq. 25 and Eq. S46).  Lattice units, c_s^2 = 1/3, G = -1.
#include "thermo.h"

#include <cmath>
#include <vector>

#include "../../include/lbm.h"

namespace lbm_host {

static const double kCs2 = 1.0 / 3.0;
static const double kG = -1.0;

double CS::p(double rho, double T) const {
    const double e = 0.25 * b * rho, om = 1.0 - e;
    return rho * R * T * (1.0 + e + e * e - e * e * e) / (om * om * om) - a * rho * rho;
}

// d(rho Z)/d rho = (1 + 4e + 4e^2 - 4e^3 + e^4) / (1 - e)^4 for the C-S compressibility Z.
double CS::dp(double rho, double T) const {
    const double e = 0.25 * b * rho, om = 1.0 - e;
    const double num = 1.0 + e * (4.0 + e * (4.0 + e * (-4.0 + e)));
    return R * T * num / (om * om * om * om) - 2.0 * a * rho;
}

double CS::mu(double rho, double T) const {
    const double e = 0.25 * b * rho, om = 1.0 - e;
    const double RT = R * T;
    return RT * (3.0 - e) / (om * om * om) + RT * std::log(rho) + RT - 2.0 * a * rho;
}

// Bisection for a sign change of f on [lo, hi] down to the last representable bit.
template <class F>
static bool bisect(F f, double lo, double hi, double* root) {
    double flo = f(lo), fhi = f(hi);
    if (!(flo * fhi <= 0.0)) return false;
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = f(mid);
        if (fm == 0.0) {
            lo = hi = mid;
            break;
        }
        if ((fm < 0.0) == (flo < 0.0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    *root = 0.5 * (lo + hi);
    return true;
}

int critical(const CS& eos, double* rho_c, double* T_c, double* p_c) {
    if (!(eos.a > 0 && eos.b > 0 && eos.R > 0)) return LBM_ERR_ARG;
    // dp/drho = 0:      R T g(e) = 2 a rho,  g = (1 + 4e + 4e^2 - 4e^3 + e^4)/(1-e)^4
    // d2p/drho2 = 0:    R T (b/4) h(e) = 2 a, h = dg/de = (8 + 20e - 4e^2)/(1-e)^5
    // eliminating T:    e h(e) = g(e)
    auto q = [](double e) {
        const double g_num = 1.0 + e * (4.0 + e * (4.0 + e * (-4.0 + e)));
        return e * (8.0 + 20.0 * e - 4.0 * e * e) - (1.0 - e) * g_num;
    };
    double e;
    if (!bisect(q, 1e-6, 0.5, &e)) return LBM_ERR_NOCONVERGE;
    const double h = (8.0 + 20.0 * e - 4.0 * e * e) / std::pow(1.0 - e, 5);
    *rho_c = 4.0 * e / eos.b;
    *T_c = 8.0 * eos.a / (eos.b * eos.R * h);
    *p_c = eos.p(*rho_c, *T_c);
    return LBM_OK;
}

int maxwell(const CS& eos, double T, double* rho_v, double* rho_l, double* p0) {
    double rc, Tc, pc;
    int rc_ = critical(eos, &rc, &Tc, &pc);
    if (rc_) return rc_;
    if (!(T > 0 && T < Tc)) return LBM_ERR_ARG;
    const double top = 4.0 / eos.b * (1.0 - 1e-12);
    double s1, s2;  // spinodal densities, dp/drho = 0 below and above rho_c
    if (!bisect([&](double r) { return eos.dp(r, T); }, 1e-300, rc, &s1)) return LBM_ERR_NOCONVERGE;
    if (!bisect([&](double r) { return eos.dp(r, T); }, rc, top, &s2)) return LBM_ERR_NOCONVERGE;
    const double pmax = eos.p(s1, T);
    const double pmin = std::fmax(eos.p(s2, T), 0.0);
    bool ok = true;
    auto roots = [&](double pp, double* rv, double* rl) {
        ok &= bisect([&](double r) { return eos.p(r, T) - pp; }, 1e-300, s1, rv);
        ok &= bisect([&](double r) { return eos.p(r, T) - pp; }, s2, top, rl);
    };
    auto g = [&](double pp) {
        double rv, rl;
        roots(pp, &rv, &rl);
        return eos.mu(rl, T) - eos.mu(rv, T);
    };
    const double d = 1e-13 * pmax;
    double pstar;
    if (!bisect(g, pmin + d, pmax - d, &pstar) || !ok) return LBM_ERR_NOCONVERGE;
    roots(pstar, rho_v, rho_l);
    *p0 = pstar;
    return ok ? LBM_OK : LBM_ERR_NOCONVERGE;
}

// psi (Eq. 11 with G = -1) and its density derivative.
static inline double psi_of(const CS& eos, double r, double T) {
    return std::sqrt(2.0 * (eos.p(r, T) - kCs2 * r) / kG);
}
static inline double dpsi_of(const CS& eos, double r, double T) {
    return (eos.dp(r, T) - kCs2) / (kG * psi_of(eos, r, T));
}

// Composite Simpson rule of f on [lo, hi] with n (even) panels.
template <class F>
static double simpson(F f, double lo, double hi, int n) {
    const double h = (hi - lo) / n;
    double s = f(lo) + f(hi);
    for (int k = 1; k < n; ++k) s += (k & 1 ? 4.0 : 2.0) * f(lo + k * h);
    return s * h / 3.0;
}

int li_epsilon(const CS& eos, double T, double rv, double rl, double p0, double* eps_out) {
    // F(eps)  = int (p - p0) psi' / psi^(1+eps) d rho                  (Eq. S13)
    // F'(eps) = -int (p - p0) psi' ln(psi) / psi^(1+eps) d rho          (d/d eps of S13)
    // Newton at a given panel count, started from *eps (2 on the first level, the previous
    // level's root afterwards: one or two steps suffice once the rule is fine enough).
    auto solve = [&](int n, double* eps) {
        double e = *eps;
        for (int it = 0; it < 100; ++it) {
            // Simpson's rule in s = ln(rho) (d rho = rho ds): the integrand varies sharply near
            // the small vapour density in rho but smoothly in ln(rho).
            const double F = simpson([&](double s) {
                const double r = std::exp(s);
                return r * (eos.p(r, T) - p0) * dpsi_of(eos, r, T) / std::pow(psi_of(eos, r, T), 1.0 + e);
            }, std::log(rv), std::log(rl), n);
            const double dF = simpson([&](double s) {
                const double r = std::exp(s);
                const double ps = psi_of(eos, r, T);
                return -r * (eos.p(r, T) - p0) * dpsi_of(eos, r, T) * std::log(ps) / std::pow(ps, 1.0 + e);
            }, std::log(rv), std::log(rl), n);
            if (!(std::isfinite(F) && std::isfinite(dF)) || dF == 0.0) return false;
            const double step = -F / dF;
            e += step;
            if (std::fabs(step) < 1e-15 * std::fmax(1.0, std::fabs(e))) break;
        }
        *eps = e;
        return std::isfinite(e);
    };
    double e0 = 2.0;  // initial guess of Appendix B
    int n = 256;
    if (!solve(n, &e0)) return LBM_ERR_NOCONVERGE;
    double e1 = e0;
    for (;;) {
        n *= 2;
        if (!solve(n, &e1)) return LBM_ERR_NOCONVERGE;
        if (std::fabs(e1 - e0) < 1e-12 || n >= (1 << 20)) break;
        e0 = e1;
    }
    *eps_out = e1;
    return LBM_OK;
}

// Integrate a planar profile given (d rho/dx)^2 = A(rho) * int_{rho_v}^{rho} B(r) dr on a
// uniform density grid (cumulative trapezoid on a fine grid), then
//   width = (rho_l - rho_v)/max d rho/dx,  gamma = int C(rho) d rho/dx d rho.
template <class FA, class FB, class FC>
static void profile(double rv, double rl, FA A, FB B, FC C, double* width, double* gamma) {
    const int n = 40000;
    const double h = (rl - rv) / n;
    double inner = 0.0, bprev = B(rv), smax = 0.0, gam = 0.0, cprev = 0.0;
    for (int k = 1; k <= n; ++k) {
        const double r = rv + k * h;
        const double b = B(r);
        inner += 0.5 * h * (bprev + b);
        bprev = b;
        const double z2 = A(r) * inner;
        const double s = z2 > 0.0 ? std::sqrt(z2) : 0.0;
        if (s > smax) smax = s;
        const double c = C(r) * s;
        gam += 0.5 * h * (cprev + c);
        cprev = c;
    }
    *width = (rl - rv) / smax;
    *gamma = gam;
}

int fe_theory(const CS& eos, double T, double rv, double rl, double p0, double kappa, double* width,
              double* gamma) {
    // Eq. (26): (d rho/dx)^2 = (2 rho/kappa) int (p - p0)/rho^2; gamma = kappa int (d rho/dx) d rho.
    profile(rv, rl, [&](double r) { return 2.0 * r / kappa; },
            [&](double r) { return (eos.p(r, T) - p0) / (r * r); }, [&](double) { return kappa; }, width, gamma);
    return (std::isfinite(*width) && std::isfinite(*gamma)) ? LBM_OK : LBM_ERR_NOCONVERGE;
}

int pp_theory(const CS& eos, double T, double rv, double rl, double p0, double eps, double kP, double kLi,
              double* width, double* gamma) {
    // Eq. (S44): (psi' d rho/dx)^2 = 8 psi^eps / G * int (p0 - p)/kP psi'/psi^(1+eps)
    // Eq. (S46): gamma = -(G/6)(kP - kLi) int psi'^2 (d rho/dx) d rho
    profile(rv, rl,
            [&](double r) {
                const double d = dpsi_of(eos, r, T);
                return 8.0 * std::pow(psi_of(eos, r, T), eps) / (kG * d * d);
            },
            [&](double r) {
                return (p0 - eos.p(r, T)) / kP * dpsi_of(eos, r, T) / std::pow(psi_of(eos, r, T), 1.0 + eps);
            },
            [&](double r) {
                const double d = dpsi_of(eos, r, T);
                return -(kG / 6.0) * (kP - kLi) * d * d;
            },
            width, gamma);
    return (std::isfinite(*width) && std::isfinite(*gamma)) ? LBM_OK : LBM_ERR_NOCONVERGE;
}

// A droplet of radius r in its own vapour: mu_b(rho_v) = mu_b(rho_l) and p(rho_l) - p(rho_v) =
// gamma / r (2-D Laplace law).  Newton's method on the two residuals from the planar pair, with
// d mu_b / d rho = p'(rho) / rho (Gibbs-Duhem at constant T); converged when the Newton steps
// reach the rounding level of the residuals (1e-13 relative).
int kelvin_2d(const CS& eos, double T, double gamma, double radius, double* rho_v, double* rho_l) {
    if (!(radius > 0) || !std::isfinite(gamma) || !(*rho_v > 0) || !(*rho_l > *rho_v)) return LBM_ERR_ARG;
    double rv = *rho_v, rl = *rho_l;
    double last_v = 1.0, last_l = 1.0;  // relative size of the last Newton step
    for (int it = 0; it < 60; ++it) {
        const double f1 = eos.mu(rl, T) - eos.mu(rv, T);
        const double f2 = eos.p(rl, T) - eos.p(rv, T) - gamma / radius;
        const double pv = eos.dp(rv, T), pl = eos.dp(rl, T);
        const double j11 = -pv / rv, j12 = pl / rl, j21 = -pv, j22 = pl;
        const double det = j11 * j22 - j12 * j21;
        if (!(std::fabs(det) > 0)) return LBM_ERR_NOCONVERGE;
        const double dv = (-f1 * j22 + f2 * j12) / det, dl = (-j11 * f2 + j21 * f1) / det;
        rv += dv;
        rl += dl;
        if (!(rv > 0) || !(rl > rv)) return LBM_ERR_NOCONVERGE;
        last_v = std::fabs(dv) / rv;
        last_l = std::fabs(dl) / rl;
        if (last_v <= 1e-15 && last_l <= 1e-15) break;
    }
    // quadratic convergence ends in steps at the rounding level of the residuals
    if (!(last_v <= 1e-13 && last_l <= 1e-13)) return LBM_ERR_NOCONVERGE;
    *rho_v = rv;
    *rho_l = rl;
    return LBM_OK;
}

}  // namespace lbm_host
