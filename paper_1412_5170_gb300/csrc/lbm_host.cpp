// lbm_host.cpp -- host FP64 helpers of liblbm: critical temperature, Maxwell
// coexistence densities, parameter validation and built-in initial fields.
#include "lbm_host.h"

#include <cmath>
#include <limits>

namespace {

// Carnahan-Starling EOS of Eq. 29 with a = 1, b = 4, R = 1 (eta = rho), K = 1.
double cs_p(double r, double T) { return r * T * (1 + r + r * r - r * r * r) / ((1 - r) * (1 - r) * (1 - r)) - r * r; }
double cs_dp(double r, double T)
{
    const double q = 1 - r;
    return T * (1 + 4 * r + 4 * r * r - 4 * r * r * r + r * r * r * r) / (q * q * q * q) - 2 * r;
}
// Chemical potential mu = a + p/rho with the CS Helmholtz energy per particle
// a = T ln rho + T rho (4 - 3 rho)/(1 - rho)^2 - rho.  Equal p and mu at the two
// densities is the equal-area rule of Eq. 19.
double cs_mu(double r, double T) { return T * std::log(r) + T * r * (4 - 3 * r) / ((1 - r) * (1 - r)) - r + cs_p(r, T) / r; }

template <typename F>
double bisect(F f, double lo, double hi, int iters = 200)
{
    double flo = f(lo);
    for (int i = 0; i < iters; ++i) {
        const double mid = 0.5 * (lo + hi);
        const double fm = f(mid);
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
    }
    return 0.5 * (lo + hi);
}

uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

}  // namespace

extern "C" double lbm_tc(void)
{
    // a = 0.4963 R^2 Tc^2/pc, b = 0.18727 R Tc/pc  =>  Tc = (0.18727/0.4963) a/(b R).
    return (0.18727 / 0.4963) * 1.0 / (4.0 * 1.0);
}

namespace {

// Spinodal densities s1 < s2 of the CS isotherm at temperature T (dp/drho
// changes sign + -> - at s1 and - -> + at s2); false if there are none.
bool spinodals(double T, double& s1, double& s2)
{
    const int N = 20000;
    double prev = cs_dp(1e-6, T), rprev = 1e-6;
    s1 = s2 = -1;
    for (int i = 1; i <= N && s2 < 0; ++i) {
        const double r = 1e-6 + (0.95 - 1e-6) * i / N;
        const double d = cs_dp(r, T);
        if (s1 < 0 && prev > 0 && d <= 0) s1 = bisect([&](double x) { return cs_dp(x, T); }, rprev, r);
        else if (s1 > 0 && prev < 0 && d >= 0) s2 = bisect([&](double x) { return cs_dp(x, T); }, rprev, r);
        prev = d;
        rprev = r;
    }
    return s1 > 0 && s2 > 0;
}

// Gas and liquid densities at which the CS isotherm (scaled by K, which moves
// no root) reaches the pressure K * pc_unit.
void branches(double T, double s1, double s2, double pc_unit, double& rg, double& rl)
{
    const double lg = bisect([&](double l) { return cs_p(std::exp(l), T) - pc_unit; }, std::log(1e-30), std::log(s1));
    rg = std::exp(lg);
    rl = bisect([&](double r) { return cs_p(r, T) - pc_unit; }, s2, 1.0 - 1e-12);
}

// 8-point Gauss-Legendre nodes and weights on [-1, 1].
const double kGLx[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                        0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
const double kGLw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                        0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

// int_a^b g(rho) d rho over n intervals uniform in log rho (composite 8-point
// Gauss-Legendre in l = ln rho, d rho = rho dl).
template <typename G>
double integrate_log(G g, double a, double b, int n = 400)
{
    const double la = std::log(a), h = (std::log(b) - la) / n;
    double sum = 0;
    for (int i = 0; i < n; ++i) {
        const double c = la + (i + 0.5) * h;
        for (int j = 0; j < 8; ++j) {
            const double r = std::exp(c + 0.5 * h * kGLx[j]);
            sum += kGLw[j] * g(r) * r;
        }
    }
    return 0.5 * h * sum;
}

}  // namespace

extern "C" int lbm_mechanical(double T_over_Tc, double K, double eps, double* rho_v, double* rho_l)
{
    if (!rho_v || !rho_l || !(T_over_Tc > 0.05 && T_over_Tc < 1.0) || !finite_pos(K) || !std::isfinite(eps))
        return LBM_E_INVALID;
    const double T = T_over_Tc * lbm_tc();
    double s1, s2;
    if (!spinodals(T, s1, s2)) return LBM_E_INVALID;
    // Eq. 18 with p0 = K p_CS (Eq. 30) and, from Eq. 7 with G = -1,
    // psi^2 = 2 (rho/3 - p0), so psi' / psi^(1+eps) = (1/3 - p0') / psi^(2+eps).
    auto mech = [&](double pc_unit) {
        double rg, rl;
        branches(T, s1, s2, pc_unit, rg, rl);
        const double pc = K * pc_unit;
        return integrate_log([&](double r) {
            const double p0 = K * cs_p(r, T);
            const double psi2 = 2.0 * (r / 3.0 - p0);
            return (pc - p0) * (1.0 / 3.0 - K * cs_dp(r, T)) / std::pow(psi2, 1.0 + 0.5 * eps);
        }, rg, rl);
    };
    const double p_hi = cs_p(s1, T);
    const double p_lo = std::fmax(cs_p(s2, T), 0.0);
    const double lo = p_lo > 0 ? p_lo * (1 + 1e-12) : p_hi * 1e-14;
    const double hi = p_hi * (1 - 1e-14);
    const double flo = mech(lo), fhi = mech(hi);
    if (!std::isfinite(flo) || !std::isfinite(fhi) || (flo < 0) == (fhi < 0)) return LBM_E_INVALID;
    const double pc = bisect(mech, lo, hi, 120);
    double rg, rl;
    branches(T, s1, s2, pc, rg, rl);
    *rho_v = rg;
    *rho_l = rl;
    return LBM_OK;
}

extern "C" int lbm_maxwell(double T_over_Tc, double* rho_v, double* rho_l)
{
    if (!rho_v || !rho_l || !(T_over_Tc > 0.05 && T_over_Tc < 1.0)) return LBM_E_INVALID;
    const double T = T_over_Tc * lbm_tc();
    // Spinodals: dp/drho changes sign + -> - at s1 and - -> + at s2.
    const int N = 20000;
    double s1 = -1, s2 = -1, prev = cs_dp(1e-6, T), rprev = 1e-6;
    for (int i = 1; i <= N && s2 < 0; ++i) {
        const double r = 1e-6 + (0.95 - 1e-6) * i / N;
        const double d = cs_dp(r, T);
        if (s1 < 0 && prev > 0 && d <= 0) s1 = bisect([&](double x) { return cs_dp(x, T); }, rprev, r);
        else if (s1 > 0 && prev < 0 && d >= 0) s2 = bisect([&](double x) { return cs_dp(x, T); }, rprev, r);
        prev = d;
        rprev = r;
    }
    if (s1 < 0 || s2 < 0) return LBM_E_INVALID;
    const double p_hi = cs_p(s1, T);
    const double p_lo = std::fmax(cs_p(s2, T), 0.0);
    auto branches = [&](double pc, double& rg, double& rl) {
        // gas: p increasing on (0, s1); bisect in log rho
        const double lg = bisect([&](double l) { return cs_p(std::exp(l), T) - pc; }, std::log(1e-30), std::log(s1));
        rg = std::exp(lg);
        rl = bisect([&](double r) { return cs_p(r, T) - pc; }, s2, 1.0 - 1e-12);
    };
    auto dmu = [&](double pc) {
        double rg, rl;
        branches(pc, rg, rl);
        return cs_mu(rl, T) - cs_mu(rg, T);
    };
    const double lo = p_lo > 0 ? p_lo * (1 + 1e-12) : p_hi * 1e-14;
    const double pc = bisect(dmu, lo, p_hi * (1 - 1e-14));
    double rg, rl;
    branches(pc, rg, rl);
    *rho_v = rg;
    *rho_l = rl;
    return LBM_OK;
}

int lbm_validate_params(const lbm_params* p)
{
    if (!p) return LBM_E_INVALID;
    if (p->nx < 1 || p->ny < 1 || (int64_t)p->nx * p->ny > (int64_t)std::numeric_limits<int32_t>::max()) return LBM_E_INVALID;
    if (!(p->T_over_Tc > 0 && p->T_over_Tc < 1)) return LBM_E_INVALID;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return LBM_E_INVALID;
    if (!finite_pos(p->K) || !std::isfinite(p->A)) return LBM_E_INVALID;
    if (p->collision != LBM_BGK && p->collision != LBM_MRT) return LBM_E_INVALID;
    if (p->forcing < LBM_GUO || p->forcing > LBM_LI) return LBM_E_INVALID;
    if (!std::isfinite(p->sigma)) return LBM_E_INVALID;
    if (p->forcing == LBM_LI) {
        // Li et al.'s model: BGK collision, the Eq. 4 force (Eq. 6 with A = 0), sigma >= 0
        if (p->collision != LBM_BGK) return LBM_E_UNSUPPORTED;
        if (p->A != 0.0 || !(p->sigma >= 0.0)) return LBM_E_INVALID;
    } else if (p->sigma != 0.0) {
        return LBM_E_INVALID;
    }
    if (p->precision != LBM_FP64 && p->precision != LBM_FP32_DEV) return LBM_E_INVALID;
    if (p->reserved != 0) return LBM_E_INVALID;
    if (p->collision == LBM_MRT) {
        if (p->forcing != LBM_GUO) return LBM_E_UNSUPPORTED;
        for (double s : {p->s_e, p->s_eps, p->s_q})
            if (!(s > 0 && s < 2)) return LBM_E_INVALID;
    }
    if (p->precision == LBM_FP32_DEV && !(std::isfinite(p->rho_ref) && p->rho_ref >= 0)) return LBM_E_INVALID;
    return LBM_OK;
}

int lbm_preset_field(int nx, int ny, int kind, double size, double width, double rho_l, double rho_v,
                     int32_t cell, uint64_t seed, double noise_amp, std::vector<double>& out)
{
    if (nx < 1 || ny < 1 || !(width > 0) || !std::isfinite(size)) return LBM_E_INVALID;
    if (kind < LBM_SLAB || kind > LBM_DROPLET_ARRAY) return LBM_E_INVALID;
    if (kind == LBM_DROPLET_ARRAY && cell < 1) return LBM_E_INVALID;
    out.assign((size_t)nx * ny, 0.0);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double d;
            if (kind == LBM_SLAB) {
                d = std::fabs(y - ny / 2.0) - size;
            } else if (kind == LBM_DROPLET_ARRAY) {
                const double cx = std::floor(double(x) / cell) * cell + cell / 2.0;
                const double cy = std::floor(double(y) / cell) * cell + cell / 2.0;
                d = std::hypot(x - cx, y - cy) - size;
            } else {
                d = std::hypot(x - nx / 2.0, y - ny / 2.0) - size;
            }
            const double inside = 0.5 * (1.0 - std::tanh(2.0 * d / width));
            double r = (kind == LBM_BUBBLE) ? rho_l + (rho_v - rho_l) * inside : rho_v + (rho_l - rho_v) * inside;
            if (noise_amp != 0.0) {
                const uint64_t z = splitmix64(seed ^ (uint64_t)((size_t)y * nx + x));
                const double xi = double(z >> 11) * (1.0 / 9007199254740992.0);
                r += noise_amp * (2.0 * xi - 1.0);
            }
            out[(size_t)y * nx + x] = r;
        }
    return LBM_OK;
}
