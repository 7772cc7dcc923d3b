// lbm_host.h -- host-side helpers of liblbm shared by its translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "lbm.h"
// LBM_HOST_ARITHMETIC: the per-node arithmetic compiled by a host compiler
// (a test build, with __device__ and __forceinline__ defined beforehand)
#if defined(__CUDACC__) || defined(LBM_HOST_ARITHMETIC)
#include "lbm_device.cuh"
#endif

extern "C" {
double lbm_tc(void);
int lbm_maxwell(double T_over_Tc, double* rho_v, double* rho_l);
}

// LBM_OK or LBM_E_INVALID / LBM_E_UNSUPPORTED for a parameter set.
int lbm_validate_params(const lbm_params* p);

// Initial density field of lbm_init_preset (row-major ny*nx).
int lbm_preset_field(int nx, int ny, int kind, double size, double width, double rho_l, double rho_v,
                     int32_t cell, uint64_t seed, double noise_amp, std::vector<double>& out);

// Polls of a bounded stage wait (mbarrier try_wait) before the staged kernels
// declare a row copy stuck, flag a timeout, drain and return.
constexpr long long kStageWaitPolls = 1ll << 26;

// Pipelined strip kernel (lbm_strip*.cu): whether it supports p, its tuning
// configurations (threads per CTA, row stages), and one step with one of them.
// first_wait: polls of each CTA's first stage wait (the others make
// kStageWaitPolls); 0 makes that wait give up at once, as a stuck copy would
// (the failure-detection test of the timeout path).
struct StripConfig { int threads, stages, warp; };
bool lbm_strip_supported(const lbm_params* p);
int lbm_strip_config_count(int precision);
StripConfig lbm_strip_config(int precision, int cfg);
int lbm_strip_launch(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                     long long first_wait = kStageWaitPolls);

#if defined(__CUDACC__) || defined(LBM_HOST_ARITHMETIC)
// Kernel constants of a parameter set in the compute type C.
template <typename C>
lbm::Coef<C> make_coef(const lbm_params& p)
{
    lbm::Coef<C> k;
    k.T = C(p.T_over_Tc * lbm_tc());
    k.K = C(p.K);
    k.half_A = C(0.5 * p.A);
    k.one_m_A = C(1.0 - p.A);
    k.omega = C(1.0 / p.tau);
    k.tau = C(p.tau);
    k.guo_pre = C(1.0 - 0.5 / p.tau);
    k.s_e = C(p.s_e);
    k.s_eps = C(p.s_eps);
    k.s_q = C(p.s_q);
    k.rho_ref = C(p.precision == LBM_FP64 ? 0.0 : p.rho_ref);
    k.li_c = C(p.forcing == LBM_LI ? p.sigma / (p.tau - 0.5) : 0.0);
    const double rate[4] = {p.s_e, p.s_eps, p.s_q, 1.0 / p.tau};
    const double norm[4] = {36.0, 36.0, 12.0, 4.0};
    for (int i = 0; i < 4; ++i) {
        k.r0[i] = C((1.0 - rate[i]) / norm[i]);
        k.r1[i] = C(rate[i] / norm[i]);
        k.r2[i] = C((1.0 - 0.5 * rate[i]) / norm[i]);
    }
    // FP32: omega and Guo's 1 - omega/2 both exact floats (omega moved by at
    // most one ulp of 1 - omega/2 where needed), so that the momentum a step
    // adds, omega F/2 + (1 - omega/2) F, is exactly F; the Shan-Chen shift
    // tau = 1/omega as hi + lo.
    k.A = C(p.A);
    k.tau_lo = C(0);
    k.h_e = C(1.0f - 0.5f * float(p.s_e));
    k.h_eps = C(1.0f - 0.5f * float(p.s_eps));
    k.h_q = C(1.0f - 0.5f * float(p.s_q));
    if (p.precision != LBM_FP64) {
        float om = float(1.0 / p.tau);
        float gp = float(1.0 - 0.5 * double(om));
        if (double(gp) != 1.0 - 0.5 * double(om)) om = float(2.0 * (1.0 - double(gp)));
        k.omega = C(om);
        k.guo_pre = C(gp);
        const double t = 1.0 / double(om);
        k.tau = C(t);
        k.tau_lo = C(t - double(k.tau));
    }
    return k;
}
#endif  // __CUDACC__ || LBM_HOST_ARITHMETIC
