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

// Pipelined strip kernel (lbm_strip*.cu): whether it supports p, its tuning
// configurations (threads per CTA, row stages), and one step with one of them.
struct StripConfig { int threads, stages, warp; };
bool lbm_strip_supported(const lbm_params* p);
int lbm_strip_config_count(int precision);
StripConfig lbm_strip_config(int precision, int cfg);
int lbm_strip_launch(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* status, cudaStream_t s);

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
    return k;
}
#endif  // __CUDACC__ || LBM_HOST_ARITHMETIC
