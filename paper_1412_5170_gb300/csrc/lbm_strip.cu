// lbm_strip.cu -- host dispatch of the pipelined strip kernel over precision
// and tuning configuration (see lbm_strip.cuh for the kernel).
#include "lbm_host.h"

extern const StripConfig kStripF32[];
extern const int kStripF32Count;
extern const StripConfig kPipeF32[];
extern const int kPipeF32Count;
int lbm_pipe_launch_f32(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* st, cudaStream_t s,
                        long long first_wait);
extern const StripConfig kStripF64[];
extern const int kStripF64Count;
int lbm_strip_launch_f32(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* st, cudaStream_t s,
                         long long first_wait);
int lbm_strip_launch_f64(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* st, cudaStream_t s,
                         long long first_wait);

bool lbm_strip_supported(const lbm_params* p)
{
    return p && p->nx >= 4 && p->nx % 4 == 0;
}

// FP32: the strip configurations, then the pipelined ones.
int lbm_strip_config_count(int precision)
{
    return precision == LBM_FP64 ? kStripF64Count : kStripF32Count + kPipeF32Count;
}

StripConfig lbm_strip_config(int precision, int cfg)
{
    const int n = lbm_strip_config_count(precision);
    if (cfg < 0 || cfg >= n) return StripConfig{0, 0, 0};
    if (precision == LBM_FP64) return kStripF64[cfg];
    return cfg < kStripF32Count ? kStripF32[cfg] : kPipeF32[cfg - kStripF32Count];
}

int lbm_strip_launch(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                     long long first_wait)
{
    if (!lbm_strip_supported(p)) return LBM_E_UNSUPPORTED;
    if (p->precision == LBM_FP64) return lbm_strip_launch_f64(p, cfg, fin, fout, status, s, first_wait);
    if (cfg >= kStripF32Count) return lbm_pipe_launch_f32(p, cfg - kStripF32Count, fin, fout, status, s, first_wait);
    return lbm_strip_launch_f32(p, cfg, fin, fout, status, s, first_wait);
}
