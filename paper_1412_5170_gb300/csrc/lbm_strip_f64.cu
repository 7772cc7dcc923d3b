// lbm_strip_f64.cu -- FP64 instantiations of the strip kernel (the parity
// path; its step is bound by double-precision arithmetic on GB300).
#include "lbm_strip.cuh"

using namespace lbm;

extern const StripConfig kStripF64[] = {{64, 4, 0}, {32, 6, 0}, {64, 3, 0}};
extern const int kStripF64Count = sizeof(kStripF64) / sizeof(kStripF64[0]);

int lbm_strip_launch_f64(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* st, cudaStream_t s,
                        long long fw)
{
    switch (cfg) {
    case 0: return launch_strip_scheme<double, double, 64, 4>(p, fin, fout, st, s, fw);
    case 1: return launch_strip_scheme<double, double, 32, 6>(p, fin, fout, st, s, fw);
    case 2: return launch_strip_scheme<double, double, 64, 3>(p, fin, fout, st, s, fw);
    default: return LBM_E_INVALID;
    }
}
