// lbm_strip_f32.cu -- FP32-deviation instantiations of the strip kernel.
// Configurations (threads per CTA NT -> 4*NT-column strips, NS row stages):
// the autotuner picks among them per lattice.
#include "lbm_warp.cuh"

using namespace lbm;

// {threads, stages, warp}: warp = 1 selects the warp-per-strip kernel
// (lbm_warp.cuh) re-reading rows from shared memory, warp = 2 the one that
// keeps them in registers.
extern const StripConfig kStripF32[] = {{32, 3, 1}, {32, 4, 1}, {32, 3, 2}, {64, 3, 0}, {128, 3, 0}, {128, 4, 0}};
extern const int kStripF32Count = sizeof(kStripF32) / sizeof(kStripF32[0]);

int lbm_strip_launch_f32(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* st, cudaStream_t s)
{
    switch (cfg) {
    case 0: return launch_warp_scheme<3, false>(p, fin, fout, st, s);
    case 1: return launch_warp_scheme<4, false>(p, fin, fout, st, s);
    case 2: return launch_warp_scheme<3, true>(p, fin, fout, st, s);
    case 3: return launch_strip_scheme<float, float, 64, 3>(p, fin, fout, st, s);
    case 4: return launch_strip_scheme<float, float, 128, 3>(p, fin, fout, st, s);
    case 5: return launch_strip_scheme<float, float, 128, 4>(p, fin, fout, st, s);
    default: return LBM_E_INVALID;
    }
}
