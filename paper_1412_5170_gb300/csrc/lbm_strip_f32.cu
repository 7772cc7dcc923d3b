// lbm_strip_f32.cu -- FP32-deviation instantiations of the strip kernel.
// Configurations (threads per CTA NT -> 4*NT-column strips, NS row stages):
// the autotuner picks among them per lattice.
#include "lbm_warp.cuh"

using namespace lbm;

// {threads, stages, kind}: kind 1 / 2 select the warp-per-strip kernel
// (lbm_warp.cuh) re-reading rows from shared memory / keeping them in
// registers; kind 0 / 3 the block-strip kernel (lbm_strip.cuh) likewise;
// kind 4 the register-carrying block strip held to 128 registers so that
// 16 warps share an SM (4 CTAs of 128 threads or 2 of 256).
extern const StripConfig kStripF32[] = {{128, 3, 3}, {64, 3, 3}, {64, 4, 3}, {128, 4, 3},
                                        {32, 3, 1}, {32, 4, 1}, {128, 3, 0}, {128, 2, 4}, {256, 2, 4}, {512, 2, 4},
                                        {128, 3, 3}, {256, 2, 4}};
extern const int kStripF32Count = sizeof(kStripF32) / sizeof(kStripF32[0]);

int lbm_strip_launch_f32(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* st, cudaStream_t s,
                        long long fw)
{
    switch (cfg) {
    // The last template argument is the CTAs per SM the shared memory of the
    // configuration allows; the register budget is held to match it.
    case 0: return launch_strip_scheme<float, float, 128, 3, true, 3>(p, fin, fout, st, s, fw);
    case 1: return launch_strip_scheme<float, float, 64, 3, true, 6>(p, fin, fout, st, s, fw);
    case 2: return launch_strip_scheme<float, float, 64, 4, true, 5>(p, fin, fout, st, s, fw);
    case 3: return launch_strip_scheme<float, float, 128, 4, true, 2>(p, fin, fout, st, s, fw);
    case 4: return launch_warp_scheme<3, false>(p, fin, fout, st, s, fw);
    case 5: return launch_warp_scheme<4, false>(p, fin, fout, st, s, fw);
    case 6: return launch_strip_scheme<float, float, 128, 3, false, 3>(p, fin, fout, st, s, fw);
    // Template tail: CTAs per SM, left halo psi on thread 32 (else 0), seam copies one per lane.
    // Each was kept for being the fastest of its tile shape on the 4096^2 workload.
    case 7: return launch_strip_scheme<float, float, 128, 2, true, 4, false, true>(p, fin, fout, st, s, fw);
    case 8: return launch_strip_scheme<float, float, 256, 2, true, 2, false, false>(p, fin, fout, st, s, fw);
    case 9: return launch_strip_scheme<float, float, 512, 2, true, 1, false, true>(p, fin, fout, st, s, fw);
    case 10: return launch_strip_scheme<float, float, 128, 3, true, 3, true, false>(p, fin, fout, st, s, fw);
    case 11: return launch_strip_scheme<float, float, 256, 2, true, 2, true, true>(p, fin, fout, st, s, fw);
    default: return LBM_E_INVALID;
    }
}
