// lbm_pipe_f32.cu -- FP32-deviation instantiations of the pipelined strip
// kernel (lbm_pipe.cuh: warps synchronised only through the stage ring).
// Configurations {threads, stages, kind 5}, appended to the strip table's ids.
#include "lbm_pipe.cuh"

using namespace lbm;

extern const StripConfig kPipeF32[] = {{256, 2, 5}, {512, 2, 5}, {128, 3, 5}, {128, 2, 5}};
extern const int kPipeF32Count = sizeof(kPipeF32) / sizeof(kPipeF32[0]);

int lbm_pipe_launch_f32(const lbm_params* p, int cfg, const void* fin, void* fout, unsigned* st, cudaStream_t s,
                        long long fw)
{
    switch (cfg) {
    // Template tail: CTAs per SM that the shared memory allows (the register
    // budget is held to it), seam copies one per lane.
    case 0: return launch_pipe_scheme<float, float, 256, 2, 2, false>(p, fin, fout, st, s, fw);
    case 1: return launch_pipe_scheme<float, float, 512, 2, 1, true>(p, fin, fout, st, s, fw);
    case 2: return launch_pipe_scheme<float, float, 128, 3, 3, false>(p, fin, fout, st, s, fw);
    case 3: return launch_pipe_scheme<float, float, 128, 2, 4, true>(p, fin, fout, st, s, fw);
    default: return LBM_E_INVALID;
    }
}
