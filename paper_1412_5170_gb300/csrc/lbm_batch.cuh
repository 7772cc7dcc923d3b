// lbm_batch.cuh -- records shared by the batched step's two walks: the
// per-instance constants, the work items (instance, strip, row chunk) and
// the instance states, plus the launcher of the block-wide walk.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

struct BInst {
    long long off;        // population element offset (both buffers)
    long long node_off;   // node offset of the FP64 per-node arrays
    int nx, ny;
    int tile_off;         // first observe tile (32 x 8) of this instance
    int ntx, nty;
    int kind;             // lbm_preset of the instance's geometry
    int cell;
    double size, width, rho_l, rho_v, noise_amp;
    unsigned long long seed;
    Coef<float> k;
};
// One work item: rows [y0, y1) of the strip of columns starting at x0 of
// instance inst; down: walk the chunk's rows downwards.
struct BItem { int inst, x0, y0, y1, down, pad[3]; };

enum : int { B_RUNNING = 0, B_CONVERGED = 1, B_FAILED = 2 };

// Arguments of one batched-step launch.  queue: the work-item counter and
// the done counter, both zero between launches.
struct BatchLaunch {
    const float* fin;
    float* fout;
    const BInst* inst;
    const BItem* items;
    int nitems;
    const int* state;
    unsigned* status;   // per instance
    int* queue;
    cudaStream_t stream;
};

// The batched step with block-wide strip walks of `columns` columns and
// `stages` carried row stages (256: 64-thread CTAs, 3 stages; 512: 128-thread
// CTAs, 2 or 3 stages).  collision, forcing: lbm_collision, lbm_forcing (Guo,
// EDM or SC forcing under BGK; Guo under MRT).  Returns LBM_E_INVALID for
// another shape.
int launch_batch_block(int columns, int stages, int collision, int forcing, const BatchLaunch& L);

}  // namespace lbm
