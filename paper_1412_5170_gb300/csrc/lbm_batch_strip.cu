// lbm_batch_strip.cu -- the batched step with block-wide strip walks.  Each
// CTA of NT threads takes work items (instance, strip of 4*NT columns, row
// chunk) from the batch's queue and walks them one after another with the
// single-lattice strip walk (lbm_strip.cuh, the pull update of Eqs. 1-7,
// 20-23 and 34-36); the walk's row counter carries the stage barriers'
// phases from one item to the next.  Against the one-warp walk of
// 128-column items, a CTA keeps more row copies in flight per barrier wait
// and its x halo is a smaller share of a wider strip.
#include <algorithm>

#include "lbm.h"
#include "lbm_batch.cuh"
#include "lbm_strip.cuh"

namespace lbm {
namespace {

// Dynamic shared memory: the strip walk's stages, psi ring and barriers,
// then the item's constants and the item index at a 16-byte aligned offset
// (no static shared memory: it would move the dynamic region off the
// alignment the bulk copies need).
template <int NT, int NS>
constexpr size_t bstrip_coef_off() { return (strip_smem<float, float, NT, NS>() + 15) / 16 * 16; }
template <int NT, int NS>
constexpr size_t bstrip_smem() { return bstrip_coef_off<NT, NS>() + sizeof(Coef<float>) + 16; }

template <int COLL, int FORC, int NT, int NS, bool CARRY, int MINB, bool PSEAM>
__global__ void __launch_bounds__(NT, MINB)
k_step_batch_strip(const float* __restrict__ fin, float* __restrict__ fout, const BInst* __restrict__ inst,
                   const BItem* __restrict__ items, int n_items, const int* __restrict__ state,
                   unsigned* __restrict__ inst_status, int* __restrict__ queue)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (!staged_alignment_ok(smem, fin, fout)) {   // flag every instance of this launch
        for (int i = threadIdx.x; i < n_items; i += blockDim.x) atomicOr(&inst_status[items[i].inst], ST_ALIGN);
        return;
    }
    const StripSmem<float, float, NT, NS> sm(smem);
    Coef<float>* sk = reinterpret_cast<Coef<float>*>(smem + bstrip_coef_off<NT, NS>());
    int* sit = reinterpret_cast<int*>(smem + bstrip_coef_off<NT, NS>() + sizeof(Coef<float>));
    strip_init_barriers(sm);
    unsigned G = 0;
    for (;;) {
        if (threadIdx.x == 0) *sit = atomicAdd(&queue[0], 1);
        __syncthreads();
        const int it = *sit;
        if (it >= n_items) break;                           // uniform over the CTA
        const BItem w = items[it];
        const BInst* I = inst + w.inst;
        const bool run = state[w.inst] == B_RUNNING;        // no launch of the step writes state
        constexpr int nwords = sizeof(Coef<float>) / sizeof(float);
        if (run)
            for (int i = threadIdx.x; i < nwords; i += NT)
                reinterpret_cast<float*>(sk)[i] = reinterpret_cast<const float*>(&I->k)[i];
        // the constants are in place, and every thread has read the item index
        // before thread 0 takes the next one
        __syncthreads();
        if (!run) continue;
        unsigned bad = 0;
        // the walk ends with a CTA barrier, after which sk and sit may be rewritten
        const bool ok = strip_walk_step<float, float, COLL, FORC, NT, NS, CARRY, false, PSEAM>(
            fin + I->off, fout + I->off, I->nx, I->ny, w.x0, w.y0, w.y1, w.down != 0, *sk, sm, G, bad);
        flag_status(bad, &inst_status[w.inst]);
        if (!ok) break;   // a stage wait timed out: the instance is flagged, stop this CTA
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&queue[1], 1) == (int)gridDim.x - 1) {   // the last CTA done
            atomicExch(&queue[0], 0);
            atomicExch(&queue[1], 0);
        }
    }
}

template <int COLL, int FORC, int NT, int NS, bool CARRY, int MINB, bool PSEAM>
int launch_cfg(const BatchLaunch& L)
{
    constexpr size_t smem = bstrip_smem<NT, NS>();
    auto kern = k_step_batch_strip<COLL, FORC, NT, NS, CARRY, MINB, PSEAM>;
    static int per_sm = 0, nsm = 0;   // per instantiation (one device per process)
    if (per_sm == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return LBM_E_CUDA;
        int dev = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess || occ < 1) occ = 1;
        per_sm = occ;
    }
    if (L.nitems == 0) return LBM_OK;
    const int grid = std::max(1, std::min(nsm * per_sm, L.nitems));
    kern<<<grid, NT, smem, L.stream>>>(L.fin, L.fout, L.inst, L.items, L.nitems, L.state, L.status, L.queue);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}

template <int NT, int NS, bool CARRY, int MINB, bool PSEAM>
int launch_scheme(int collision, int forcing, const BatchLaunch& L)
{
    if (collision == LBM_MRT) return launch_cfg<MRT, GUO, NT, NS, CARRY, MINB, PSEAM>(L);
    if (forcing == LBM_GUO) return launch_cfg<BGK, GUO, NT, NS, CARRY, MINB, PSEAM>(L);
    if (forcing == LBM_EDM) return launch_cfg<BGK, EDM, NT, NS, CARRY, MINB, PSEAM>(L);
    if (forcing == LBM_SC) return launch_cfg<BGK, SC, NT, NS, CARRY, MINB, PSEAM>(L);
    if (forcing == LBM_LI) return launch_cfg<BGK, LI, NT, NS, CARRY, MINB, PSEAM>(L);
    return LBM_E_INVALID;
}

}  // namespace

// Most batch strips hold a whole instance row, so both halos wrap: the
// three pieces of every direction's row segment are issued one per lane.
// Register budgets: 168 per thread (6 CTAs of 64 threads, or 3 of 128, per
// SM) or 128 (4 CTAs of 128 threads; the MRT walk spills a little there).
int launch_batch_block(int columns, int stages, int collision, int forcing, const BatchLaunch& L)
{
    if (columns == 256 && stages == 3) return launch_scheme<64, 3, true, 6, true>(collision, forcing, L);
    if (columns == 512 && stages == 2) return launch_scheme<128, 2, true, 4, true>(collision, forcing, L);
    if (columns == 512 && stages == 3) return launch_scheme<128, 3, true, 3, true>(collision, forcing, L);
    return LBM_E_INVALID;
}

}  // namespace lbm
