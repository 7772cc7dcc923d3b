// lbm_pipe.cuh -- the strip walk with warps that do not wait for one another.
//
// Same data path as lbm_strip.cuh: a CTA of NT threads owns a strip of
// W = 4*NT columns and a chunk of rows; the nine row segments of each walk
// row (source row r - e_y(a), columns x0-4 .. x0+W+4) arrive by
// cp.async.bulk (TMA bulk copies) in a ring of NS shared-memory stages, one
// mbarrier per stage; a lane owns 4 columns and pulls them with 128-bit
// shared loads and shuffles.  What differs is the synchronisation.  In the
// strip walk every row ends at a CTA barrier, because the psi stencil of a
// warp's edge columns reads psi computed by the neighbouring warps.  Here
// every warp computes psi of its own two halo columns as well (from the same
// stage; they are its neighbours' edge columns) into a psi ring of its own,
// so the only thing the warps share is the stage ring:
//   - a warp waits for a row's stage on its mbarrier (bounded, as before);
//   - once it has pulled the row into registers it counts itself done with
//     the stage (an atomic counter per stage in shared memory), and the warp
//     that completes the count refills the stage with the row NS further on.
// A warp can thus run ahead of the slowest one by the rows already in the
// ring, and no warp idles at a barrier while another finishes its row.
//
// Walk iteration k (one warp): wait for stage k; pull row k (carried in
// registers to the next iteration); psi of row k's columns and of the
// warp's two halo columns into its ring; count the stage done (the last
// warp refills it with row k + NS); hand row k-1 -- its pulled populations
// and psi rows k-2, k-1, k -- to the row functor (StepRow: force, collision,
// 128-bit stores; ObsRow: the observables).  Rows 0 and H+1 of the walk are
// the halo rows before and after the chunk.
#pragma once
#include <cuda_runtime.h>

#include "lbm_strip.cuh"

namespace lbm {

// Shared memory of a pipelined strip CTA: NS stages [9][W+8] of T, one psi
// ring [4][136] of C per warp (column c of the warp's 128 at index 4 + c, its
// halo columns at 3 and 4 + its width), NS mbarriers, NS stage counters, and
// the number of walk rows every warp is done with.
template <typename T, typename C, int NT, int NS>
struct PipeSmem {
    static constexpr int W = 4 * NT;
    static constexpr int NW = NT / 32;
    static constexpr int SW = W + 8;     // stage row stride (elements)
    static constexpr int PW = 136;       // psi ring row stride (elements)
    static constexpr size_t kStages = sizeof(T) * NS * 9 * SW;
    static constexpr size_t kRing = sizeof(C) * NW * 4 * PW;
    static constexpr size_t bytes() { return kStages + kRing + 8 * NS + 4 * NS + 16; }
    T* stages;
    C* psi;
    uint64_t* bars;
    int* count;
    int* done;
    __device__ explicit PipeSmem(unsigned char* smem)
        : stages(reinterpret_cast<T*>(smem)),
          psi(reinterpret_cast<C*>(smem + kStages)),
          bars(reinterpret_cast<uint64_t*>(smem + kStages + kRing)),
          count(reinterpret_cast<int*>(smem + kStages + kRing + 8 * NS)),
          done(reinterpret_cast<int*>(smem + kStages + kRing + 12 * NS)) {}
};

template <typename T, typename C, int NT, int NS>
__device__ __forceinline__ void pipe_init(const PipeSmem<T, C, NT, NS>& sm)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&sm.bars[s], 1);
            sm.count[s] = 0;
        }
        *sm.done = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

// Walk one strip segment: columns [x0, x0 + min(W, nx - x0)), rows [y0, y1),
// as strip_walk (same G, down and first_wait conventions; the pulled rows are
// carried).  Returns false (ST_TIMEOUT in bad) if a stage wait gave up; the
// copies still in flight are drained (bounded) before it returns.  All
// threads of the CTA call it with the same arguments; it ends with a CTA
// barrier.
template <typename T, typename C, int NT, int NS, bool PSEAM, class Row>
__device__ __forceinline__ bool pipe_walk(const T* __restrict__ fin, int nx, int ny, int x0, int y0, int y1,
                                          bool down, const Coef<C>& k, const PipeSmem<T, C, NT, NS>& sm,
                                          unsigned& G, unsigned& bad, Row& row, long long first_wait = kWaitLimit)
{
    using SM = PipeSmem<T, C, NT, NS>;
    constexpr int SW = SM::SW, PW = SM::PW, NW = SM::NW;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int wp = min(SM::W, nx - x0);                      // strip width (multiple of 4)
    const int H = y1 - y0;
    const size_t n = (size_t)nx * ny;
    const int nrows = H + 2;                                 // walk rows incl. 2 halo rows
    const unsigned stage_bytes = unsigned(9 * (wp + 8) * sizeof(T));
    const bool left_wrap = x0 == 0, right_wrap = x0 + wp == nx;
    const unsigned base = G;
    const int cw = 128 * w;                                  // the warp's first column
    const int wpw = max(0, min(128, wp - cw));               // the warp's width (0: idle warp)
    const int c0 = cw + 4 * lane;
    const bool active = c0 < wp;
    const bool lsm = lane == 0, rsm = (lane == 31) || (c0 + 4 == wp);   // pulled neighbours from the stage
    C* const ring = sm.psi + w * 4 * PW;

    // The calling warp issues the nine segment copies of walk row kr into its
    // stage, one per lane; at the periodic seam each splits in three, issued
    // by the same lane or, with PSEAM, by three lanes.
    auto issue = [&](int kr) {
        const unsigned g = base + kr;
        uint64_t* bar = &sm.bars[g % NS];
        T* st = sm.stages + (g % NS) * 9 * SW;
        if (lane == 0) mbar_arrive_expect_tx(bar, stage_bytes);
        __syncwarp();
        const bool seam = left_wrap || right_wrap;
        if (PSEAM && seam) {
            if (lane < 27) {
                fence_proxy_async();   // order earlier generic reads of this slot before the async writes
                const int a = lane / 3, piece = lane - 3 * a;
                const int r = wrap_any((down ? y1 - kr : y0 - 1 + kr) - ey(a), ny);
                const T* src = fin + a * n + (size_t)r * nx;
                T* dst = st + a * SW;
                if (piece == 0) bulk_g2s(dst, src + (left_wrap ? nx - 4 : x0 - 4), unsigned(4 * sizeof(T)), bar);
                else if (piece == 1) bulk_g2s(dst + 4, src + x0, unsigned(wp * sizeof(T)), bar);
                else bulk_g2s(dst + 4 + wp, src + (right_wrap ? 0 : x0 + wp), unsigned(4 * sizeof(T)), bar);
            }
        } else if (lane < 9) {
            fence_proxy_async();
            const int a = lane;
            const int r = wrap_any((down ? y1 - kr : y0 - 1 + kr) - ey(a), ny);
            const T* src = fin + a * n + (size_t)r * nx;
            T* dst = st + a * SW;
            if (!seam) {
                bulk_g2s(dst, src + x0 - 4, unsigned((wp + 8) * sizeof(T)), bar);
            } else {
                bulk_g2s(dst, src + (left_wrap ? nx - 4 : x0 - 4), unsigned(4 * sizeof(T)), bar);
                bulk_g2s(dst + 4, src + x0, unsigned(wp * sizeof(T)), bar);
                bulk_g2s(dst + 4 + wp, src + (right_wrap ? 0 : x0 + wp), unsigned(4 * sizeof(T)), bar);
            }
        }
    };

    if (w == 0)
        for (int kr = 0; kr < NS && kr < nrows; ++kr) issue(kr);

    bool ok_all = true;
    C gA[9][4], gB[9][4];

    auto body = [&](int kk, C (&gn)[9][4], C (&gc)[9][4]) -> bool {
        const unsigned g = base + kk;
        const int s = g % NS;
        const T* st = sm.stages + s * 9 * SW;
        if (!__all_sync(0xffffffffu, mbar_wait(&sm.bars[s], (g / NS) & 1, kk == 0 ? first_wait : kWaitLimit)))
            return false;
        pull4_shfl<T, C>(st, SW, c0, lsm, rsm, gn);
        C* prow = ring + (kk & 3) * PW;
        // psi of the warp's two halo columns (its neighbours' edge columns):
        // lane 0 the left one, lane 31 the right one, side by side
        if (wpw > 0 && (lane == 0 || lane == 31)) {
            const int ch = lane == 0 ? cw - 1 : cw + wpw;
            prow[lane == 0 ? 3 : 4 + wpw] = psi_of_rho<C>(k.rho_ref + drho1<T, C>(st, SW, ch), k, bad);
        }
        // the warp is done reading the stage: count it; the last warp refills it
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&sm.count[s], 1) == NW - 1;
            if (last) {
                sm.count[s] = 0;
                *sm.done = kk + 1;   // every warp has pulled rows 0..kk
                __threadfence_block();
            }
        }
        if (__shfl_sync(0xffffffffu, last, 0) && kk + NS < nrows) issue(kk + NS);
        if (wpw > 0) {
            C ps[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                C s9[9];
#pragma unroll
                for (int a = 0; a < 9; ++a) s9[a] = gn[a][j];
                unsigned b = 0;
                ps[j] = psi_of_rho<C>(k.rho_ref + sum9(s9), k, b);
                if (active) bad |= b;
            }
            if (active) sts4(prow + 4 + 4 * lane, ps);
        }
        __syncwarp();
        const int kc = kk - 1;                               // hand over walk row kk-1
        if (kc >= 1 && kc <= H && wpw > 0) {                 // warp-uniform
            C rm[6], r0[6], rp[6];                           // psi at columns c0-1 .. c0+4 of rows y-1, y, y+1
            const int l4 = 4 * lane;
            psi_row6<C>(ring + ((down ? kc + 1 : kc - 1) & 3) * PW, l4, lsm, rsm, rm);
            psi_row6<C>(ring + (kc & 3) * PW, l4, lsm, rsm, r0);
            psi_row6<C>(ring + ((down ? kc - 1 : kc + 1) & 3) * PW, l4, lsm, rsm, rp);
            row(down ? y1 - kc : y0 + kc - 1, x0 + c0, active, gc, rm, r0, rp, k, bad);
        }
        return true;
    };

    for (int kk = 0; kk < nrows; kk += 2) {
        if (!body(kk, gA, gB)) { ok_all = false; break; }
        if (kk + 1 < nrows && !body(kk + 1, gB, gA)) { ok_all = false; break; }
    }
    __syncthreads();   // every warp has left the walk (each of its waits is bounded)
    if (!ok_all) bad |= ST_TIMEOUT;
    const int done = *sm.done;
    if (done < nrows) {
        // A wait gave up somewhere: rows [done, done + NS) may have copies in
        // flight (a row is issued only once every warp has pulled the row NS
        // before it); wait for them (bounded) before the CTA goes on or exits.
        if (t == 0)
            for (int kr = done; kr < done + NS && kr < nrows; ++kr)
                mbar_wait(&sm.bars[(base + kr) % NS], ((base + kr) / NS) & 1);
        __syncthreads();
        return false;
    }
    G = base + nrows;
    if (t == 0) *sm.done = 0;
    __syncthreads();
    return true;
}

// One lattice, grid (strips, row chunks), as k_step_strip.
template <typename T, typename C, int COLL, int FORC, int NT, int NS, int MINB, bool PSEAM>
__global__ void __launch_bounds__(NT, MINB)
k_step_pipe(const T* __restrict__ fin, T* __restrict__ fout, int nx, int ny, int nchunks, Coef<C> k,
            unsigned* __restrict__ status, long long first_wait)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (!staged_alignment_ok(smem, fin, fout)) {
        if (threadIdx.x == 0) atomicOr(status, ST_ALIGN);
        return;
    }
    const PipeSmem<T, C, NT, NS> sm(smem);
    const int x0 = blockIdx.x * (4 * NT);
    const int y0 = int((long long)blockIdx.y * ny / nchunks);
    const int y1 = int((long long)(blockIdx.y + 1) * ny / nchunks);
    if (y1 <= y0) return;
    pipe_init(sm);
    unsigned G = 0, bad = 0;
    StepRow<T, C, COLL, FORC> row{fout, nx, (size_t)nx * ny};
    pipe_walk<T, C, NT, NS, PSEAM>(fin, nx, ny, x0, y0, y1, (blockIdx.y & 1) != 0, k, sm, G, bad, row, first_wait);
    flag_status(bad, status);
}

template <typename T, typename C, int COLL, int FORC, int NT, int NS, int MINB, bool PSEAM>
int launch_pipe_cfg(const lbm_params* p, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                    long long first_wait)
{
    constexpr size_t smem = PipeSmem<T, C, NT, NS>::bytes();
    auto kern = k_step_pipe<T, C, COLL, FORC, NT, NS, MINB, PSEAM>;
    static int per_sm = 0, nsm = 0;    // per instantiation (one device per process)
    if (per_sm == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return LBM_E_CUDA;
        int dev = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess || occ < 1) occ = 1;
        per_sm = occ;
    }
    const int W = 4 * NT;
    const int nstrips = (p->nx + W - 1) / W;
    int nchunks = std::max(1, (nsm * per_sm) / nstrips);
    nchunks = std::min(nchunks, std::max(1, p->ny / 16));
    kern<<<dim3(nstrips, nchunks), NT, smem, s>>>((const T*)fin, (T*)fout, p->nx, p->ny, nchunks, make_coef<C>(*p),
                                                  status, first_wait);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}

template <typename T, typename C, int NT, int NS, int MINB, bool PSEAM>
int launch_pipe_scheme(const lbm_params* p, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                       long long first_wait = kWaitLimit)
{
    if (p->collision == LBM_MRT)
        return launch_pipe_cfg<T, C, MRT, GUO, NT, NS, MINB, PSEAM>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_GUO)
        return launch_pipe_cfg<T, C, BGK, GUO, NT, NS, MINB, PSEAM>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_EDM)
        return launch_pipe_cfg<T, C, BGK, EDM, NT, NS, MINB, PSEAM>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_LI)
        return launch_pipe_cfg<T, C, BGK, LI, NT, NS, MINB, PSEAM>(p, fin, fout, status, s, first_wait);
    return launch_pipe_cfg<T, C, BGK, SC, NT, NS, MINB, PSEAM>(p, fin, fout, status, s, first_wait);
}

}  // namespace lbm
