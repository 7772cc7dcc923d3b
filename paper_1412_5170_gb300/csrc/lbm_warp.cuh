// lbm_warp.cuh -- warp-per-strip fused step for FP32-deviation populations
// (the batched step's walk, and a candidate of the single-lattice autotuner):
// one warp owns a 128-column strip of a chunk of rows and walks along it
// with no block-level barrier.
//
// Per density row r the warp needs the pulled populations f*_a(x - e_a) on
// row r plus one halo column each side.  Lanes 0..8 copy the nine source row
// segments (direction a: row r - e_y(a), columns x0-4 .. x0+W+4) from HBM
// into a ring of NS shared-memory stages with cp.async.bulk (TMA bulk
// copies) completing on one mbarrier per stage.  Each lane owns 4
// consecutive columns: it reads them as one 128-bit shared load per
// direction and gets the +-1 column neighbours of the x-shifted directions
// from the adjacent lanes by warp shuffles (lane 0 and the last active lane
// read the strip's halo column from shared memory).  psi of the last three
// rows stays in registers; the psi stencil's side columns also come by
// shuffles.  Walk iteration k: wait for stage k, load row k's populations
// into registers and refill the stage with row k+NS, psi of row k, collide
// row k-1 (populations kept from the previous iteration), nine 128-bit
// stores per lane.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_strip.cuh"

namespace lbm {

constexpr unsigned kFull = 0xffffffffu;

template <int NS>
struct WarpSmem {
    static constexpr int W = 128;        // columns per warp (4 per lane)
    static constexpr int SW = W + 8;     // stage row stride (floats): column c at index 4 + c
    float* stages;                       // [NS][9][SW]
    uint64_t* bars;                      // [NS]
    __device__ explicit WarpSmem(unsigned char* smem)
        : stages(reinterpret_cast<float*>(smem)), bars(reinterpret_cast<uint64_t*>(smem + sizeof(float) * NS * 9 * SW)) {}
};

template <int NS>
constexpr size_t warp_smem() { return sizeof(float) * NS * 9 * WarpSmem<NS>::SW + 8 * NS; }

// Pulled deviations of the 4 columns [c0, c0+4) of one stage.  lane_hl is
// the last lane with columns inside the strip; it and lane 0 read their
// outer neighbour from the stage's halo, the others get it by shuffle.
template <typename C>
__device__ __forceinline__ void pull4_warp(const float* __restrict__ st, int c0, int lane, int lane_hl, C g[9][4])
{
    constexpr int SW = 136;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const float* d = st + a * SW + 4 + c0;
        const float4 v = *reinterpret_cast<const float4*>(d);
        if (ex(a) == 0) {
            g[a][0] = v.x; g[a][1] = v.y; g[a][2] = v.z; g[a][3] = v.w;
        } else if (ex(a) > 0) {            // needs column c0 - 1
            float left = __shfl_up_sync(kFull, v.w, 1);
            if (lane == 0) left = d[-1];
            g[a][0] = left; g[a][1] = v.x; g[a][2] = v.y; g[a][3] = v.z;
        } else {                           // needs column c0 + 4
            float right = __shfl_down_sync(kFull, v.x, 1);
            if (lane == lane_hl) right = d[4];
            g[a][0] = v.y; g[a][1] = v.z; g[a][2] = v.w; g[a][3] = right;
        }
    }
}

// psi of the strip's two halo columns (x0 - 1 and x0 + wp) of one stage,
// computed by the whole warp at once: lanes 0..8 load the left column's nine
// pulled values and lanes 16..24 the right column's, every lane of each half
// gathers its column's nine values by shuffles and evaluates the EOS (the
// summation order is that of sum9, as for every other column).  Lanes 0..15
// return the left value, lanes 16..31 the right one.
template <typename C>
__device__ __forceinline__ C halo_psi(const float* __restrict__ st, int lane, int wp, const Coef<C>& k,
                                      unsigned& bad)
{
    constexpr int SW = 136;
    const int half = lane >> 4, a = lane & 15;
    float v = 0.f;
    if (a < 9) v = st[a * SW + (half ? 4 + wp : 3) - ex(a)];
    C s9[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) s9[j] = C(__shfl_sync(kFull, v, (lane & 16) + j));
    unsigned b = 0;
    const C p = psi_of_rho<C>(k.rho_ref + sum9(s9), k, b);
    if (lane == 0 || lane == 16) bad |= b;
    return p;
}

// Walk the strip segment [x0, x0 + min(128, nx - x0)) x [y0, y1).  G counts
// walk rows over all segments this warp has walked (row G uses stage G % NS
// in its (G / NS)-th phase).  CARRY: the pulled populations of a row are
// loaded once, kept in registers for the next iteration's collision, and the
// stage is refilled right away (NS rows in flight, more registers); without
// CARRY the collision re-reads them from the stage, which is refilled after
// it (NS - 1 rows in flight, fewer registers, more resident warps).  Returns
// false with ST_TIMEOUT set if a stage wait gave up (copies in flight are
// drained, bounded).
// down: walk the rows from y1 - 1 to y0 (walk row kr is density row y1 - kr,
// and the psi rows y - 1 and y + 1 of the stencil trade places), so that two
// neighbouring chunks walked in opposite directions read their shared halo
// rows at about the same time.
template <typename C, int COLL, int FORC, int NS, bool CARRY>
__device__ __forceinline__ bool warp_walk(const float* __restrict__ fin, float* __restrict__ fout, int nx, int ny,
                                          int x0, int y0, int y1, bool down, const Coef<C>& k,
                                          const WarpSmem<NS>& sm, unsigned& G, unsigned& bad,
                                          long long first_wait = kWaitLimit)
{
    constexpr int SW = WarpSmem<NS>::SW;
    const int lane = threadIdx.x & 31;
    const int wp = min(WarpSmem<NS>::W, nx - x0);
    const int lane_hl = wp / 4 - 1;
    const int c0 = 4 * lane;
    const bool active = c0 < wp;
    const int H = y1 - y0;
    const int nrows = H + 2;
    const size_t n = (size_t)nx * ny;
    const unsigned stage_bytes = unsigned(9 * (wp + 8) * sizeof(float));
    const bool left_wrap = x0 == 0, right_wrap = x0 + wp == nx;
    const unsigned base = G;
    int nissued = 0;                 // walk rows whose copies have been issued
    // lane a < 9: source row of direction a for the next copy (advanced by one per copy)
    int src_row = lane < 9 ? wrap_any((down ? y1 : y0 - 1) - ey(lane), ny) : 0;
    const float* plane = fin + (lane < 9 ? lane : 0) * n;

    auto issue = [&]() {
        const unsigned g = base + nissued;
        ++nissued;
        uint64_t* bar = &sm.bars[g % NS];
        float* st = sm.stages + (g % NS) * 9 * SW;
        if (lane == 0) mbar_arrive_expect_tx(bar, stage_bytes);
        __syncwarp();
        if (lane < 9) {
            fence_proxy_async();   // earlier generic reads of this slot before the async writes
            const float* row = plane + (size_t)src_row * nx;
            float* dst = st + lane * SW;
            if (!left_wrap && !right_wrap) {
                bulk_g2s(dst, row + x0 - 4, unsigned((wp + 8) * sizeof(float)), bar);
            } else {
                bulk_g2s(dst, row + (left_wrap ? nx - 4 : x0 - 4), 16u, bar);
                bulk_g2s(dst + 4, row + x0, unsigned(wp * sizeof(float)), bar);
                bulk_g2s(dst + 4 + wp, row + (right_wrap ? 0 : x0 + wp), 16u, bar);
            }
            if (down) src_row = (src_row == 0) ? ny - 1 : src_row - 1;
            else src_row = (src_row + 1 == ny) ? 0 : src_row + 1;
        }
    };

    for (int kr = 0; kr < NS && kr < nrows; ++kr) issue();   // without CARRY the ring keeps row k-1 and k

    C pm[4] = {0, 0, 0, 0}, pc[4] = {0, 0, 0, 0};   // psi of walk rows k-2, k-1 (own columns)
    C hm = 0, hc = 0;                                // halo psi of rows k-2, k-1 (lanes < 16: left)
    unsigned mybad = 0;
    int kdone = 0;
    bool ok_all = true;
    C gA[9][4], gB[9][4];

    // One walk iteration: load row kk into gn, psi of row kk, collide row kk-1 from gc.
    auto body = [&](int kk, C (&gn)[9][4], C (&gc)[9][4]) -> bool {
        const unsigned g = base + kk;
        const float* st = sm.stages + (g % NS) * 9 * SW;
        if (!__all_sync(kFull, mbar_wait(&sm.bars[g % NS], (g / NS) & 1, kk == 0 ? first_wait : kWaitLimit)))
            return false;
        pull4_warp<C>(st, c0, lane, lane_hl, gn);
        const C hn = halo_psi<C>(st, lane, wp, k, mybad);
        if constexpr (CARRY) {
            __syncwarp();
            if (nissued < nrows) issue();   // the stage of row kk is consumed: refill it
        }
        C pn[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            C s9[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) s9[a] = gn[a][j];
            unsigned b = 0;
            pn[j] = psi_of_rho<C>(k.rho_ref + sum9(s9), k, b);
            if (active) mybad |= b;
        }
        const int kc = kk - 1;   // collide walk row kk-1 (a chunk row when 1 <= kk-1 <= H)
        // psi at columns c0-1 and c0+4 of rows y-1, y, y+1 (pm, pc, pn)
        C lm1 = __shfl_up_sync(kFull, pm[3], 1), l0 = __shfl_up_sync(kFull, pc[3], 1),
          lp1 = __shfl_up_sync(kFull, pn[3], 1);
        C rm1 = __shfl_down_sync(kFull, pm[0], 1), r0 = __shfl_down_sync(kFull, pc[0], 1),
          rp1 = __shfl_down_sync(kFull, pn[0], 1);
        const C hrm = __shfl_sync(kFull, hm, 16), hr0 = __shfl_sync(kFull, hc, 16), hrp = __shfl_sync(kFull, hn, 16);
        if (lane == 0) { lm1 = hm; l0 = hc; lp1 = hn; }
        if (lane == lane_hl) { rm1 = hrm; r0 = hr0; rp1 = hrp; }
        const bool chunk_row = kc >= 1 && kc <= H;   // warp-uniform
        if constexpr (!CARRY) {
            // every lane takes part: pull4_warp exchanges columns by full-warp shuffles
            if (chunk_row) pull4_warp<C>(sm.stages + ((base + kc) % NS) * 9 * SW, c0, lane, lane_hl, gc);
        }
        if (chunk_row && active) {
            // walk rows k-2 and k are density rows y-1 and y+1 walking up, y+1 and y-1 down
            const C row_a[6] = {lm1, pm[0], pm[1], pm[2], pm[3], rm1};
            const C row_0[6] = {l0, pc[0], pc[1], pc[2], pc[3], r0};
            const C row_b[6] = {lp1, pn[0], pn[1], pn[2], pn[3], rp1};
            C row_m[6], row_p[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                row_m[j] = down ? row_b[j] : row_a[j];
                row_p[j] = down ? row_a[j] : row_b[j];
            }
            float o[9][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                Stencil<C> q{row_0[j + 1], row_0[j + 2], row_p[j + 1], row_0[j], row_m[j + 1],
                             row_p[j + 2], row_p[j], row_m[j], row_m[j + 2]};
                C Fx, Fy, vx, vy, rho, gj[9];
                force<C>(q, k, Fx, Fy);
#pragma unroll
                for (int a = 0; a < 9; ++a) gj[a] = gc[a][j];
                collide<C, COLL, FORC>(gj, Fx, Fy, k, vx, vy, rho, q.c);
                if (!isfinite(gj[0])) mybad |= ST_NONFINITE;   // g0 closes on all others
#pragma unroll
                for (int a = 0; a < 9; ++a) o[a][j] = float(gj[a]);
            }
            float* out = fout + (size_t)(down ? y1 - kc : y0 + kc - 1) * nx + x0 + c0;
#pragma unroll
            for (int a = 0; a < 9; ++a)
                *reinterpret_cast<float4*>(out + a * n) = make_float4(o[a][0], o[a][1], o[a][2], o[a][3]);
        }
        if constexpr (!CARRY) {
            if (kc >= 0) {   // the stage of walk row kc is no longer read: refill it
                __syncwarp();
                if (nissued < nrows) issue();
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) { pm[j] = pc[j]; pc[j] = pn[j]; }
        hm = hc; hc = hn;
        return true;
    };

    for (int kk = 0; kk < nrows; kk += 2) {
        if (!body(kk, gA, gB)) { ok_all = false; kdone = kk; break; }
        if (kk + 1 < nrows && !body(kk + 1, gB, gA)) { ok_all = false; kdone = kk + 1; break; }
        kdone = kk + 2;
    }
    if (!ok_all) {
        bad |= ST_TIMEOUT;
        if (lane == 0) {   // drain the copies issued for rows never consumed (bounded)
            for (int kr = kdone; kr < nissued; ++kr) mbar_wait(&sm.bars[(base + kr) % NS], ((base + kr) / NS) & 1);
        }
        __syncwarp();
        bad |= mybad;
        return false;
    }
    bad |= mybad;
    G = base + nrows;
    __syncwarp();
    return true;
}

template <int NS>
__device__ __forceinline__ void warp_init_barriers(const WarpSmem<NS>& sm)
{
    if ((threadIdx.x & 31) == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&sm.bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();
}

// One lattice: grid (strips of 128 columns, row chunks), one warp per CTA.
template <typename C, int COLL, int FORC, int NS, bool CARRY>
__global__ void __launch_bounds__(32, CARRY ? 12 : 16)
k_step_warp(const float* __restrict__ fin, float* __restrict__ fout, int nx, int ny, int nchunks, Coef<C> k,
            unsigned* __restrict__ status, long long first_wait)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (!staged_alignment_ok(smem, fin, fout)) {
        if (threadIdx.x == 0) atomicOr(status, ST_ALIGN);
        return;
    }
    const WarpSmem<NS> sm(smem);
    const int x0 = blockIdx.x * WarpSmem<NS>::W;
    const int y0 = int((long long)blockIdx.y * ny / nchunks);
    const int y1 = int((long long)(blockIdx.y + 1) * ny / nchunks);
    if (y1 <= y0) return;
    warp_init_barriers(sm);
    unsigned G = 0, bad = 0;
    warp_walk<C, COLL, FORC, NS, CARRY>(fin, fout, nx, ny, x0, y0, y1, (blockIdx.y & 1) != 0, k, sm, G, bad,
                                        first_wait);
    flag_status(bad, status);
}

template <typename C, int COLL, int FORC, int NS, bool CARRY>
int launch_warp_cfg(const lbm_params* p, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                    long long first_wait)
{
    constexpr size_t smem = warp_smem<NS>();
    auto kern = k_step_warp<C, COLL, FORC, NS, CARRY>;
    static int per_sm = 0, nsm = 0;
    if (per_sm == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return LBM_E_CUDA;
        int dev = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32, smem) != cudaSuccess || occ < 1) occ = 1;
        per_sm = occ;
    }
    const int nstrips = (p->nx + 127) / 128;
    int nchunks = std::max(1, (nsm * per_sm) / nstrips);
    nchunks = std::min(nchunks, std::max(1, p->ny / 16));
    const Coef<C> k = make_coef<C>(*p);
    kern<<<dim3(nstrips, nchunks), 32, smem, s>>>((const float*)fin, (float*)fout, p->nx, p->ny, nchunks, k, status,
                                                  first_wait);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}

template <int NS, bool CARRY>
int launch_warp_scheme(const lbm_params* p, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                       long long first_wait = kWaitLimit)
{
    if (p->collision == LBM_MRT) return launch_warp_cfg<float, MRT, GUO, NS, CARRY>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_GUO) return launch_warp_cfg<float, BGK, GUO, NS, CARRY>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_EDM) return launch_warp_cfg<float, BGK, EDM, NS, CARRY>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_LI) return launch_warp_cfg<float, BGK, LI, NS, CARRY>(p, fin, fout, status, s, first_wait);
    return launch_warp_cfg<float, BGK, SC, NS, CARRY>(p, fin, fout, status, s, first_wait);
}

}  // namespace lbm
