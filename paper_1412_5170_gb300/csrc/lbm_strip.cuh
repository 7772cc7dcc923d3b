// lbm_strip.cuh -- the pipelined strip kernel: one fused D2Q9 time step
// (pull streaming, Eq. 3 moments, Eq. 7/29/30 psi, Eq. 6 force, BGK/MRT
// collision with Guo/EDM/SC forcing) for lattices with nx % 4 == 0.
//
// Each CTA owns a strip of W = 4*NT columns and a chunk of rows, and walks
// its rows one by one: up on even chunks, down on odd ones, so the halo rows
// that two neighbouring chunks share are read by both at about the same time
// (the start or the end of both walks) and the second read hits L2.  For density row r it needs the pulled populations
// f*_a(x - e_a) on row r and one column of halo on each side; those come
// from nine row segments (one per direction, source row r - e_y(a), columns
// x0-4 .. x0+W+4) that one warp copies into a shared-memory ring of NS
// stages with cp.async.bulk (TMA bulk copies) completing on one mbarrier per
// stage.  Every population is read from HBM once per step plus the 8-column
// and 2-row halos (served mostly by L2), never re-read for the psi stencil.
//
// Iteration k of the row walk:
//   1. wait for stage k (bounded wait)
//   2. psi of density row k (the strip's columns plus one halo column on
//      each side) into a 4-row psi ring
//   3. __syncthreads_or (also the collective timeout exit)
//   4. refill the stage freed by row k-2 with row k-2+NS (one warp)
//   5. collide row k-1: pulled populations from its stage, F from psi rows
//      k-2..k, nine 128-bit stores of the post-collision deviations
// Rows 0 and H+1 of the walk are the halo rows before and after the chunk.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "lbm_host.h"
#include "lbm_kernels.cuh"

namespace lbm {

constexpr long long kWaitLimit = kStageWaitPolls;   // try_wait polls before a stage is declared stuck

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait on one phase of an mbarrier (at most limit polls); false if
// it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit = kWaitLimit)
{
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Bulk global -> shared copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Alignment the staged kernels rely on: 128 bytes for the dynamic shared
// memory base (bulk-copy destinations, 128-bit shared loads, mbarriers) and
// 16 bytes for the population buffers (bulk-copy sources, 128-bit stores).
// A CTA that finds either violated flags ST_ALIGN and does no memory access.
__device__ __forceinline__ bool staged_alignment_ok(const void* smem, const void* fin, const void* fout)
{
    return (((uintptr_t)__cvta_generic_to_shared(smem) & 127u) == 0) &&
           ((((uintptr_t)fin | (uintptr_t)fout) & 15u) == 0);
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void lds4(const float* p, float v[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void lds4(const double* p, double v[4])
{
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void sts4(float* p, const float v[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void sts4(double* p, const double v[4])
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void stg4(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void stg4(double* p, double a, double b, double c, double d)
{
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
    *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
}

// Pulled deviations of the 4 nodes [4t, 4t+4) of a stage.  Row segment of
// direction a starts at column x0 - 4, so node column c sits at index 4 + c
// and its pulled value f*_a(c - e_x) at 4 + c - e_x.
template <typename T, typename C>
__device__ __forceinline__ void pull4(const T* __restrict__ st, int stride, int c0, C g[9][4])
{
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const T* d = st + a * stride + 4 + c0;
        T v[4];
        lds4(d, v);
        if (ex(a) == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) g[a][j] = C(v[j]);
        } else if (ex(a) > 0) {
            g[a][0] = C(d[-1]); g[a][1] = C(v[0]); g[a][2] = C(v[1]); g[a][3] = C(v[2]);
        } else {
            g[a][0] = C(v[1]); g[a][1] = C(v[2]); g[a][2] = C(v[3]); g[a][3] = C(d[4]);
        }
    }
}

// Pulled deviations of the 4 nodes [c0, c0+4) of a stage, with the +-1 column
// neighbours of the x-shifted directions taken from the adjacent lanes by
// shuffles; lanes with lsm (rsm) read their left (right) neighbour from the
// stage instead (warp edges, strip edges).  Every lane of the warp must call it.
template <typename T, typename C>
__device__ __forceinline__ void pull4_shfl(const T* __restrict__ st, int stride, int c0, bool lsm, bool rsm,
                                           C g[9][4])
{
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const T* d = st + a * stride + 4 + c0;
        T v[4];
        lds4(d, v);
        if (ex(a) == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) g[a][j] = C(v[j]);
        } else if (ex(a) > 0) {
            T left = __shfl_up_sync(0xffffffffu, v[3], 1);
            if (lsm) left = d[-1];
            g[a][0] = C(left); g[a][1] = C(v[0]); g[a][2] = C(v[1]); g[a][3] = C(v[2]);
        } else {
            T right = __shfl_down_sync(0xffffffffu, v[0], 1);
            if (rsm) right = d[4];
            g[a][0] = C(v[1]); g[a][1] = C(v[2]); g[a][2] = C(v[3]); g[a][3] = C(right);
        }
    }
}

// Six psi values of one ring row around the lane's columns (c0-1 .. c0+4):
// own four by one 128-bit load, the sides by shuffles or from shared memory.
template <typename C>
__device__ __forceinline__ void psi_row6(const C* __restrict__ prow, int c0, bool lsm, bool rsm, C r[6])
{
    C v[4];
    lds4(prow + 4 + c0, v);
    C left = __shfl_up_sync(0xffffffffu, v[3], 1);
    C right = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lsm) left = prow[3 + c0];
    if (rsm) right = prow[8 + c0];
    r[0] = left; r[1] = v[0]; r[2] = v[1]; r[3] = v[2]; r[4] = v[3]; r[5] = right;
}

// Pulled deviations of a single node at strip column c (c may be -1 or W).
template <typename T, typename C>
__device__ __forceinline__ C drho1(const T* __restrict__ st, int stride, int c)
{
    C s[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) s[a] = C(st[a * stride + 4 + c - ex(a)]);
    return sum9(s);
}

// Shared-memory carve-up of a strip CTA: NS stages [9][W+8] of T, a 4-row psi
// ring [4][W+8] of C, NS mbarriers.
template <typename T, typename C, int NT, int NS>
struct StripSmem {
    static constexpr int W = 4 * NT;
    static constexpr int SW = W + 8;     // stage row stride (elements)
    static constexpr int PW = W + 8;     // psi ring row stride: column c at index 4 + c
    T* stages;
    C* psi;
    uint64_t* bars;
    __device__ explicit StripSmem(unsigned char* smem)
        : stages(reinterpret_cast<T*>(smem)),
          psi(reinterpret_cast<C*>(smem + sizeof(T) * NS * 9 * SW)),
          bars(reinterpret_cast<uint64_t*>(smem + sizeof(T) * NS * 9 * SW + sizeof(C) * 4 * PW)) {}
};

template <typename T, typename C, int NT, int NS>
__device__ __forceinline__ void strip_init_barriers(const StripSmem<T, C, NT, NS>& sm)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&sm.bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// What a strip walk does with each chunk row once its psi neighbours are in
// the ring: called by every thread with the density row y, the lane's first
// column x (nodes x .. x+3, valid where active), its pulled deviations g, and
// psi at columns x-1 .. x+4 of rows y-1 (rm), y (r0) and y+1 (rp).
//
// StepRow, the time step: Eq. 6 force, the collision, and nine 128-bit
// stores of the post-collision deviations.
template <typename T, typename C, int COLL, int FORC>
struct StepRow {
    T* __restrict__ fout;
    int nx;
    size_t n;
    __device__ __forceinline__ void operator()(int y, int x, bool active, C (&gc)[9][4], const C (&rm)[6],
                                               const C (&r0)[6], const C (&rp)[6], const Coef<C>& k,
                                               unsigned& bad) const
    {
        if (!active) return;
        T o[9][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Stencil<C> q{r0[j + 1], r0[j + 2], rp[j + 1], r0[j], rm[j + 1], rp[j + 2], rp[j], rm[j], rm[j + 2]};
            C Fx, Fy, vx, vy, rho, gj[9];
            force<C>(q, k, Fx, Fy);
#pragma unroll
            for (int a = 0; a < 9; ++a) gj[a] = gc[a][j];
            collide<C, COLL, FORC>(gj, Fx, Fy, k, vx, vy, rho, q.c);
#pragma unroll
            for (int a = 0; a < 9; ++a) o[a][j] = T(gj[a]);
        }
        // g0 depends on all the others, and a sum of four stays non-finite
        // if one is (the populations are far below overflow)
        if (!isfinite((o[0][0] + o[0][1]) + (o[0][2] + o[0][3]))) bad |= ST_NONFINITE;
        T* out = fout + (size_t)y * nx + x;
#pragma unroll
        for (int a = 0; a < 9; ++a) stg4(out + a * n, o[a][0], o[a][1], o[a][2], o[a][3]);
    }
};

// Walk one strip segment: columns [x0, x0 + min(W, nx - x0)), rows [y0, y1).
// G counts walk rows over every segment this CTA has walked: row G uses
// stage G % NS in its (G / NS)-th phase, so segments can follow one another
// without re-initialising the barriers.  CARRY: a row's pulled populations
// stay in registers from its psi pass to its collision one iteration later,
// and its stage is refilled right after the psi pass (NS rows in flight);
// otherwise the collision re-reads the stage, refilled after it.  Returns
// false (with ST_TIMEOUT in bad) if a stage wait gave up; the copies already
// issued are then drained (bounded) and the CTA must stop.  down: walk the
// rows from y1 - 1 to y0 instead of y0 to y1 - 1 (walk row kr is density row
// y1 - kr instead of y0 - 1 + kr; the psi rows y - 1 and y + 1 of the
// stencil swap ring slots).  All threads of the CTA call this with the same
// arguments.
template <typename T, typename C, int NT, int NS, bool CARRY, bool HALO1, bool PSEAM, class Row>
__device__ __forceinline__ bool strip_walk(const T* __restrict__ fin, int nx, int ny, int x0, int y0, int y1,
                                           bool down, const Coef<C>& k, const StripSmem<T, C, NT, NS>& sm,
                                           unsigned& G, unsigned& bad, Row& row,
                                           long long first_wait = kWaitLimit)
{
    using SM = StripSmem<T, C, NT, NS>;
    constexpr int SW = SM::SW, PW = SM::PW;
    const int t = threadIdx.x, lane = t & 31;
    const int wp = min(SM::W, nx - x0);                      // strip width (multiple of 4)
    const int H = y1 - y0;
    const size_t n = (size_t)nx * ny;
    const int nrows = H + 2;                                 // walk rows incl. 2 halo rows
    const unsigned stage_bytes = unsigned(9 * (wp + 8) * sizeof(T));
    const bool left_wrap = x0 == 0, right_wrap = x0 + wp == nx;
    const unsigned base = G;
    const int c0 = 4 * t;
    const bool active = c0 < wp;
    const bool lsm = lane == 0, rsm = (lane == 31) || (c0 + 4 == wp);   // neighbours from shared memory
    int nissued = 0;

    // Warp 0 issues the nine segment copies of the next walk row into its stage,
    // one per lane; at the periodic seam each splits in three, issued by the
    // same lane or, with PSEAM, by three lanes.
    auto issue = [&]() {
        const int kr = nissued++;
        if (t >= 32) return;
        const unsigned g = base + kr;
        uint64_t* bar = &sm.bars[g % NS];
        T* st = sm.stages + (g % NS) * 9 * SW;
        if (t == 0) mbar_arrive_expect_tx(bar, stage_bytes);
        __syncwarp();
        const bool seam = left_wrap || right_wrap;   // uniform over the CTA
        if (PSEAM && seam) {
            // one copy per lane at the periodic seam: direction t / 3, piece t % 3 (the
            // segment's left halo, its body, its right halo)
            if (t < 27) {
                fence_proxy_async();   // order earlier generic reads of this slot before the async writes
                const int a = t / 3, piece = t - 3 * a;
                const int r = wrap_any((down ? y1 - kr : y0 - 1 + kr) - ey(a), ny);
                const T* row = fin + a * n + (size_t)r * nx;
                T* dst = st + a * SW;
                if (piece == 0) bulk_g2s(dst, row + (left_wrap ? nx - 4 : x0 - 4), unsigned(4 * sizeof(T)), bar);
                else if (piece == 1) bulk_g2s(dst + 4, row + x0, unsigned(wp * sizeof(T)), bar);
                else bulk_g2s(dst + 4 + wp, row + (right_wrap ? 0 : x0 + wp), unsigned(4 * sizeof(T)), bar);
            }
        } else if (t < 9) {
            fence_proxy_async();   // order earlier generic reads of this slot before the async writes
            const int a = t;
            const int r = wrap_any((down ? y1 - kr : y0 - 1 + kr) - ey(a), ny);
            const T* row = fin + a * n + (size_t)r * nx;
            T* dst = st + a * SW;
            if (!seam) {
                bulk_g2s(dst, row + x0 - 4, unsigned((wp + 8) * sizeof(T)), bar);
            } else {
                bulk_g2s(dst, row + (left_wrap ? nx - 4 : x0 - 4), unsigned(4 * sizeof(T)), bar);
                bulk_g2s(dst + 4, row + x0, unsigned(wp * sizeof(T)), bar);
                bulk_g2s(dst + 4 + wp, row + (right_wrap ? 0 : x0 + wp), unsigned(4 * sizeof(T)), bar);
            }
        }
    };

    for (int kr = 0; kr < (CARRY ? NS : NS - 2) && kr < nrows; ++kr) issue();

    int kdone = 0;
    bool ok_all = true;
    C gA[9][4], gB[9][4];

    auto body = [&](int kk, C (&gn)[9][4], C (&gc)[9][4]) -> bool {
        const unsigned g = base + kk;
        const T* st = sm.stages + (g % NS) * 9 * SW;
        const bool ok = mbar_wait(&sm.bars[g % NS], (g / NS) & 1, kk == 0 ? first_wait : kWaitLimit);
        C* prow = sm.psi + (kk & 3) * PW;
        if (ok) {
            pull4_shfl<T, C>(st, SW, c0, lsm, rsm, gn);
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
            if (active) sts4(prow + 4 + c0, ps);
            // the two halo columns' psi: the left one by thread 0, or with HALO1 by thread 32,
            // off the warp that issues the bulk copies (which helps some tile shapes)
            constexpr int kLeftHalo = (HALO1 && NT >= 64) ? 32 : 0;
            if (t == kLeftHalo) prow[3] = psi_of_rho<C>(k.rho_ref + drho1<T, C>(st, SW, -1), k, bad);
            if (t == NT - 1) prow[4 + wp] = psi_of_rho<C>(k.rho_ref + drho1<T, C>(st, SW, wp), k, bad);
        }
        if (__syncthreads_or(!ok)) return false;
        // Refill a stage every thread is done with: with CARRY the one of row kk
        // (read only by the psi pass above), otherwise the one of row kk-2 (its
        // collision ran in the previous iteration, before this barrier).
        if (nissued < nrows) issue();
        // collide walk row kk-1 (a chunk row when 1 <= kk-1 <= H)
        const int kc = kk - 1;
        if (kc >= 1 && kc <= H) {                // uniform over the CTA
            if (!CARRY) pull4_shfl<T, C>(sm.stages + ((base + kc) % NS) * 9 * SW, SW, c0, lsm, rsm, gc);
            C rm[6], r0[6], rp[6];               // psi at columns c0-1 .. c0+4 of rows y-1, y, y+1
            psi_row6<C>(sm.psi + ((down ? kc + 1 : kc - 1) & 3) * PW, c0, lsm, rsm, rm);
            psi_row6<C>(sm.psi + (kc & 3) * PW, c0, lsm, rsm, r0);
            psi_row6<C>(sm.psi + ((down ? kc - 1 : kc + 1) & 3) * PW, c0, lsm, rsm, rp);
            row(down ? y1 - kc : y0 + kc - 1, x0 + c0, active, gc, rm, r0, rp, k, bad);
        }
        return true;
    };

    for (int kk = 0; kk < nrows; kk += 2) {
        if (!body(kk, gA, gB)) { ok_all = false; kdone = kk; break; }
        if (kk + 1 < nrows && !body(kk + 1, gB, gA)) { ok_all = false; kdone = kk + 1; break; }
        kdone = kk + 2;
    }
    if (!ok_all) {
        bad |= ST_TIMEOUT;
        // Drain copies already issued for rows the walk never consumed (bounded).
        if (t == 0)
            for (int kr = kdone; kr < nissued; ++kr) mbar_wait(&sm.bars[(base + kr) % NS], ((base + kr) / NS) & 1);
        __syncthreads();
        return false;
    }
    G = base + nrows;
    __syncthreads();   // every read of this segment's stages is done before the next segment's copies
    return true;
}

// A strip walk of the time step (StepRow) from fin into fout.
template <typename T, typename C, int COLL, int FORC, int NT, int NS, bool CARRY, bool HALO1 = false,
          bool PSEAM = false>
__device__ __forceinline__ bool strip_walk_step(const T* __restrict__ fin, T* __restrict__ fout, int nx, int ny,
                                                int x0, int y0, int y1, bool down, const Coef<C>& k,
                                                const StripSmem<T, C, NT, NS>& sm, unsigned& G, unsigned& bad,
                                                long long first_wait = kWaitLimit)
{
    StepRow<T, C, COLL, FORC> row{fout, nx, (size_t)nx * ny};
    return strip_walk<T, C, NT, NS, CARRY, HALO1, PSEAM>(fin, nx, ny, x0, y0, y1, down, k, sm, G, bad, row,
                                                         first_wait);
}

// One lattice, grid (strips, row chunks).  MINB > 1 asks the compiler to fit
// MINB CTAs per SM in the register file (at the price of spills if needed).
// Launched as a programmatic dependent of the previous kernel on the stream
// (launch_strip_cfg): each CTA first waits until that kernel has completed
// and its writes are visible (griddepcontrol.wait), so no CTA touches global
// memory early; it then lets the next step's CTAs be scheduled as soon as
// SMs free up, which hides the launch gap between consecutive steps.  The
// dependents are launched only once every CTA of this grid has passed its
// launch_dependents (or exited), so a waiting dependent CTA never holds an
// SM that a CTA of this grid has yet to start on.
template <typename T, typename C, int COLL, int FORC, int NT, int NS, bool CARRY, int MINB, bool HALO1, bool PSEAM>
__global__ void __launch_bounds__(NT, MINB)
k_step_strip(const T* __restrict__ fin, T* __restrict__ fout, int nx, int ny, int nchunks, Coef<C> k,
             unsigned* __restrict__ status, long long first_wait)
{
    extern __shared__ __align__(128) unsigned char smem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (!staged_alignment_ok(smem, fin, fout)) {
        if (threadIdx.x == 0) atomicOr(status, ST_ALIGN);
        return;
    }
    const StripSmem<T, C, NT, NS> sm(smem);
    const int x0 = blockIdx.x * (4 * NT);
    const int y0 = int((long long)blockIdx.y * ny / nchunks);
    const int y1 = int((long long)(blockIdx.y + 1) * ny / nchunks);
    if (y1 <= y0) return;
    strip_init_barriers(sm);
    unsigned G = 0, bad = 0;
    strip_walk_step<T, C, COLL, FORC, NT, NS, CARRY, HALO1, PSEAM>(fin, fout, nx, ny, x0, y0, y1,
                                                                   (blockIdx.y & 1) != 0, k, sm, G, bad, first_wait);
    flag_status(bad, status);
}

template <typename T, typename C, int NT, int NS>
constexpr size_t strip_smem()
{
    return sizeof(T) * NS * 9 * (4 * NT + 8) + sizeof(C) * 4 * (4 * NT + 8) + 8 * NS;
}

// One launch over the whole lattice: strips of 4*NT columns, and as many row
// chunks as fill every resident CTA slot once (one wave), but no chunk shorter
// than 16 rows, so the two halo rows per chunk stay a small overhead.
template <typename T, typename C, int COLL, int FORC, int NT, int NS, bool CARRY, int MINB, bool HALO1, bool PSEAM>
int launch_strip_cfg(const lbm_params* p, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                     long long first_wait)
{
    constexpr size_t smem = strip_smem<T, C, NT, NS>();
    auto kern = k_step_strip<T, C, COLL, FORC, NT, NS, CARRY, MINB, HALO1, PSEAM>;
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
    const Coef<C> k = make_coef<C>(*p);
    // programmatic dependent launch (see k_step_strip)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(nstrips, nchunks);
    lc.blockDim = dim3(NT);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&lc, kern, (const T*)fin, (T*)fout, p->nx, p->ny, nchunks, k, status,
                                             first_wait);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}

template <typename T, typename C, int NT, int NS, bool CARRY = false, int MINB = 1, bool HALO1 = false,
          bool PSEAM = false>
int launch_strip_scheme(const lbm_params* p, const void* fin, void* fout, unsigned* status, cudaStream_t s,
                        long long first_wait = kWaitLimit)
{
    if (p->collision == LBM_MRT)
        return launch_strip_cfg<T, C, MRT, GUO, NT, NS, CARRY, MINB, HALO1, PSEAM>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_GUO)
        return launch_strip_cfg<T, C, BGK, GUO, NT, NS, CARRY, MINB, HALO1, PSEAM>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_EDM)
        return launch_strip_cfg<T, C, BGK, EDM, NT, NS, CARRY, MINB, HALO1, PSEAM>(p, fin, fout, status, s, first_wait);
    if (p->forcing == LBM_LI)
        return launch_strip_cfg<T, C, BGK, LI, NT, NS, CARRY, MINB, HALO1, PSEAM>(p, fin, fout, status, s, first_wait);
    return launch_strip_cfg<T, C, BGK, SC, NT, NS, CARRY, MINB, HALO1, PSEAM>(p, fin, fout, status, s, first_wait);
}

}  // namespace lbm
