// lbm_batch.cu -- many independent lattices stepped together: one launch per
// time step covers every running instance through a table of work items
// (one-warp walks of 128-column strips here, block-wide walks of wider
// strips in lbm_batch_strip.cu), check intervals are captured in CUDA graphs, and convergence and
// failure are decided per instance on the device.  Also the warm-start
// helpers: radial density profiles of instances and initial fields built
// from a profile, optionally with the populations at rest.
//
// Layout: all instances' FP32-deviation populations live in two buffers,
// instance i at element offset off_i with its own [9][ny][nx] block; FP64
// per-node arrays (density output, snapshot) at node offset node_off_i.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_batch.cuh"
#include "lbm_host.h"
#include "lbm_warp.cuh"

namespace lbm {

struct BTile { int inst, tx, ty; };

// Per-instance observables and convergence record (device).
struct BObs {
    double mass, max_v, max_dv, max_drho, rho_min, rho_max;
    double rho_center, rho_corner, rho_row_mid, rho_row0;
};
struct BPart {
    double sum[3];        // mass, row ny/2, row 0
    double mx[5];         // max_v, max_dv, max_drho, rho_max, -rho_min
    unsigned status, pad;
};
// Convergence snapshot per node in the compute type: v and the density
// deviation drho (rho = rho_ref + drho).
struct __align__(16) Snap { float vx, vy, drho, pad; };

constexpr int kBatchWarps = 1;   // warps (independent 128-column walkers) per CTA

// Dynamic shared memory of one batched-step CTA: per warp its stage ring and
// barriers (warp_smem), then one Coef per warp at a 16-byte aligned offset.
// (No static shared memory: it would shift the dynamic region off the
// 128-byte alignment the stage ring's bulk copies and 128-bit loads need.)
template <int NS>
constexpr size_t batch_coef_off() { return (kBatchWarps * warp_smem<NS>() + 15) / 16 * 16; }

// One time step of every running instance.  Each warp takes work items
// (instance, 128-column strip, row chunk) from a queue -- queue[0], a counter
// it increments atomically, the items sorted longest first -- until none is
// left; the instance's constants are staged in shared memory per item.  Each
// warp then counts itself done in queue[1], and the last one clears both
// counters, so every launch starts from zero whatever ran before it.
template <int COLL, int FORC, int NS, bool CARRY>
__global__ void __launch_bounds__(32 * kBatchWarps, 16 / kBatchWarps)
k_step_batch(const float* __restrict__ fin, float* __restrict__ fout, const BInst* __restrict__ inst,
             const BItem* __restrict__ items, int n_items, const int* __restrict__ state,
             unsigned* __restrict__ inst_status, int* __restrict__ queue)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (!staged_alignment_ok(smem, fin, fout)) {   // flag every instance of this launch
        for (int i = threadIdx.x; i < n_items; i += blockDim.x) atomicOr(&inst_status[items[i].inst], ST_ALIGN);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpSmem<NS> sm(smem + warp * warp_smem<NS>());
    Coef<float>* sk = reinterpret_cast<Coef<float>*>(smem + batch_coef_off<NS>()) + warp;
    warp_init_barriers(sm);
    unsigned G = 0;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&queue[0], 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const BItem w = items[it];
        if (state[w.inst] != B_RUNNING) continue;          // uniform over the warp
        const BInst* I = inst + w.inst;
        constexpr int nwords = sizeof(Coef<float>) / sizeof(float);
        if (lane < nwords) reinterpret_cast<float*>(sk)[lane] = reinterpret_cast<const float*>(&I->k)[lane];
        __syncwarp();
        unsigned bad = 0;
        const bool ok = warp_walk<float, COLL, FORC, NS, CARRY>(fin + I->off, fout + I->off, I->nx, I->ny, w.x0,
                                                                w.y0, w.y1, w.down != 0, *sk, sm, G, bad);
        flag_status(bad, &inst_status[w.inst]);
        __syncwarp();
        if (!ok) break;   // a stage wait timed out: the instance is flagged, stop this warp
    }
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(&queue[1], 1) == (int)(gridDim.x * kBatchWarps) - 1) {   // the last warp done
            atomicExch(&queue[0], 0);
            atomicExch(&queue[1], 0);
        }
    }
}

template <int NS>
constexpr size_t batch_smem() { return batch_coef_off<NS>() + kBatchWarps * sizeof(Coef<float>); }

enum : int { BO_RHO = 1, BO_SNAP = 2, BO_ALL = 4 };

// Observables per 32 x 8 tile of every running instance (every instance with
// BO_ALL): rho and v = u + F/(2 rho); with BO_SNAP the changes against the
// snapshot (vx, vy, rho) of the previous check, which is then replaced; with
// BO_RHO the FP64 density field.
__global__ void __launch_bounds__(GTX * GTY)
k_observe_batch(const float* __restrict__ f, const BInst* __restrict__ inst, const BTile* __restrict__ tiles,
                const int* __restrict__ state, Snap* __restrict__ snap, double* __restrict__ rho_out,
                BPart* __restrict__ parts, BObs* __restrict__ obs, int mode)
{
    __shared__ float sp[(GTY + 2) * (GTX + 2)];
    __shared__ double red[8][GTX * GTY / 32];
    __shared__ unsigned sbad;
    const BTile tl = tiles[blockIdx.x];
    if (!(mode & BO_ALL) && state[tl.inst] != B_RUNNING) return;   // uniform over the block
    const BInst* I = inst + tl.inst;
    const int nx = I->nx, ny = I->ny;
    const Coef<float> k = I->k;
    const float* fi = f + I->off;
    const size_t n = (size_t)nx * ny;
    const int x0 = tl.tx * GTX, y0 = tl.ty * GTY;
    unsigned bad = 0;
    if (threadIdx.x == 0) sbad = 0;
    for (int i = threadIdx.x; i < (GTX + 2) * (GTY + 2); i += blockDim.x) {
        const int x = wrap_any(x0 + i % (GTX + 2) - 1, nx);
        const int y = wrap_any(y0 + i / (GTX + 2) - 1, ny);
        float g[9];
        pull_node<float, float>(fi, x, y, nx, ny, n, g);
        sp[i] = psi_of_rho<float>(k.rho_ref + sum9(g), k, bad);
    }
    __syncthreads();
    const int tx = threadIdx.x % GTX, ty = threadIdx.x / GTX;
    const int x = x0 + tx, y = y0 + ty;
    // Per-node work in FP32 (maxima are exact in any precision; only the
    // mass and probe-row sums take FP64 arithmetic, the row sums only in the
    // warps that hold those rows: a warp is one tile row).
    double rho = 0;
    float mv = 0.f, dv = 0.f, dr = 0.f, dmax = -1e30f, ndmin = -1e30f;
    if (x < nx && y < ny) {
        float g[9];
        pull_node<float, float>(fi, x, y, nx, ny, n, g);
        const int W = GTX + 2, c = (ty + 1) * W + tx + 1;
        Stencil<float> q{sp[c], sp[c + 1], sp[c + W], sp[c - 1], sp[c - W],
                         sp[c + W + 1], sp[c + W - 1], sp[c - W - 1], sp[c - W + 1]};
        float Fx, Fy, drho, jx, jy;
        force<float>(q, k, Fx, Fy);
        moments<float>(g, drho, jx, jy);
        const float rc = k.rho_ref + drho;
        rho = double(k.rho_ref) + double(drho);
        const float vx = jx / rc + 0.5f * Fx / rc;
        const float vy = jy / rc + 0.5f * Fy / rc;
        if (!isfinite(drho) || !isfinite(vx) || !isfinite(vy)) bad |= ST_NONFINITE;
        const size_t o = (size_t)I->node_off + (size_t)y * nx + x;
        if (mode & BO_RHO) rho_out[o] = rho;
        dv = 1e30f;
        dr = 1e30f;
        if (mode & BO_SNAP) {
            const Snap s = snap[o];
            const float ddx = vx - s.vx, ddy = vy - s.vy;
            dv = sqrtf(ddx * ddx + ddy * ddy);
            dr = fabsf(drho - s.drho) / rc;
            if (isnan(dv)) dv = 1e30f;
            if (isnan(dr)) dr = 1e30f;
            snap[o] = Snap{vx, vy, drho, 0.f};
        }
        mv = sqrtf(vx * vx + vy * vy);
        if (isnan(mv)) mv = 1e30f;
        dmax = drho;
        ndmin = -drho;
        if (x == nx / 2 && y == ny / 2) obs[tl.inst].rho_center = rho;
        if (x == 0 && y == 0) obs[tl.inst].rho_corner = rho;
    }
    const bool mid_row = y == ny / 2, row_0 = y == 0;   // uniform over the warp
    double v[8];
    v[0] = warp_sum(rho);
    v[1] = mid_row ? warp_sum(rho) : 0.0;
    v[2] = row_0 ? warp_sum(rho) : 0.0;
    v[3] = double(warp_max(mv));
    v[4] = double(warp_max(dv));
    v[5] = double(warp_max(dr));
    v[6] = double(k.rho_ref) + double(warp_max(dmax));
    v[7] = -(double(k.rho_ref) + double(-warp_max(ndmin)));
    const unsigned wb = __reduce_or_sync(0xffffffffu, bad);
    const int wid = threadIdx.x / 32;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        for (int j = 0; j < 8; ++j) red[j][wid] = v[j];
        if (wb) atomicOr(&sbad, wb);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        BPart p;
        p.sum[0] = p.sum[1] = p.sum[2] = 0;
        for (int j = 0; j < 5; ++j) p.mx[j] = -1e300;
        for (int w = 0; w < GTX * GTY / 32; ++w) {
            for (int j = 0; j < 3; ++j) p.sum[j] += red[j][w];
            for (int j = 0; j < 5; ++j) p.mx[j] = fmax(p.mx[j], red[3 + j][w]);
        }
        p.status = sbad;
        p.pad = 0;
        parts[I->tile_off + tl.ty * I->ntx + tl.tx] = p;
    }
}

// What is left of a probe's approach to its limit, estimated from its last
// two changes d (this interval) and dp (the one before) as a geometric series
// with ratio r = d / dp (Aitken's extrapolation): |d| r / (1 - r) for
// 0 <= r < 1, |d| for an alternating approach (r < 0, the limit lies within
// the last change), infinite while the changes do not shrink (r >= 1),
// before two changes are known (dp NaN) or after a standstill (dp = 0);
// zero for a probe that did not move.
__device__ __forceinline__ double coex_tail(double d, double dp)
{
    if (d == 0.0) return 0.0;
    if (!(dp != 0.0)) return HUGE_VAL;
    const double r = d / dp;
    if (!(r < 1.0)) return HUGE_VAL;
    return r < 0.0 ? fabs(d) : fabs(d) * r / (1.0 - r);
}

// Per-instance fixed-order reduction of the tile partials, then the
// convergence / failure decision: a running instance stops as converged when
// max|v - v_snap| < tol_v, max|rho - rho_snap|/rho < tol_rho, or both of its
// coexistence densities (liquid and vapour probe: centre and corner node of a
// droplet or bubble, mid and edge row of a slab) changed by less than tol_coex
// relative since the previous check -- with coex_rule LBM_COEX_TAIL, also
// their estimated remaining changes (coex_tail) from the last two pairs of
// changes -- (a tolerance <= 0
// disables it), and -- with or without a decision -- as failed when a kernel
// flagged it.  probe_prev holds
// each instance's probes at the previous check and their changes then.
// probes at the previous check, their changes then and the changes before
struct ProbeHist { double pl, pv, dl, dv, dl2, dv2; };

__global__ void __launch_bounds__(256)
k_reduce_batch(const BInst* __restrict__ inst, const BPart* __restrict__ parts, int* __restrict__ state,
               int* __restrict__ fail_code, const unsigned* __restrict__ inst_status, BObs* __restrict__ obs,
               ProbeHist* __restrict__ probe_prev, double tol_v, double tol_rho, double tol_coex, int coex_rule,
               int decide, int all)
{
    const int i = blockIdx.x;
    if (!all && state[i] != B_RUNNING) return;
    const BInst* I = inst + i;
    const int nt = I->ntx * I->nty;
    __shared__ double red[8][256];
    __shared__ unsigned sbad[256];
    double v[8] = {0, 0, 0, -1e300, -1e300, -1e300, -1e300, -1e300};
    unsigned bad = 0;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const BPart p = parts[I->tile_off + t];
        for (int j = 0; j < 3; ++j) v[j] += p.sum[j];
        for (int j = 0; j < 5; ++j) v[3 + j] = fmax(v[3 + j], p.mx[j]);
        bad |= p.status;
    }
    for (int j = 0; j < 8; ++j) red[j][threadIdx.x] = v[j];
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int o = threadIdx.x + s;
            for (int j = 0; j < 3; ++j) red[j][threadIdx.x] += red[j][o];
            for (int j = 3; j < 8; ++j) red[j][threadIdx.x] = fmax(red[j][threadIdx.x], red[j][o]);
            sbad[threadIdx.x] |= sbad[o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        BObs& o = obs[i];
        o.mass = red[0][0];
        o.rho_row_mid = red[1][0] / I->nx;
        o.rho_row0 = red[2][0] / I->nx;
        o.max_v = red[3][0];
        o.max_dv = red[4][0];
        o.max_drho = red[5][0];
        o.rho_max = red[6][0];
        o.rho_min = -red[7][0];
        const unsigned b = sbad[0] | inst_status[i];
        if (state[i] != B_RUNNING) return;
        if (b) {   // a kernel flagged this instance: failed, with or without a decision
            state[i] = B_FAILED;
            fail_code[i] = (b & ST_NONFINITE) ? LBM_E_NONFINITE
                           : (b & ST_EOS) ? LBM_E_EOS_DOMAIN
                           : (b & ST_TIMEOUT) ? LBM_E_TIMEOUT : LBM_E_CUDA;
            return;
        }
        if (!decide) return;
        const bool slab = I->kind == LBM_SLAB;
        const double pl = slab ? o.rho_row_mid : o.rho_center, pv = slab ? o.rho_row0 : o.rho_corner;
        const ProbeHist pp = probe_prev[i];
        const double dl = pl - pp.pl, dv = pv - pp.pv;
        double dcoex = fmax(fabs(dl) / fabs(pl), fabs(dv) / fabs(pv));   // NaN before the first check
        if (coex_rule == LBM_COEX_TAIL && dcoex == dcoex) {
            // the estimate from this check's pair of changes and from the previous pair: both
            // must be small, so that one change whose sign the rounding noise flipped cannot
            // pass a slow monotone approach for an alternating one
            const double tl = fmax(coex_tail(dl, pp.dl), coex_tail(pp.dl, pp.dl2));
            const double tv = fmax(coex_tail(dv, pp.dv), coex_tail(pp.dv, pp.dv2));
            dcoex = fmax(dcoex, fmax(tl / fabs(pl), tv / fabs(pv)));
        }
        probe_prev[i] = ProbeHist{pl, pv, dl, dv, pp.dl, pp.dv};
        if ((tol_v > 0 && o.max_dv < tol_v) || (tol_rho > 0 && o.max_drho < tol_rho) ||
            (tol_coex > 0 && dcoex < tol_coex))
            state[i] = B_CONVERGED;
    }
}

__device__ __forceinline__ unsigned long long splitmix64_dev(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Signed distance to the liquid of node (x, y) of an instance (slab, droplet,
// bubble: distance to the gas region is returned negated by the caller).
__device__ __forceinline__ double preset_distance(const BInst* I, int x, int y)
{
    if (I->kind == LBM_SLAB) return fabs(y - I->ny / 2.0) - I->size;
    if (I->kind == LBM_DROPLET_ARRAY) {
        const double cx = floor(double(x) / I->cell) * I->cell + I->cell / 2.0;
        const double cy = floor(double(y) / I->cell) * I->cell + I->cell / 2.0;
        return hypot(x - cx, y - cy) - I->size;
    }
    return hypot(x - I->nx / 2.0, y - I->ny / 2.0) - I->size;
}

// Grid of an instance's radial profile (mirrors lbm_profile_geom): sample k
// at signed position centre + spacing (k - (nb - 1)/2) from the centre / mid-row.
struct BGeom { int use, pad; double centre, spacing; };

// Distance of node (x, y) from the centre of a droplet or bubble, or from the
// mid-row of a slab.
__device__ __forceinline__ double radial_distance(const BInst* I, int x, int y)
{
    if (I->kind == LBM_SLAB) return fabs(y - I->ny / 2.0);
    return hypot(x - I->nx / 2.0, y - I->ny / 2.0);
}

// Profile density at distance r: linear between samples, end values beyond.
__device__ __forceinline__ double profile_at(const double* p, int nb, const BGeom& g, double r)
{
    const double u = (r - g.centre) / g.spacing + 0.5 * (nb - 1);
    if (!(u > 0.0)) return p[0];
    if (u >= nb - 1) return p[nb - 1];
    const int k0 = int(u);
    const double t = u - k0;
    return p[k0] + t * (p[k0 + 1] - p[k0]);
}

// Initial density rho0 of every instance into the FP64 node array: its
// preset (tanh profile plus SplitMix64 noise) or, where geom[i].use, its
// radial profile.
__global__ void k_rho0_batch(const BInst* __restrict__ inst, int n_inst, double* __restrict__ rho0,
                             const double* __restrict__ prof, const BGeom* __restrict__ geom, int nb)
{
    const int i = blockIdx.y;
    if (i >= n_inst) return;
    const BInst* I = inst + i;
    const int nx = I->nx, ny = I->ny;
    const size_t n = (size_t)nx * ny;
    const bool use_prof = prof && geom[i].use;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const int x = int(id % nx), y = int(id / nx);
        double r;
        if (use_prof) {
            r = profile_at(prof + (size_t)i * nb, nb, geom[i], radial_distance(I, x, y));
        } else {
            const double d = preset_distance(I, x, y);
            const double in = 0.5 * (1.0 - tanh(2.0 * d / I->width));
            r = (I->kind == LBM_BUBBLE) ? I->rho_l + (I->rho_v - I->rho_l) * in
                                        : I->rho_v + (I->rho_l - I->rho_v) * in;
            if (I->noise_amp != 0.0) {
                const unsigned long long z = splitmix64_dev(I->seed ^ (unsigned long long)((size_t)y * nx + x));
                r += I->noise_amp * (2.0 * (double(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0);
            }
        }
        rho0[I->node_off + id] = r;
    }
}

// Rest velocity u0 = -F/(2 rho0) of the profile instances (into the vx, vy
// slots of the per-node snapshot array): psi and the Eq. 6 force of rho0 in
// the instance's compute type, exactly as the time step evaluates them.
__global__ void k_rest_velocity(const BInst* __restrict__ inst, int n_inst, const double* __restrict__ rho0,
                                const BGeom* __restrict__ geom, Snap* __restrict__ u0)
{
    const int i = blockIdx.y;
    if (i >= n_inst || !geom[i].use) return;
    const BInst* I = inst + i;
    const int nx = I->nx, ny = I->ny;
    const size_t n = (size_t)nx * ny;
    const Coef<float> k = I->k;
    const double* r0 = rho0 + I->node_off;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const int x = int(id % nx), y = int(id / nx);
        unsigned bad = 0;
        auto psi_at = [&](int dx, int dy) {
            const int xs = wrap_any(x + dx, nx), ys = wrap_any(y + dy, ny);
            const float drho = float(r0[(size_t)ys * nx + xs] - double(k.rho_ref));
            return psi_of_rho<float>(k.rho_ref + drho, k, bad);
        };
        const Stencil<float> q{psi_at(0, 0), psi_at(1, 0), psi_at(0, 1), psi_at(-1, 0), psi_at(0, -1),
                               psi_at(1, 1), psi_at(-1, 1), psi_at(-1, -1), psi_at(1, -1)};
        float Fx, Fy;
        force<float>(q, k, Fx, Fy);
        const float rho = k.rho_ref + float(r0[id] - double(k.rho_ref));
        Snap& o = u0[I->node_off + id];
        o.vx = -0.5f * Fx / rho;
        o.vy = -0.5f * Fy / rho;
    }
}

// Populations from rho0 (and, for the rest-started instances, u0) as
// pull-convention FP32 deviations: the value stored at x for direction a is
// the one that arrives at x + e_a, f_a = w_a rho0 (1 + 3 e.u + 9/2 (e.u)^2 -
// 3/2 u.u) there (Eq. 2 with c_s^2 = 1/3), minus w_a rho_ref.
__global__ void k_pops_batch(const BInst* __restrict__ inst, int n_inst, float* __restrict__ f,
                             const double* __restrict__ rho0, const Snap* __restrict__ u0,
                             const BGeom* __restrict__ geom)
{
    const int i = blockIdx.y;
    if (i >= n_inst) return;
    const BInst* I = inst + i;
    const int nx = I->nx, ny = I->ny;
    const size_t n = (size_t)nx * ny;
    const double* r0 = rho0 + I->node_off;
    const bool rest = u0 && geom && geom[i].use;
    for (size_t id = blockIdx.x * (size_t)blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x) {
        const int x = int(id % nx), y = int(id / nx);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int xs = ex(a) > 0 ? inc1(x, nx) : (ex(a) < 0 ? dec1(x, nx) : x);
            const int ys = ey(a) > 0 ? inc1(y, ny) : (ey(a) < 0 ? dec1(y, ny) : y);
            const size_t src = (size_t)ys * nx + xs;
            const double w = wt<double>(a), r = r0[src];
            double v = w * r - w * double(I->k.rho_ref);
            if (rest) {
                const Snap u = u0[I->node_off + src];
                const double ux = u.vx, uy = u.vy;
                const double eu = ex(a) * ux + ey(a) * uy;
                v += w * r * (3.0 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy));
            }
            f[I->off + a * n + id] = float(v);
        }
    }
}

// Radial density profile of instance i from its FP64 density field on its
// sample grid: at r_k = |centre + spacing (k - (nb - 1)/2)| the mean over 64
// directions of the bilinearly interpolated density at distance r_k from the
// centre (droplet, bubble), or the mean over x and both sides of the
// mid-row at y = ny/2 +- r_k (slab), with r_k held at most half the period
// minus one.  One block per (sample, instance).
__global__ void k_radial_profile(const BInst* __restrict__ inst, const double* __restrict__ rho, int nb,
                                 const BGeom* __restrict__ geom, double* __restrict__ prof)
{
    const int i = blockIdx.y, kb = blockIdx.x;
    const BInst* I = inst + i;
    const int nx = I->nx, ny = I->ny;
    const double* r = rho + I->node_off;
    // Distances beyond the half period would wrap onto the next image of the
    // droplet or slab: they are held at the farthest point of the period.
    const double rmax = (I->kind == LBM_SLAB ? ny : min(nx, ny)) / 2.0 - 1.0;
    const double dist = fmin(fabs(geom[i].centre + geom[i].spacing * (kb - 0.5 * (nb - 1))), rmax);
    __shared__ double acc[128];
    double sum = 0;
    int cnt = 0;
    auto at = [&](int x, int y) { return r[(size_t)wrap_any(y, ny) * nx + wrap_any(x, nx)]; };
    if (I->kind == LBM_SLAB) {
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            for (int side = -1; side <= 1; side += 2) {
                const double yy = ny / 2.0 + side * dist;
                const int y0 = int(floor(yy));
                const double t = yy - y0;
                sum += (1 - t) * at(x, y0) + t * at(x, y0 + 1);
                ++cnt;
            }
        }
    } else {
        for (int d = threadIdx.x; d < 64; d += blockDim.x) {
            const double th = 2.0 * 3.14159265358979323846 * d / 64;
            const double xx = nx / 2.0 + dist * cos(th), yy = ny / 2.0 + dist * sin(th);
            const int x0 = int(floor(xx)), y0 = int(floor(yy));
            const double tx = xx - x0, ty = yy - y0;
            sum += (1 - tx) * (1 - ty) * at(x0, y0) + tx * (1 - ty) * at(x0 + 1, y0) +
                   (1 - tx) * ty * at(x0, y0 + 1) + tx * ty * at(x0 + 1, y0 + 1);
            ++cnt;
        }
    }
    acc[threadIdx.x] = sum;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) acc[threadIdx.x] += acc[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int total = (I->kind == LBM_SLAB) ? 2 * nx : 64;
        prof[(size_t)i * nb + kb] = acc[0] / total;
    }
    (void)cnt;
}

}  // namespace lbm

using namespace lbm;

struct lbm_batch {
    int n;
    int collision, forcing;
    double s_e, s_eps, s_q;
    cudaStream_t stream;
    std::vector<BInst> hinst;
    BInst* dinst = nullptr;
    float* f[2] = {nullptr, nullptr};
    int cur = 0;
    double* rho = nullptr;       // FP64 density output / profiles input
    Snap* snap = nullptr;
    BPart* parts = nullptr;
    BTile* tiles = nullptr;
    int ntiles = 0;
    BItem* items = nullptr;
    int nitems = 0;
    int items_cap = 0;
    int items_for = 0;           // running instances when the work items were last built
    int* state = nullptr;        // device
    int* fail = nullptr;         // device
    unsigned* status = nullptr;  // device, per instance
    int* queue = nullptr;        // device: the step's work-item counter and walkers-done counter
    BObs* obs = nullptr;         // device
    ProbeHist* probe_prev = nullptr;   // device: coexistence probes at the previous check, and their changes then
    int coex_rule = LBM_COEX_CHANGE;
    // pinned host mirrors
    int* h_state = nullptr;
    int* h_fail = nullptr;
    BObs* h_obs = nullptr;
    std::vector<long long> steps;
    long long total_steps = 0;
    // tuning
    int cols = 128;              // strip width of a work item: 128 (one warp), 256 or 512 (a CTA)
    int ns = 3;                  // stages per warp (3 or 4; 2 or 3 with carry)
    int carry = 0;               // rows carried in registers from the psi pass to the collision
    int rows = 64;               // rows per work item
    int grid = 0;
    // graph cache
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long g_every = 0;
    double g_tol_v = 0, g_tol_rho = 0, g_tol_coex = 0;
};

namespace {

int cuda_ok(cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    std::fprintf(stderr, "liblbm (batch): CUDA error %s\n", cudaGetErrorString(e));
    return LBM_E_CUDA;
}
#define B_CUDA(call)                     \
    do {                                 \
        int s_ = cuda_ok(call);          \
        if (s_ != LBM_OK) return s_;     \
    } while (0)

void drop_graphs(lbm_batch* b)
{
    for (auto& g : b->gexec)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

// Work items of the running instances: strips of b->cols columns cut into
// row chunks of about b->rows rows.  When the running instances hold too few strip rows
// to give every SM about sixteen items at that length (small batches, and
// the tail of a run when a few instances remain), the chunks shrink -- down
// to 16 rows -- so a step is spread over more warps (up to the 14-16 a
// batched-step SM holds) and its latency (one row walk) shortens.
int build_items(lbm_batch* b, const int* host_state)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
    }
    long long strip_rows = 0;
    for (int i = 0; i < b->n; ++i) {
        if (host_state && host_state[i] != B_RUNNING) continue;
        const BInst& I = b->hinst[i];
        strip_rows += (long long)((I.nx + b->cols - 1) / b->cols) * I.ny;
    }
    // About 16 items per SM: while many instances run, items of the tuned
    // height; as they converge, shorter ones (down to 4 rows), so that the
    // last few instances still spread over the whole GPU.
    const long long target = 16LL * nsm;
    const int rows = (int)std::max<long long>(std::min<long long>(b->rows, strip_rows / target), std::min(4, b->rows));
    std::vector<BItem> it;
    b->items_for = 0;
    for (int i = 0; i < b->n; ++i) {
        if (host_state && host_state[i] != B_RUNNING) continue;
        b->items_for += 1;
        const BInst& I = b->hinst[i];
        const int nstrips = (I.nx + b->cols - 1) / b->cols;
        const int nch = std::max(1, (I.ny + rows / 2) / rows);
        for (int c = 0; c < nch; ++c) {
            const int y0 = int((long long)c * I.ny / nch), y1 = int((long long)(c + 1) * I.ny / nch);
            if (y1 <= y0) continue;
            for (int s = 0; s < nstrips; ++s) it.push_back(BItem{i, s * b->cols, y0, y1, c & 1, {0, 0, 0}});
        }
    }
    // longest items first, so the walkers taking them from the queue finish evenly
    std::stable_sort(it.begin(), it.end(), [](const BItem& a, const BItem& c) { return (a.y1 - a.y0) > (c.y1 - c.y0); });
    if ((int)it.size() > b->items_cap) {
        if (b->items) cudaFree(b->items);
        b->items_cap = std::max<int>(it.size(), 1);
        B_CUDA(cudaMalloc(&b->items, sizeof(BItem) * b->items_cap));
    }
    b->nitems = (int)it.size();
    if (b->nitems)
        B_CUDA(cudaMemcpyAsync(b->items, it.data(), sizeof(BItem) * b->nitems, cudaMemcpyHostToDevice, b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    drop_graphs(b);
    return LBM_OK;
}

template <int COLL, int FORC, int NS, bool CARRY>
int launch_batch_step(lbm_batch* b, const float* fin, float* fout)
{
    constexpr size_t smem = batch_smem<NS>();
    auto kern = k_step_batch<COLL, FORC, NS, CARRY>;
    static int per_sm = 0, nsm = 0;
    if (per_sm == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return LBM_E_CUDA;
        int dev = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * kBatchWarps, smem) != cudaSuccess || occ < 1)
            occ = 1;
        per_sm = occ;
    }
    if (b->nitems == 0) return LBM_OK;
    const int want = (b->nitems + kBatchWarps - 1) / kBatchWarps;
    const int grid = std::max(1, std::min(nsm * per_sm, want));
    kern<<<grid, 32 * kBatchWarps, smem, b->stream>>>(fin, fout, b->dinst, b->items, b->nitems, b->state, b->status,
                                                       b->queue);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}

template <int NS, bool CARRY>
int launch_batch_scheme(lbm_batch* b, const float* fin, float* fout)
{
    if (b->collision == LBM_MRT) return launch_batch_step<MRT, GUO, NS, CARRY>(b, fin, fout);
    if (b->forcing == LBM_GUO) return launch_batch_step<BGK, GUO, NS, CARRY>(b, fin, fout);
    if (b->forcing == LBM_EDM) return launch_batch_step<BGK, EDM, NS, CARRY>(b, fin, fout);
    if (b->forcing == LBM_LI) return launch_batch_step<BGK, LI, NS, CARRY>(b, fin, fout);
    return launch_batch_step<BGK, SC, NS, CARRY>(b, fin, fout);
}

// The step with the batch's tuning: block-wide walks of wider strips, or
// one-warp walks with ns stages, rows carried in registers or re-read from
// the stage ring.
int launch_batch_tuned(lbm_batch* b, const float* fin, float* fout)
{
    if (b->cols != 128)
        return launch_batch_block(b->cols, b->ns, b->collision, b->forcing,
                                  BatchLaunch{fin, fout, b->dinst, b->items, b->nitems, b->state, b->status, b->queue,
                                              b->stream});
    if (b->carry) return b->ns == 3 ? launch_batch_scheme<3, true>(b, fin, fout)
                                    : launch_batch_scheme<2, true>(b, fin, fout);
    return b->ns == 4 ? launch_batch_scheme<4, false>(b, fin, fout) : launch_batch_scheme<3, false>(b, fin, fout);
}

int step_once(lbm_batch* b)
{
    const float* fin = b->f[b->cur];
    float* fout = b->f[b->cur ^ 1];
    const int s = launch_batch_tuned(b, fin, fout);
    if (s != LBM_OK) return s;
    b->cur ^= 1;
    return LBM_OK;
}

// mode: BO_* flags; decide: apply the convergence / failure decision.
int observe(lbm_batch* b, int mode, double tol_v, double tol_rho, double tol_coex, int decide)
{
    if (b->ntiles) {
        k_observe_batch<<<b->ntiles, GTX * GTY, 0, b->stream>>>(b->f[b->cur], b->dinst, b->tiles, b->state, b->snap,
                                                               b->rho, b->parts, b->obs, mode);
        B_CUDA(cudaGetLastError());
    }
    k_reduce_batch<<<b->n, 256, 0, b->stream>>>(b->dinst, b->parts, b->state, b->fail, b->status, b->obs,
                                                 b->probe_prev, tol_v, tol_rho, tol_coex, b->coex_rule, decide,
                                                 (mode & BO_ALL) ? 1 : 0);
    B_CUDA(cudaGetLastError());
    B_CUDA(cudaMemcpyAsync(b->h_state, b->state, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(cudaMemcpyAsync(b->h_fail, b->fail, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(cudaMemcpyAsync(b->h_obs, b->obs, sizeof(BObs) * b->n, cudaMemcpyDeviceToHost, b->stream));
    return LBM_OK;
}

// One check interval: `every` steps, then observe + decide.  Captured once in
// a CUDA graph per buffer parity and replayed.
int interval(lbm_batch* b, long long every, double tol_v, double tol_rho, double tol_coex)
{
    if (b->g_every != every || b->g_tol_v != tol_v || b->g_tol_rho != tol_rho || b->g_tol_coex != tol_coex) {
        drop_graphs(b);
        b->g_every = every;
        b->g_tol_v = tol_v;
        b->g_tol_rho = tol_rho;
        b->g_tol_coex = tol_coex;
    }
    const int parity = b->cur;
    if (!b->gexec[parity]) {
        cudaGraph_t graph;
        B_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int s = LBM_OK;
        for (long long i = 0; i < every && s == LBM_OK; ++i) s = step_once(b);
        if (s == LBM_OK) s = observe(b, BO_SNAP, tol_v, tol_rho, tol_coex, 1);
        const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        b->cur = parity;   // capture recorded the launches; the state did not move
        if (s != LBM_OK) return s;
        B_CUDA(e);
        const cudaError_t ie = cudaGraphInstantiate(&b->gexec[parity], graph, 0);
        cudaGraphDestroy(graph);
        B_CUDA(ie);
    }
    B_CUDA(cudaGraphLaunch(b->gexec[parity], b->stream));
    if (every & 1) b->cur ^= 1;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_batch_params* bp, const lbm_instance* inst, int n, lbm_batch** out)
{
    if (!bp || !inst || n < 1 || !out) return LBM_E_INVALID;
    *out = nullptr;
    if (bp->precision != LBM_FP32_DEV) return LBM_E_UNSUPPORTED;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_E_INVALID;
    b->n = n;
    b->collision = bp->collision;
    b->forcing = bp->forcing;
    b->s_e = bp->s_e;
    b->s_eps = bp->s_eps;
    b->s_q = bp->s_q;
    long long off = 0, node_off = 0;
    int tile_off = 0;
    std::vector<BTile> tiles;
    for (int i = 0; i < n; ++i) {
        const lbm_instance& in = inst[i];
        lbm_params p;
        std::memset(&p, 0, sizeof(p));
        p.nx = in.nx;
        p.ny = in.ny;
        p.collision = bp->collision;
        p.forcing = bp->forcing;
        p.precision = LBM_FP32_DEV;
        p.T_over_Tc = in.T_over_Tc;
        p.tau = in.tau;
        p.A = in.A;
        p.K = in.K;
        p.s_e = bp->s_e;
        p.s_eps = bp->s_eps;
        p.s_q = bp->s_q;
        p.sigma = bp->sigma;
        double rv = in.rho_v, rl = in.rho_l;
        if (rv <= 0 || rl <= 0) {
            if (lbm_maxwell(in.T_over_Tc, &rv, &rl) != LBM_OK) { delete b; return LBM_E_INVALID; }
        }
        p.rho_ref = rv;
        int v = lbm_validate_params(&p);
        if (v == LBM_OK && (in.nx % 4 != 0)) v = LBM_E_UNSUPPORTED;
        if (v == LBM_OK && (in.kind < LBM_SLAB || in.kind > LBM_DROPLET_ARRAY || !(in.width > 0) ||
                            (in.kind == LBM_DROPLET_ARRAY && in.cell < 1)))
            v = LBM_E_INVALID;
        if (v != LBM_OK) { delete b; return v; }
        BInst I;
        std::memset(&I, 0, sizeof(I));
        I.off = off;
        I.node_off = node_off;
        I.nx = in.nx;
        I.ny = in.ny;
        I.tile_off = tile_off;
        I.ntx = (in.nx + GTX - 1) / GTX;
        I.nty = (in.ny + GTY - 1) / GTY;
        I.kind = in.kind;
        I.cell = in.cell;
        I.size = in.size;
        I.width = in.width;
        I.rho_l = rl;
        I.rho_v = rv;
        I.noise_amp = in.noise_amp;
        I.seed = in.seed;
        I.k = make_coef<float>(p);
        for (int ty = 0; ty < I.nty; ++ty)
            for (int tx = 0; tx < I.ntx; ++tx) tiles.push_back(BTile{i, tx, ty});
        tile_off += I.ntx * I.nty;
        const long long nodes = (long long)in.nx * in.ny;
        off += (9 * nodes + 63) / 64 * 64;          // 256-byte aligned blocks
        node_off += (nodes + 31) / 32 * 32;
        b->hinst.push_back(I);
    }
    b->ntiles = (int)tiles.size();
    b->steps.assign(n, 0);
    auto fail = [&](cudaError_t e) { lbm_batch_destroy(b); return cuda_ok(e); };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) { delete b; return cuda_ok(e); }
    if ((e = cudaMalloc(&b->dinst, sizeof(BInst) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->f[0], sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->f[1], sizeof(float) * off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->rho, sizeof(double) * node_off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->snap, sizeof(Snap) * node_off)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->parts, sizeof(BPart) * std::max(1, b->ntiles))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->tiles, sizeof(BTile) * std::max(1, b->ntiles))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->state, sizeof(int) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->fail, sizeof(int) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->status, sizeof(unsigned) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->queue, sizeof(int) * 2)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(b->queue, 0, sizeof(int) * 2)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->obs, sizeof(BObs) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->probe_prev, sizeof(ProbeHist) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost(&b->h_state, sizeof(int) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost(&b->h_fail, sizeof(int) * n)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost(&b->h_obs, sizeof(BObs) * n)) != cudaSuccess) return fail(e);
    cudaMemcpyAsync(b->dinst, b->hinst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->tiles, tiles.data(), sizeof(BTile) * b->ntiles, cudaMemcpyHostToDevice, b->stream);
    cudaMemsetAsync(b->f[0], 0, sizeof(float) * off, b->stream);
    cudaMemsetAsync(b->f[1], 0, sizeof(float) * off, b->stream);
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return fail(e);
    int s = build_items(b, nullptr);
    // one-time kernel set-up (shared-memory attribute, occupancy) outside any graph capture
    const int saved = b->nitems;
    b->nitems = 0;
    if (s == LBM_OK) s = launch_batch_scheme<3, false>(b, b->f[0], b->f[1]);
    if (s == LBM_OK) s = launch_batch_scheme<4, false>(b, b->f[0], b->f[1]);
    if (s == LBM_OK) s = launch_batch_scheme<2, true>(b, b->f[0], b->f[1]);
    if (s == LBM_OK) s = launch_batch_scheme<3, true>(b, b->f[0], b->f[1]);
    b->nitems = saved;
    if (s != LBM_OK) { lbm_batch_destroy(b); return s; }
    std::fill(b->h_state, b->h_state + b->n, (int)B_RUNNING);
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    cudaFree(b->dinst);
    cudaFree(b->f[0]);
    cudaFree(b->f[1]);
    cudaFree(b->rho);
    cudaFree(b->snap);
    cudaFree(b->parts);
    cudaFree(b->tiles);
    cudaFree(b->items);
    cudaFree(b->state);
    cudaFree(b->fail);
    cudaFree(b->status);
    cudaFree(b->queue);
    cudaFree(b->obs);
    cudaFree(b->probe_prev);
    cudaFreeHost(b->h_state);
    cudaFreeHost(b->h_fail);
    cudaFreeHost(b->h_obs);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

static int reset_run_state(lbm_batch* b)
{
    B_CUDA(cudaMemsetAsync(b->state, 0, sizeof(int) * b->n, b->stream));
    B_CUDA(cudaMemsetAsync(b->fail, 0, sizeof(int) * b->n, b->stream));
    B_CUDA(cudaMemsetAsync(b->status, 0, sizeof(unsigned) * b->n, b->stream));
    B_CUDA(cudaMemsetAsync(b->obs, 0, sizeof(BObs) * b->n, b->stream));
    B_CUDA(cudaMemsetAsync(b->probe_prev, 0xff, sizeof(ProbeHist) * b->n, b->stream));   // NaN: no previous check
    long long nodes = 0;
    for (const BInst& I : b->hinst) nodes = std::max<long long>(nodes, I.node_off + (long long)I.nx * I.ny);
    B_CUDA(cudaMemsetAsync(b->snap, 0xff, sizeof(Snap) * nodes, b->stream));   // NaN: no snapshot yet
    std::fill(b->steps.begin(), b->steps.end(), 0);
    b->total_steps = 0;
    b->cur = 0;
    drop_graphs(b);
    B_CUDA(cudaStreamSynchronize(b->stream));
    std::fill(b->h_state, b->h_state + b->n, (int)B_RUNNING);
    return build_items(b, nullptr);
}

// Copy n profile grids to the device (caller frees); nullptr on failure.
static BGeom* device_geom(lbm_batch* b, const lbm_profile_geom* g)
{
    std::vector<BGeom> h(b->n);
    for (int i = 0; i < b->n; ++i) h[i] = BGeom{g[i].use ? 1 : 0, 0, g[i].centre, g[i].spacing};
    BGeom* d = nullptr;
    if (cudaMalloc(&d, sizeof(BGeom) * b->n) != cudaSuccess) return nullptr;
    if (cudaMemcpyAsync(d, h.data(), sizeof(BGeom) * b->n, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    return d;
}

// rho0 into the FP64 node array, then (rest) u0 into the snapshot array's
// velocity slots, then the populations; the snapshot is cleared again after.
static int init_fields(lbm_batch* b, const double* prof, int nb, const BGeom* dgeom, bool rest)
{
    int s = reset_run_state(b);
    if (s != LBM_OK) return s;
    const dim3 grid(64, b->n);
    k_rho0_batch<<<grid, 256, 0, b->stream>>>(b->dinst, b->n, b->rho, prof, dgeom, nb);
    if (rest) k_rest_velocity<<<grid, 256, 0, b->stream>>>(b->dinst, b->n, b->rho, dgeom, b->snap);
    k_pops_batch<<<grid, 256, 0, b->stream>>>(b->dinst, b->n, b->f[0], b->rho, rest ? b->snap : nullptr,
                                              prof ? dgeom : nullptr);
    B_CUDA(cudaGetLastError());
    if (rest) {
        long long nodes = 0;
        for (const BInst& I : b->hinst) nodes = std::max<long long>(nodes, I.node_off + (long long)I.nx * I.ny);
        B_CUDA(cudaMemsetAsync(b->snap, 0xff, sizeof(Snap) * nodes, b->stream));   // NaN: no snapshot yet
    }
    B_CUDA(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_init(lbm_batch* b)
{
    if (!b) return LBM_E_INVALID;
    return init_fields(b, nullptr, 0, nullptr, false);
}

int lbm_batch_init_profiles(lbm_batch* b, const double* profiles_dev, int nb, const lbm_profile_geom* geom_host,
                            int flags)
{
    if (!b || !profiles_dev || !geom_host || nb < 2 || nb > 4096 || (flags & ~LBM_INIT_REST)) return LBM_E_INVALID;
    for (int i = 0; i < b->n; ++i)
        if (geom_host[i].use && !(std::isfinite(geom_host[i].centre) && geom_host[i].spacing > 0 &&
                                  std::isfinite(geom_host[i].spacing)))
            return LBM_E_INVALID;
    BGeom* dgeom = device_geom(b, geom_host);
    if (!dgeom) return LBM_E_CUDA;
    const int s = init_fields(b, profiles_dev, nb, dgeom, (flags & LBM_INIT_REST) != 0);
    cudaFree(dgeom);
    return s;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps)
{
    if (!b || nsteps < 0) return LBM_E_INVALID;
    for (int64_t i = 0; i < nsteps; ++i) {
        const int s = step_once(b);
        if (s != LBM_OK) return s;
    }
    for (int i = 0; i < b->n; ++i)
        if (b->h_state[i] == B_RUNNING) b->steps[i] += nsteps;
    b->total_steps += nsteps;
    B_CUDA(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_observe(lbm_batch* b)
{
    if (!b) return LBM_E_INVALID;
    const int s = observe(b, BO_RHO | BO_ALL, 0, 0, 0, 0);
    if (s != LBM_OK) return s;
    B_CUDA(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_run_to_steady(lbm_batch* b, double tol_v, double tol_rho, double tol_coex, int64_t check_every,
                            int64_t max_steps, int64_t* steps_done)
{
    if (!b || check_every < 1 || max_steps < 0 || (!(tol_v > 0) && !(tol_rho > 0) && !(tol_coex > 0)))
        return LBM_E_INVALID;
    int64_t done = 0;
    int active = 0;
    for (int i = 0; i < b->n; ++i) active += b->h_state[i] == B_RUNNING;
    std::vector<int> before(b->n);
    while (done < max_steps && active > 0) {
        const int64_t k = std::min<int64_t>(check_every, max_steps - done);
        std::copy(b->h_state, b->h_state + b->n, before.begin());   // the graph's copy-out rewrites h_state
        int s;
        if (k == check_every) {
            s = interval(b, k, tol_v, tol_rho, tol_coex);
        } else {   // last partial interval: plain launches
            s = LBM_OK;
            for (int64_t i = 0; i < k && s == LBM_OK; ++i) s = step_once(b);
            if (s == LBM_OK) s = observe(b, BO_SNAP, tol_v, tol_rho, tol_coex, 1);
        }
        if (s != LBM_OK) return s;
        B_CUDA(cudaStreamSynchronize(b->stream));             // h_state now holds the decision of this interval
        for (int i = 0; i < b->n; ++i)
            if (before[i] == B_RUNNING) b->steps[i] += k;
        done += k;
        b->total_steps += k;
        active = 0;
        for (int i = 0; i < b->n; ++i) active += b->h_state[i] == B_RUNNING;
        if (active > 0 && active * 4 < b->items_for * 3) {   // compact the work items to the running instances
            s = build_items(b, b->h_state);
            if (s != LBM_OK) return s;
        }
    }
    if (steps_done) *steps_done = done;
    return active == 0 ? LBM_OK : LBM_E_NOT_CONVERGED;
}

int lbm_batch_set_coex_rule(lbm_batch* b, int rule)
{
    if (!b || (rule != LBM_COEX_CHANGE && rule != LBM_COEX_TAIL)) return LBM_E_INVALID;
    if (rule != b->coex_rule) {
        b->coex_rule = rule;
        drop_graphs(b);   // the captured intervals carry the rule as a kernel argument
    }
    return LBM_OK;
}

int lbm_batch_results(lbm_batch* b, int32_t* state, int32_t* code, int64_t* steps, double* obs)
{
    if (!b) return LBM_E_INVALID;
    for (int i = 0; i < b->n; ++i) {
        if (state) state[i] = b->h_state[i];
        if (code) code[i] = b->h_fail[i];
        if (steps) steps[i] = b->steps[i];
        if (obs) std::memcpy(obs + (size_t)i * LBM_BATCH_NOBS, &b->h_obs[i], sizeof(double) * LBM_BATCH_NOBS);
    }
    return LBM_OK;
}

int lbm_batch_read_density(lbm_batch* b, int i, double* rho_host)
{
    if (!b || i < 0 || i >= b->n || !rho_host) return LBM_E_INVALID;
    const int s = observe(b, BO_RHO | BO_ALL, 0, 0, 0, 0);
    if (s != LBM_OK) return s;
    const BInst& I = b->hinst[i];
    B_CUDA(cudaMemcpyAsync(rho_host, b->rho + I.node_off, sizeof(double) * I.nx * I.ny, cudaMemcpyDeviceToHost,
                           b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_profiles(lbm_batch* b, int nb, const lbm_profile_geom* geom_host, double* prof_host)
{
    if (!b || nb < 2 || nb > 4096 || !geom_host || !prof_host) return LBM_E_INVALID;
    for (int i = 0; i < b->n; ++i)
        if (!(std::isfinite(geom_host[i].centre) && std::isfinite(geom_host[i].spacing))) return LBM_E_INVALID;
    BGeom* dgeom = device_geom(b, geom_host);
    if (!dgeom) return LBM_E_CUDA;
    double* dprof = nullptr;
    if (cudaMalloc(&dprof, sizeof(double) * nb * b->n) != cudaSuccess) {
        cudaFree(dgeom);
        return LBM_E_CUDA;
    }
    int s = observe(b, BO_RHO | BO_ALL, 0, 0, 0, 0);
    if (s == LBM_OK) {
        k_radial_profile<<<dim3(nb, b->n), 128, 0, b->stream>>>(b->dinst, b->rho, nb, dgeom, dprof);
        s = cuda_ok(cudaGetLastError());
    }
    if (s == LBM_OK)
        s = cuda_ok(cudaMemcpyAsync(prof_host, dprof, sizeof(double) * nb * b->n, cudaMemcpyDeviceToHost, b->stream));
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    cudaFree(dprof);
    cudaFree(dgeom);
    if (s != LBM_OK) return s;
    return cuda_ok(e);
}

int lbm_batch_set_tuning(lbm_batch* b, int columns, int stages, int rows_per_item, int carry)
{
    if (!b || rows_per_item < 8) return LBM_E_INVALID;
    if (columns == 128) {
        if (carry ? (stages != 2 && stages != 3) : (stages != 3 && stages != 4)) return LBM_E_INVALID;
    } else if (!carry || !((columns == 256 && stages == 3) || (columns == 512 && (stages == 2 || stages == 3)))) {
        return LBM_E_INVALID;
    }
    b->cols = columns;
    b->ns = stages;
    b->carry = carry ? 1 : 0;
    b->rows = rows_per_item;
    return build_items(b, b->h_state);
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, int* columns, int* stages, int* rows_per_item, int* carry,
                       double* ms_per_step)
{
    if (!b || trial_steps < 1) return LBM_E_INVALID;
    cudaEvent_t e0, e1;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    // (columns, stages, carry): the one-warp walks, then the block walks
    constexpr int ncand = 7;
    const int cand_cols[ncand] = {128, 128, 128, 128, 256, 512, 512};
    const int cand_ns[ncand] = {3, 4, 2, 3, 3, 2, 3};
    const int cand_carry[ncand] = {0, 0, 1, 1, 1, 1, 1};
    const int cand_rows[4] = {32, 64, 128, 256};
    float best = 3.4e38f;
    int bcols = b->cols, bns = b->ns, brows = b->rows, bcarry = b->carry;
    int status = LBM_OK;
    const int cur0 = b->cur;
    for (int ci = 0; ci < ncand && status == LBM_OK; ++ci)
        for (int ri = 0; ri < 4 && status == LBM_OK; ++ri) {
            b->cols = cand_cols[ci];
            b->ns = cand_ns[ci];
            b->carry = cand_carry[ci];
            b->rows = cand_rows[ri];
            if ((status = build_items(b, b->h_state)) != LBM_OK) break;
            // trials read the current state and write the spare buffer only
            const float* fin = b->f[cur0];
            float* fout = b->f[cur0 ^ 1];
            auto one = [&]() { return launch_batch_tuned(b, fin, fout); };
            if ((status = one()) != LBM_OK) break;
            cudaEventRecord(e0, b->stream);
            for (int i = 0; i < trial_steps && status == LBM_OK; ++i) status = one();
            cudaEventRecord(e1, b->stream);
            if ((status = cuda_ok(cudaEventSynchronize(e1))) != LBM_OK) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= trial_steps;
            if (ms < best) { best = ms; bcols = b->cols; bns = b->ns; brows = b->rows; bcarry = b->carry; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cur = cur0;
    b->cols = bcols;
    b->ns = bns;
    b->rows = brows;
    b->carry = bcarry;
    const int s = build_items(b, b->h_state);
    if (status != LBM_OK) return status;
    if (s != LBM_OK) return s;
    if (columns) *columns = bcols;
    if (stages) *stages = bns;
    if (rows_per_item) *rows_per_item = brows;
    if (carry) *carry = bcarry;
    if (ms_per_step) *ms_per_step = best;
    return LBM_OK;
}

int64_t lbm_batch_nodes(lbm_batch* b)
{
    if (!b) return -1;
    int64_t s = 0;
    for (const BInst& I : b->hinst) s += (int64_t)I.nx * I.ny;
    return s;
}

}  // extern "C"
