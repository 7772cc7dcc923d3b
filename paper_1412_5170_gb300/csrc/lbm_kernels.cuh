// lbm_kernels.cuh -- device kernels of liblbm and the host-side launch
// helpers they share.  Population buffers hold post-collision deviations
// f*_a(x, t-1) - w_a rho_ref in the pull convention: the population that
// arrives at x at time t is f*_a(x - e_a, t-1) (Eq. 1 / Eq. 36 streaming).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// FP64 reduction record, one per block of the observe kernel.
struct Partial {
    double mass, row_mid, row0;
    double max_v, max_dv, rho_max, neg_rho_min;
    unsigned status, pad;
};

// Device copy of the lattice observables (mirrors lbm_stats).
struct DevStats {
    double mass, max_v, max_dv, rho_min, rho_max;
    double rho_center, rho_corner, rho_row_mid, rho_row0;
    unsigned status, pad;
};

__device__ __forceinline__ int wrap_any(int v, int n) { int r = v % n; return r < 0 ? r + n : r; }
// x in [0, n): x - 1 and x + 1 with periodic wrap (valid for any n >= 1).
__device__ __forceinline__ int dec1(int x, int n) { return x == 0 ? n - 1 : x - 1; }
__device__ __forceinline__ int inc1(int x, int n) { return x == n - 1 ? 0 : x + 1; }

// Pulled deviations at node (x, y): g_a = f*_a(x - e_a, y - e_a).
template <typename T, typename C>
__device__ __forceinline__ void pull_node(const T* __restrict__ f, int x, int y, int nx, int ny, size_t n, C g[9])
{
    const int xm = dec1(x, nx), xp = inc1(x, nx);
    const int ym = dec1(y, ny), yp = inc1(y, ny);
    const size_t r0 = (size_t)y * nx, rm = (size_t)ym * nx, rp = (size_t)yp * nx;
    g[0] = C(f[0 * n + r0 + x]);
    g[1] = C(f[1 * n + r0 + xm]);
    g[2] = C(f[2 * n + rm + x]);
    g[3] = C(f[3 * n + r0 + xp]);
    g[4] = C(f[4 * n + rp + x]);
    g[5] = C(f[5 * n + rm + xm]);
    g[6] = C(f[6 * n + rm + xp]);
    g[7] = C(f[7 * n + rp + xp]);
    g[8] = C(f[8 * n + rp + xm]);
}

template <typename C>
__device__ __forceinline__ C sum9(const C g[9])
{
    if constexpr (sizeof(C) == sizeof(float))
        return g[0] + moving_sum(g);   // the FP32 collision's density, same order
    else
        return ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
}

__device__ __forceinline__ void flag_status(unsigned bad, unsigned* status)
{
    const unsigned w = __reduce_or_sync(0xffffffffu, bad);
    if (w && (threadIdx.x & 31) == 0) atomicOr(status, w);
}

// ---------------------------------------------------------------------------
// Generic fused step: one node per thread on a TX x TY tile.  psi on the tile
// plus a one-node ring is computed from pulled populations into shared
// memory, then each thread computes F from the psi stencil, collides and
// writes its nine post-collision deviations.  Works for any nx, ny >= 1.
// ---------------------------------------------------------------------------
constexpr int GTX = 32, GTY = 8;

template <typename T, typename C, int COLL, int FORC>
__global__ void __launch_bounds__(GTX * GTY)
k_step_generic(const T* __restrict__ fin, T* __restrict__ fout, int nx, int ny, Coef<C> k,
               unsigned* __restrict__ status)
{
    __shared__ C sp[(GTY + 2) * (GTX + 2)];
    const int x0 = blockIdx.x * GTX, y0 = blockIdx.y * GTY;
    const size_t n = (size_t)nx * ny;
    unsigned bad = 0;
    for (int i = threadIdx.x; i < (GTX + 2) * (GTY + 2); i += blockDim.x) {
        const int x = wrap_any(x0 + i % (GTX + 2) - 1, nx);
        const int y = wrap_any(y0 + i / (GTX + 2) - 1, ny);
        C g[9];
        pull_node<T, C>(fin, x, y, nx, ny, n, g);
        sp[i] = psi_of_rho<C>(k.rho_ref + sum9(g), k, bad);
    }
    __syncthreads();
    const int tx = threadIdx.x % GTX, ty = threadIdx.x / GTX;
    const int x = x0 + tx, y = y0 + ty;
    if (x < nx && y < ny) {
        C g[9];
        pull_node<T, C>(fin, x, y, nx, ny, n, g);
        const int W = GTX + 2, c = (ty + 1) * W + tx + 1;
        Stencil<C> q{sp[c], sp[c + 1], sp[c + W], sp[c - 1], sp[c - W],
                     sp[c + W + 1], sp[c + W - 1], sp[c - W - 1], sp[c - W + 1]};
        C Fx, Fy, vx, vy, rho;
        force<C>(q, k, Fx, Fy);
        collide<C, COLL, FORC>(g, Fx, Fy, k, vx, vy, rho, q.c);
        bad |= finite_bits<C>(g);
        const size_t o = (size_t)y * nx + x;
#pragma unroll
        for (int a = 0; a < 9; ++a) fout[a * n + o] = T(g[a]);
    }
    flag_status(bad, status);
}

// ---------------------------------------------------------------------------
// Observe: rho, v = u + F/(2 rho) at time t for every node, optional FP64
// field output, optional snapshot compare/store, and one FP64 Partial per
// block (fixed-order warp-shuffle + shared-memory tree: deterministic).
// ---------------------------------------------------------------------------
enum : int { OBS_FIELDS = 1, OBS_REDUCE = 2, OBS_SNAP_CMP = 4, OBS_SNAP_STORE = 8 };

// Velocity snapshot of one node in the compute type (v is computed in it, so
// a float snapshot of the FP32 path loses nothing).
template <typename C> struct VSnapOf;
template <> struct VSnapOf<float> { using type = float2; };
template <> struct VSnapOf<double> { using type = double2; };
template <typename C> using VSnap = typename VSnapOf<C>::type;
__device__ __forceinline__ float2 make_vsnap(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 make_vsnap(double x, double y) { return make_double2(x, y); }

// rho - rho_ref and v = u + F/(2 rho) of one node from its pulled deviations
// (Eq. 3 and Sec. 3.2), as every observation computes them (FP32: the
// reciprocal Newton-refined).
template <typename C>
__device__ __forceinline__ void node_velocity(const C g[9], C Fx, C Fy, const Coef<C>& k, C& drho, C& vx, C& vy)
{
    C jx, jy;
    moments<C>(g, drho, jx, jy);
    const C rc = k.rho_ref + drho;
    if constexpr (sizeof(C) == sizeof(float)) {
        const float inv = rcp_nr(rc);
        vx = fma_rn(0.5f * Fx, inv, jx * inv);
        vy = fma_rn(0.5f * Fy, inv, jy * inv);
    } else {
        vx = jx / rc + C(0.5) * Fx / rc;
        vy = jy / rc + C(0.5) * Fy / rc;
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename C> __device__ __forceinline__ C obs_huge();
template <> __device__ __forceinline__ double obs_huge<double>() { return 1e300; }
template <> __device__ __forceinline__ float obs_huge<float>() { return 1e30f; }

// The per-node work stays in the compute type C: |v|, |v - v_snap| and the
// density extremes (tracked as max drho and max -drho, then rho = rho_ref +
// drho once per block -- exact, since that sum rounds monotonically in drho)
// are maxima, which are exact in any precision, so only the mass and the two
// probe-row sums need FP64 arithmetic; the row sums are taken only by the
// warps that hold those rows (a warp is one tile row).  This keeps the FP32
// path off the FP64 pipe, which is narrow on this GPU.
template <typename T, typename C>
__global__ void __launch_bounds__(GTX * GTY)
k_observe(const T* __restrict__ fin, int nx, int ny, Coef<C> k, int mode,
          double* __restrict__ rho_o, double* __restrict__ vx_o, double* __restrict__ vy_o,
          VSnap<C>* __restrict__ vsnap, Partial* __restrict__ parts, DevStats* __restrict__ ds,
          const unsigned* __restrict__ status)
{
    __shared__ C sp[(GTY + 2) * (GTX + 2)];
    __shared__ double red[7][GTX * GTY / 32];
    const int x0 = blockIdx.x * GTX, y0 = blockIdx.y * GTY;
    const size_t n = (size_t)nx * ny;
    unsigned bad = 0;
    for (int i = threadIdx.x; i < (GTX + 2) * (GTY + 2); i += blockDim.x) {
        const int x = wrap_any(x0 + i % (GTX + 2) - 1, nx);
        const int y = wrap_any(y0 + i / (GTX + 2) - 1, ny);
        C g[9];
        pull_node<T, C>(fin, x, y, nx, ny, n, g);
        sp[i] = psi_of_rho<C>(k.rho_ref + sum9(g), k, bad);
    }
    __syncthreads();
    const int tx = threadIdx.x % GTX, ty = threadIdx.x / GTX;
    const int x = x0 + tx, y = y0 + ty;
    double mass = 0, rho = 0;
    C mv = 0, mdv = 0, dmax = -obs_huge<C>(), ndmin = -obs_huge<C>();
    if (x < nx && y < ny) {
        C g[9];
        pull_node<T, C>(fin, x, y, nx, ny, n, g);
        const int W = GTX + 2, c = (ty + 1) * W + tx + 1;
        Stencil<C> q{sp[c], sp[c + 1], sp[c + W], sp[c - 1], sp[c - W],
                     sp[c + W + 1], sp[c + W - 1], sp[c - W - 1], sp[c - W + 1]};
        C Fx, Fy, drho, vx, vy;
        force<C>(q, k, Fx, Fy);
        node_velocity<C>(g, Fx, Fy, k, drho, vx, vy);
        rho = double(k.rho_ref) + double(drho);
        if (!isfinite(drho) || !isfinite(vx) || !isfinite(vy)) bad |= ST_NONFINITE;
        const size_t o = (size_t)y * nx + x;
        if (mode & OBS_FIELDS) {
            if (rho_o) rho_o[o] = rho;
            if (vx_o) vx_o[o] = double(vx);
            if (vy_o) vy_o[o] = double(vy);
        }
        if (mode & OBS_SNAP_CMP) {
            const VSnap<C> s = vsnap[o];
            const C dx = vx - C(s.x), dy = vy - C(s.y);
            mdv = sqrt(dx * dx + dy * dy);
            if (isnan(mdv)) mdv = obs_huge<C>();
        }
        if (mode & OBS_SNAP_STORE) vsnap[o] = make_vsnap(vx, vy);
        mass = rho;
        mv = sqrt(vx * vx + vy * vy);
        if (isnan(mv)) mv = obs_huge<C>();
        dmax = drho;
        ndmin = -drho;
        if (ds && x == nx / 2 && y == ny / 2) ds->rho_center = rho;
        if (ds && x == 0 && y == 0) ds->rho_corner = rho;
    }
    if (mode & OBS_REDUCE) {
        const unsigned allbad = __reduce_or_sync(0xffffffffu, bad);
        const bool mid_row = y == ny / 2, row_0 = y == 0;      // uniform over the warp
        double v[7] = {warp_sum(mass), mid_row ? warp_sum(rho) : 0.0, row_0 ? warp_sum(rho) : 0.0,
                       double(warp_max(mv)), double(warp_max(mdv)), 0.0, 0.0};
        const C wdmax = warp_max(dmax), wndmin = warp_max(ndmin);
        v[5] = double(k.rho_ref) + double(wdmax);
        v[6] = -(double(k.rho_ref) + double(-wndmin));
        __shared__ unsigned sbad;
        if (threadIdx.x == 0) sbad = 0;
        __syncthreads();
        const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < 7; ++j) red[j][wid] = v[j];
            if (allbad) atomicOr(&sbad, allbad);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            constexpr int NW = GTX * GTY / 32;
            Partial p;
            p.mass = p.row_mid = p.row0 = 0;
            p.max_v = p.max_dv = p.rho_max = p.neg_rho_min = -1e300;
            for (int w = 0; w < NW; ++w) {
                p.mass += red[0][w]; p.row_mid += red[1][w]; p.row0 += red[2][w];
                p.max_v = fmax(p.max_v, red[3][w]); p.max_dv = fmax(p.max_dv, red[4][w]);
                p.rho_max = fmax(p.rho_max, red[5][w]); p.neg_rho_min = fmax(p.neg_rho_min, red[6][w]);
            }
            p.status = sbad | (status ? *status : 0u);
            p.pad = 0;
            parts[blockIdx.y * gridDim.x + blockIdx.x] = p;
        }
    }
}

// Fixed-order reduction of the per-block partials into DevStats.
static __global__ void __launch_bounds__(256)
k_reduce_final(const Partial* __restrict__ parts, int nparts, int nx, DevStats* __restrict__ ds)
{
    __shared__ double red[7][256];
    __shared__ unsigned sbad[256];
    double v[7] = {0, 0, 0, -1e300, -1e300, -1e300, -1e300};
    unsigned bad = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const Partial p = parts[i];
        v[0] += p.mass; v[1] += p.row_mid; v[2] += p.row0;
        v[3] = fmax(v[3], p.max_v); v[4] = fmax(v[4], p.max_dv);
        v[5] = fmax(v[5], p.rho_max); v[6] = fmax(v[6], p.neg_rho_min);
        bad |= p.status;
    }
    for (int j = 0; j < 7; ++j) red[j][threadIdx.x] = v[j];
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int o = threadIdx.x + s;
            red[0][threadIdx.x] += red[0][o]; red[1][threadIdx.x] += red[1][o]; red[2][threadIdx.x] += red[2][o];
            for (int j = 3; j < 7; ++j) red[j][threadIdx.x] = fmax(red[j][threadIdx.x], red[j][o]);
            sbad[threadIdx.x] |= sbad[o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ds->mass = red[0][0];
        ds->rho_row_mid = red[1][0] / nx;
        ds->rho_row0 = red[2][0] / nx;
        ds->max_v = red[3][0];
        ds->max_dv = red[4][0];
        ds->rho_max = red[5][0];
        ds->rho_min = -red[6][0];
        ds->status = sbad[0];
    }
}

// ---------------------------------------------------------------------------
// State conversion between post-streaming populations f_a(x, t) (FP64, the
// user-facing form) and the stored pull-convention deviations
// f*_a(x, t-1) - w_a rho_ref = f_a(x + e_a, t) - w_a rho_ref.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_init_rest(const double* __restrict__ rho0, T* __restrict__ fs, int nx, int ny, double rho_ref)
{
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = int(i % nx), y = int(i / nx);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int xs = ex(a) > 0 ? inc1(x, nx) : (ex(a) < 0 ? dec1(x, nx) : x);
            const int ys = ey(a) > 0 ? inc1(y, ny) : (ey(a) < 0 ? dec1(y, ny) : y);
            const double w = wt<double>(a);
            fs[a * n + i] = T(w * rho0[(size_t)ys * nx + xs] - w * rho_ref);
        }
    }
}

// FP32-deviation initial state in two passes, off the FP64 pipe: the density
// deviation of every node once, dev = float(rho0 - rho_ref), then
// g_a(x) = w_a dev(x + e_a) (the stored f*_a(x) of a start at rest).
static __global__ void k_init_dev_f32(const double* __restrict__ rho0, float* __restrict__ dev, size_t n, double rho_ref)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dev[i] = float(rho0[i] - rho_ref);
}

static __global__ void k_init_rest_f32(const float* __restrict__ dev, float* __restrict__ fs, int nx, int ny)
{
    const size_t n = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = int(i % nx), y = int(i / nx);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int xs = ex(a) > 0 ? inc1(x, nx) : (ex(a) < 0 ? dec1(x, nx) : x);
            const int ys = ey(a) > 0 ? inc1(y, ny) : (ey(a) < 0 ? dec1(y, ny) : y);
            fs[a * n + i] = wt<float>(a) * dev[(size_t)ys * nx + xs];
        }
    }
}

// One plane a: stored <- post-streaming (dir = +1) or post-streaming <- stored (dir = -1).
template <typename T>
__global__ void k_plane_convert(T* __restrict__ fs, double* __restrict__ plane, int a, int nx, int ny,
                                double rho_ref, int to_stored)
{
    const size_t n = (size_t)nx * ny;
    const double w = wt<double>(a);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = int(i % nx), y = int(i / nx);
        if (to_stored) {   // fs_a(x) = f_a(x + e_a)
            const int xs = ex(a) > 0 ? inc1(x, nx) : (ex(a) < 0 ? dec1(x, nx) : x);
            const int ys = ey(a) > 0 ? inc1(y, ny) : (ey(a) < 0 ? dec1(y, ny) : y);
            fs[a * n + i] = T(plane[(size_t)ys * nx + xs] - w * rho_ref);
        } else {           // f_a(x) = fs_a(x - e_a)
            const int xs = ex(a) > 0 ? dec1(x, nx) : (ex(a) < 0 ? inc1(x, nx) : x);
            const int ys = ey(a) > 0 ? dec1(y, ny) : (ey(a) < 0 ? inc1(y, ny) : y);
            plane[i] = double(fs[a * n + (size_t)ys * nx + xs]) + w * rho_ref;
        }
    }
}

// The observation with the strip walk (lbm_observe.cu), for lattices the strip
// kernel supports (nx % 4 == 0): mode as k_observe; with OBS_REDUCE the per-CTA
// partials (parts, at least as many as the generic observation's tiles) are
// reduced in the same launch by the last CTA to finish, in a fixed order,
// into ds (ticket: a device counter that is 0 between launches).  vsnap holds
// VSnap<C> of the precision's compute type.
int observe_strip_launch(const lbm_params* p, const void* f, int mode, double* rho, double* vx, double* vy,
                         void* vsnap, Partial* parts, unsigned* ticket, DevStats* ds, const unsigned* status,
                         cudaStream_t s);

}  // namespace lbm
