// lbm_observe.cu -- the lattice observables (rho, v = u + F/(2 rho) at time t,
// FP64 mass, max |v|, max |v - v_snap|, density extremes and probes, status)
// with the strip walk of the time step (lbm_strip.cuh): the same TMA row
// copies, psi ring and pulled populations, but each chunk row is observed
// instead of collided, so a node's populations are read from HBM once
// (36 B per node in FP32, 72 B in FP64) and nothing is written unless the
// moment fields or the velocity snapshot are asked for.
//
// With OBS_REDUCE every CTA leaves one FP64 Partial, and the last CTA to
// finish (a ticket counter) reduces all of them in a fixed order into the
// DevStats record in the same launch: the result is the same bit for bit
// from run to run.
#include <algorithm>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_strip.cuh"

namespace lbm {
namespace {

// Observes each chunk row of the walk: per node Eq. 6's force, rho and v,
// then the optional moment fields (FP64, 128-bit stores), the snapshot
// compare / store, and the running reductions.  The mass is N rho_ref plus
// the sum of the deviations drho: in FP64 for an FP64 lattice; for FP32
// deviations a float pair (sum, error) kept by Knuth's TwoSum, which carries
// every addition's rounding exactly into the error term (six FP32 additions
// a node instead of a conversion and an addition on this GPU's narrow FP64
// pipe), converted to FP64 once per thread.  The maxima are taken on |v|^2
// and |v - v_snap|^2 in the compute type (exact) and rooted once per CTA.
template <typename T, typename C>
struct ObsRow {
    int mode, nx, ny;
    double* __restrict__ rho_o;
    double* __restrict__ vx_o;
    double* __restrict__ vy_o;
    VSnap<C>* __restrict__ vsnap;
    DevStats* __restrict__ ds;
    double dmass, row_mid, row0;
    C mv2, mdv2, dmax, ndmin;
    float ms = 0.f, me = 0.f;   // FP32: running sum of drho and its accumulated rounding

    __device__ __forceinline__ void operator()(int y, int x, bool active, C (&gc)[9][4], const C (&rm)[6],
                                               const C (&r0)[6], const C (&rp)[6], const Coef<C>& k,
                                               unsigned& bad)
    {
        if (!active) return;
        C d4[4], vx4[4], vy4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Stencil<C> q{r0[j + 1], r0[j + 2], rp[j + 1], r0[j], rm[j + 1], rp[j + 2], rp[j], rm[j], rm[j + 2]};
            C Fx, Fy, g[9];
            force<C>(q, k, Fx, Fy);
#pragma unroll
            for (int a = 0; a < 9; ++a) g[a] = gc[a][j];
            node_velocity<C>(g, Fx, Fy, k, d4[j], vx4[j], vy4[j]);
            const C s2 = vx4[j] * vx4[j] + vy4[j] * vy4[j];
            mv2 = (s2 > mv2 || s2 != s2) ? s2 : mv2;      // NaN wins (reported as huge)
            dmax = d4[j] > dmax ? d4[j] : dmax;
            ndmin = -d4[j] > ndmin ? -d4[j] : ndmin;
            if constexpr (sizeof(C) == sizeof(float)) {
                const float t = ms + d4[j];
                const float bp = t - ms;
                me += (ms - (t - bp)) + (d4[j] - bp);
                ms = t;
            } else {
                dmass += double(d4[j]);
            }
        }
        if (!isfinite(dmax) || !isfinite(ndmin) || !isfinite(mv2)) bad |= ST_NONFINITE;
        if (y == ny / 2 || y == 0 || (mode & OBS_FIELDS)) {
            double rho4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) rho4[j] = double(k.rho_ref) + double(d4[j]);
            if (y == ny / 2) row_mid += (rho4[0] + rho4[1]) + (rho4[2] + rho4[3]);
            if (y == 0) row0 += (rho4[0] + rho4[1]) + (rho4[2] + rho4[3]);
            if (ds && y == ny / 2 && x <= nx / 2 && nx / 2 < x + 4) {
                const int j = nx / 2 - x;
                ds->rho_center = j == 0 ? rho4[0] : (j == 1 ? rho4[1] : (j == 2 ? rho4[2] : rho4[3]));
            }
            if (ds && y == 0 && x == 0) ds->rho_corner = rho4[0];
            if (mode & OBS_FIELDS) {
                const size_t o = (size_t)y * nx + x;   // x % 4 == 0 and nx % 4 == 0: 4-node aligned
                stg4(rho_o + o, rho4[0], rho4[1], rho4[2], rho4[3]);
                stg4(vx_o + o, double(vx4[0]), double(vx4[1]), double(vx4[2]), double(vx4[3]));
                stg4(vy_o + o, double(vy4[0]), double(vy4[1]), double(vy4[2]), double(vy4[3]));
            }
        }
        const size_t o = (size_t)y * nx + x;
        if (mode & OBS_SNAP_CMP) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const VSnap<C> sv = vsnap[o + j];
                const C dx = vx4[j] - C(sv.x), dy = vy4[j] - C(sv.y);
                const C d2 = dx * dx + dy * dy;
                mdv2 = (d2 > mdv2 || d2 != d2) ? d2 : mdv2;
            }
        }
        if (mode & OBS_SNAP_STORE) {
#pragma unroll
            for (int j = 0; j < 4; ++j) vsnap[o + j] = make_vsnap(vx4[j], vy4[j]);
        }
    }
};

// max over a warp of a squared magnitude, then its root (NaN -> huge)
template <typename C>
__device__ __forceinline__ double warp_max_root(C v2)
{
    const C w = warp_max(v2 != v2 ? obs_huge<C>() : v2);
    return double(sqrt(w));
}

// One CTA per (strip, row chunk), as the step kernel.  Every CTA reaches the
// reduction, whatever happened to its walk (a misaligned buffer, an empty
// chunk, a stage wait that gave up), so the ticket always completes.
template <typename T, typename C, int NT, int NS, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_observe_strip(const T* __restrict__ fin, int nx, int ny, int nchunks, Coef<C> k, int mode,
                double* __restrict__ rho_o, double* __restrict__ vx_o, double* __restrict__ vy_o,
                VSnap<C>* __restrict__ vsnap, Partial* __restrict__ parts, unsigned* __restrict__ ticket,
                DevStats* __restrict__ ds, const unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const StripSmem<T, C, NT, NS> sm(smem);
    ObsRow<T, C> row{mode, nx, ny, rho_o, vx_o, vy_o, vsnap, (mode & OBS_REDUCE) ? ds : nullptr,
                     0.0, 0.0, 0.0, C(0), C(0), -obs_huge<C>(), -obs_huge<C>()};
    // (only nodes of this CTA's rows enter the sums; N rho_ref is added to the mass per CTA below)
    unsigned bad = 0;
    const int x0 = blockIdx.x * (4 * NT);
    const int y0 = int((long long)blockIdx.y * ny / nchunks);
    const int y1 = int((long long)(blockIdx.y + 1) * ny / nchunks);
    if (!staged_alignment_ok(smem, fin, fin)) {
        bad |= ST_ALIGN;
    } else if (y1 > y0) {
        strip_init_barriers(sm);
        unsigned G = 0;
        strip_walk<T, C, NT, NS, true, false, true>(fin, nx, ny, x0, y0, y1, (blockIdx.y & 1) != 0, k, sm, G, bad,
                                                    row);
    }
    if (!(mode & OBS_REDUCE)) return;

    // CTA partial: warp shuffles, then the warps in order (the stages are free now).
    __syncthreads();
    constexpr int NW = NT / 32;
    double* red = reinterpret_cast<double*>(smem);             // [7][NW]
    unsigned* sbad = reinterpret_cast<unsigned*>(red + 7 * NW);  // [NW]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // nodes this CTA observed: its rows times its strip's columns
    const double cta_nodes = double(y1 > y0 ? y1 - y0 : 0) * double(min(4 * NT, nx - x0));
    if constexpr (sizeof(C) == sizeof(float)) row.dmass = double(row.ms) + double(row.me);
    double v[7] = {warp_sum(row.dmass), warp_sum(row.row_mid), warp_sum(row.row0), warp_max_root(row.mv2),
                   warp_max_root(row.mdv2), 0.0, 0.0};
    const C wdmax = warp_max(row.dmax), wndmin = warp_max(row.ndmin);
    v[5] = double(k.rho_ref) + double(wdmax);
    v[6] = -(double(k.rho_ref) + double(-wndmin));
    const unsigned wbad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 7; ++j) red[j * NW + wid] = v[j];
        sbad[wid] = wbad;
    }
    __syncthreads();
    const unsigned nparts = gridDim.x * gridDim.y;
    // (no static shared memory: it would move the dynamic region off the
    // alignment the bulk copies need)
    unsigned* last = sbad + NW;
    if (threadIdx.x == 0) {
        Partial p;
        p.mass = p.row_mid = p.row0 = 0;
        p.max_v = p.max_dv = p.rho_max = p.neg_rho_min = -1e300;
        p.status = 0;
        p.mass = cta_nodes * double(k.rho_ref);
        for (int w = 0; w < NW; ++w) {
            p.mass += red[0 * NW + w]; p.row_mid += red[1 * NW + w]; p.row0 += red[2 * NW + w];
            p.max_v = fmax(p.max_v, red[3 * NW + w]); p.max_dv = fmax(p.max_dv, red[4 * NW + w]);
            p.rho_max = fmax(p.rho_max, red[5 * NW + w]); p.neg_rho_min = fmax(p.neg_rho_min, red[6 * NW + w]);
            p.status |= sbad[w];
        }
        p.pad = 0;
        parts[blockIdx.y * gridDim.x + blockIdx.x] = p;
        __threadfence();
        *last = atomicAdd(ticket, 1u) == nparts - 1;
    }
    __syncthreads();
    if (!*last) return;

    // The last CTA: every partial is written and fenced; fold them in a fixed
    // order (thread t takes t, t + NT, ...; then the warps; then thread 0).
    __threadfence();
    double a[7] = {0, 0, 0, -1e300, -1e300, -1e300, -1e300};
    unsigned b = 0;
    for (unsigned i = threadIdx.x; i < nparts; i += NT) {
        const Partial* q = parts + i;
        a[0] += __ldcg(&q->mass); a[1] += __ldcg(&q->row_mid); a[2] += __ldcg(&q->row0);
        a[3] = fmax(a[3], __ldcg(&q->max_v)); a[4] = fmax(a[4], __ldcg(&q->max_dv));
        a[5] = fmax(a[5], __ldcg(&q->rho_max)); a[6] = fmax(a[6], __ldcg(&q->neg_rho_min));
        b |= __ldcg(&q->status);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) a[j] = warp_sum(a[j]);
#pragma unroll
    for (int j = 3; j < 7; ++j) a[j] = warp_max(a[j]);
    b = __reduce_or_sync(0xffffffffu, b);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 7; ++j) red[j * NW + wid] = a[j];
        sbad[wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double f[7] = {0, 0, 0, -1e300, -1e300, -1e300, -1e300};
        unsigned fb = status ? *status : 0u;
        for (int w = 0; w < NW; ++w) {
            for (int j = 0; j < 3; ++j) f[j] += red[j * NW + w];
            for (int j = 3; j < 7; ++j) f[j] = fmax(f[j], red[j * NW + w]);
            fb |= sbad[w];
        }
        ds->mass = f[0];
        ds->rho_row_mid = f[1] / nx;
        ds->rho_row0 = f[2] / nx;
        ds->max_v = f[3];
        ds->max_dv = f[4];
        ds->rho_max = f[5];
        ds->rho_min = -f[6];
        ds->status = fb;
        *ticket = 0;   // ready for the next launch
    }
}

template <typename T, typename C, int NT, int NS, int MINB>
int launch(const lbm_params* p, const void* f, int mode, double* rho, double* vx, double* vy, void* vsnap,
           Partial* parts, unsigned* ticket, DevStats* ds, const unsigned* status, cudaStream_t s)
{
    constexpr size_t smem = strip_smem<T, C, NT, NS>();
    static_assert(smem >= (7 * sizeof(double) + sizeof(unsigned)) * (NT / 32) + sizeof(unsigned), "reduction scratch");
    auto kern = k_observe_strip<T, C, NT, NS, MINB>;
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
    const int W = 4 * NT;
    const int nstrips = (p->nx + W - 1) / W;
    int nchunks = std::max(1, (nsm * per_sm) / nstrips);
    nchunks = std::min(nchunks, std::max(1, p->ny / 16));
    kern<<<dim3(nstrips, nchunks), NT, smem, s>>>((const T*)f, p->nx, p->ny, nchunks, make_coef<C>(*p), mode, rho,
                                                  vx, vy, (VSnap<C>*)vsnap, parts, ticket, ds, status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}

}  // namespace

int observe_strip_launch(const lbm_params* p, const void* f, int mode, double* rho, double* vx, double* vy,
                         void* vsnap, Partial* parts, unsigned* ticket, DevStats* ds, const unsigned* status,
                         cudaStream_t s)
{
    if (!lbm_strip_supported(p)) return LBM_E_UNSUPPORTED;
    if (p->precision == LBM_FP64)
        return launch<double, double, 64, 4, 2>(p, f, mode, rho, vx, vy, vsnap, parts, ticket, ds, status, s);
    return launch<float, float, 256, 2, 2>(p, f, mode, rho, vx, vy, vsnap, parts, ticket, ds, status, s);
}

}  // namespace lbm
