// The library's per-node arithmetic (lbm_device.cuh, with the kernel
// constants of make_coef) compiled by a host compiler and driven by a plain
// pull step over a periodic lattice, in FP64 or in FP32 deviations, so that
// CPU tests can hold it against the oracle without a GPU.  Test infrastructure: the step loop here
// is the generic kernel's order (psi of every pulled density, then Eq. 6's
// force from the 3 x 3 psi stencil, then the collision), one node at a time.
//
// Storage is the library's: the post-collision populations f*_a(x) of the
// previous step, pulled as f_a(x, t) = f*_a(x - e_a).
#include <cmath>
#define __device__
#define __host__
#define __forceinline__ inline
// the library's float division and square root, as IEEE operations (the GPU
// uses faster approximations of a few ulp, far below the FP32 tolerances)
inline float __fdividef(float a, float b) { return a / b; }
inline float rsqrtf(float a) { return 1.0f / std::sqrt(a); }
using std::isfinite;
#define LBM_HOST_ARITHMETIC 1
#include "lbm_host.h"

#include <algorithm>
#include <vector>

using namespace lbm;

namespace {

int wrap(int i, int n)
{
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// T: the stored type and the compute type (double: populations, rho_ref = 0;
// float: deviations g = f - w rho_ref, as the FP32 kernels keep them).
template <typename T, int COLL, int FORC>
int run(const lbm_params* p, T* f, int nsteps)
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    const Coef<T> k = make_coef<T>(*p);
    std::vector<T> out(9 * n), psi(n);
    unsigned bad = 0;
    auto pull = [&](int x, int y, T g[9]) {
        for (int a = 0; a < 9; ++a) g[a] = f[a * n + (size_t)wrap(y - ey(a), ny) * nx + wrap(x - ex(a), nx)];
    };
    for (int s = 0; s < nsteps; ++s) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                T g[9], drho, jx, jy;
                pull(x, y, g);
                moments(g, drho, jx, jy);
                psi[(size_t)y * nx + x] = psi_of_rho<T>(k.rho_ref + drho, k, bad);
            }
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                T g[9], Fx, Fy, vx, vy, rho;
                pull(x, y, g);
                auto P = [&](int dx, int dy) { return psi[(size_t)wrap(y + dy, ny) * nx + wrap(x + dx, nx)]; };
                const Stencil<T> q{P(0, 0), P(1, 0), P(0, 1), P(-1, 0), P(0, -1),
                                   P(1, 1), P(-1, 1), P(-1, -1), P(1, -1)};
                force<T>(q, k, Fx, Fy);
                collide<T, COLL, FORC>(g, Fx, Fy, k, vx, vy, rho, q.c);
                for (int a = 0; a < 9; ++a) out[a * n + (size_t)y * nx + x] = g[a];
            }
        std::copy(out.begin(), out.end(), f);
    }
    return bad ? LBM_E_EOS_DOMAIN : LBM_OK;
}

template <typename T>
int dispatch(const lbm_params* p, T* f, int nsteps)
{
    if (p->collision == LBM_MRT) return run<T, MRT, GUO>(p, f, nsteps);
    switch (p->forcing) {
    case LBM_GUO: return run<T, BGK, GUO>(p, f, nsteps);
    case LBM_EDM: return run<T, BGK, EDM>(p, f, nsteps);
    case LBM_SC: return run<T, BGK, SC>(p, f, nsteps);
    case LBM_LI: return run<T, BGK, LI>(p, f, nsteps);
    default: return LBM_E_INVALID;
    }
}

}  // namespace

// nsteps FP64 steps of the stored populations f (9 * ny * nx doubles, in place).
extern "C" int host_run(const lbm_params* p, double* f, int nsteps) { return dispatch<double>(p, f, nsteps); }

// nsteps FP32 steps of the stored deviations g = f* - w rho_ref (9 * ny * nx
// floats, in place); p->precision must be LBM_FP32_DEV (rho_ref from p).
extern "C" int host_run_f32(const lbm_params* p, float* g, int nsteps) { return dispatch<float>(p, g, nsteps); }
