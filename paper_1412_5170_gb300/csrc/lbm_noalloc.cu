// lbm_noalloc.cu -- lbm_stats_noalloc: the whole-lattice observables of
// lbm_stats computed without allocating any memory.
//
// Who needs it: callers that cannot call cudaMalloc / cudaFree.  Examples are
// code running inside a host application whose memory pool owns the device
// and forbids direct allocation, and loops that must not stall on an
// allocation (cudaMalloc and cudaFree may synchronise the device).  They
// already own the population buffer; this entry point needs nothing else.
//
// The per-block partial results that lbm_stats keeps in its context
// workspace live here in one fixed array compiled into the library
// (g_noalloc_scratch).  Every GPU that loads the library holds that array
// until the process exits.  Its size caps the lattice: at most
// LBM_NOALLOC_MAX_TILES tiles of 32 x 8 nodes (any lattice up to
// 4096 x 4096 fits).
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_kernels.cuh"

using namespace lbm;

namespace {

constexpr size_t kPartialBytes = size_t(LBM_NOALLOC_MAX_TILES) * sizeof(Partial);
constexpr size_t kScratchBytes = kPartialBytes + 256;   // partials, then one DevStats

// The fixed scratch.  In host code this name is only a host-side stand-in,
// not a device address: the kernels get the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_dev[kMaxDevices] = {};   // device address of the scratch, per device

// Set-up, once per device with that device current: look up the device
// address of the scratch array.
int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_E_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            std::fprintf(stderr, "liblbm: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return LBM_E_CUDA;
        }
        g_scratch_dev[dev] = ptr;
    }
    *out = g_scratch_dev[dev];
    return LBM_OK;
}

template <typename T>
void launch(const lbm_params& p, const void* f, Partial* parts, DevStats* ds, cudaStream_t s)
{
    const dim3 grid((p.nx + GTX - 1) / GTX, (p.ny + GTY - 1) / GTY);
    k_observe<T, T><<<grid, GTX * GTY, 0, s>>>((const T*)f, p.nx, p.ny, make_coef<T>(p), OBS_REDUCE,
                                               nullptr, nullptr, nullptr, nullptr, parts, ds, nullptr);
}

}  // namespace

extern "C" int lbm_stats_noalloc(const lbm_params* p, const void* f_dev, void* cuda_stream, lbm_stats_t* out)
{
    if (!p || !f_dev || !out) return LBM_E_INVALID;
    const int v = lbm_validate_params(p);
    if (v != LBM_OK) return v;
    const long long tiles = (long long)((p->nx + GTX - 1) / GTX) * ((p->ny + GTY - 1) / GTY);
    if (tiles > LBM_NOALLOC_MAX_TILES) {
        std::fprintf(stderr, "liblbm: lbm_stats_noalloc: %d x %d lattice needs %lld tiles, more than the "
                     "fixed scratch holds (%d)\n", p->nx, p->ny, tiles, LBM_NOALLOC_MAX_TILES);
        return LBM_E_UNSUPPORTED;
    }
    void* base = nullptr;
    int s = scratch_address(&base);
    if (s != LBM_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Partial* parts = (Partial*)base;
    DevStats* ds = (DevStats*)((char*)base + kPartialBytes);
    // The array keeps the previous call's contents: start the observables at zero.
    if (cudaMemsetAsync(ds, 0, sizeof(DevStats), st) != cudaSuccess) return LBM_E_CUDA;
    if (p->precision == LBM_FP64) launch<double>(*p, f_dev, parts, ds, st);
    else launch<float>(*p, f_dev, parts, ds, st);
    if (cudaGetLastError() != cudaSuccess) return LBM_E_CUDA;
    k_reduce_final<<<1, 256, 0, st>>>(parts, int(tiles), p->nx, ds);
    if (cudaGetLastError() != cudaSuccess) return LBM_E_CUDA;
    DevStats h;
    if (cudaMemcpyAsync(&h, ds, sizeof(DevStats), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBM_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_E_CUDA;
    out->mass = h.mass;
    out->max_v = h.max_v;
    out->max_dv = -1.0;
    out->rho_min = h.rho_min;
    out->rho_max = h.rho_max;
    out->rho_center = h.rho_center;
    out->rho_corner = h.rho_corner;
    out->rho_row_mid = h.rho_row_mid;
    out->rho_row0 = h.rho_row0;
    out->steps = 0;
    out->status = (h.status & ST_NONFINITE) ? LBM_E_NONFINITE : ((h.status & ST_EOS) ? LBM_E_EOS_DOMAIN : LBM_OK);
    out->reserved = 0;
    return LBM_OK;
}
