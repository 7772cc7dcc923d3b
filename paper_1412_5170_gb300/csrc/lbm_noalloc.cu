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
#include <cuda.h>
#include <cudaTypedefs.h>
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
// Device address of the scratch per device, with the CUDA context it was
// looked up in: each context loads its own copy of the library's device code,
// so the address is only valid in that context.
struct ScratchAddr {
    unsigned long long ctx_id;   // 0: no entry
    void* ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

// ID of the CUDA context current on this thread (0 if none or unknown).  The
// driver gives every context an ID that is never reused in the process, so a
// context destroyed and created again (cudaDeviceReset, a caller's own
// cuCtxCreate) never matches an old entry.  The two driver calls are reached
// through the runtime's entry-point query, so the library needs no link to
// the driver library.
unsigned long long current_context_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Set-up, once per device and CUDA context, with that device current: look up
// the device address of the scratch array in the current context.  A call
// made in another context than the cached entry's (or where the context ID
// cannot be read) looks the address up again.
int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_E_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = current_context_id();
    if (id != 0 && g_scratch[dev].ctx_id == id) {
        *out = g_scratch[dev].ptr;
        return LBM_OK;
    }
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        std::fprintf(stderr, "liblbm: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
        return LBM_E_CUDA;
    }
    if (id == 0) id = current_context_id();   // the look-up made the runtime's context current
    g_scratch[dev] = ScratchAddr{id, ptr};
    *out = ptr;
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
    const long long tiles = (((long long)p->nx + GTX - 1) / GTX) * (((long long)p->ny + GTY - 1) / GTY);
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
