// lbm_api.cu -- the single-lattice context of the liblbm C ABI (include/lbm.h):
// creation, initial conditions, stepping, observables, run-to-steady,
// population I/O and checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_kernels.cuh"

using namespace lbm;

struct lbm_ctx {
    lbm_params p;
    cudaStream_t stream;
    bool owns;              // workspace allocated by the library
    void* ws;
    size_t ws_bytes;
    void* f[2];             // population buffers (T = double or float)
    int cur;                // buffer holding the current state
    double *rho, *vx, *vy;  // FP64 moment fields / staging
    double2* vsnap;
    bool have_snap;
    Partial* parts;
    int nparts;
    unsigned* ticket;       // last-CTA counter of the strip observation (0 between launches)
    DevStats* dstats;
    unsigned* status;
    DevStats* hstats;       // pinned host mirror
    int64_t steps;
    int config;             // 0 = generic kernel, k >= 1 = strip configuration k-1
    bool inject_timeout = false;   // the next step's first stage waits give up at once
    // Asynchronous host I/O, set up by the first lbm_init_density_async or
    // lbm_read_moments_async: one copy stream per direction, and device
    // arrays io = [rho0 staging (n)][moment slot 0 (3n)][moment slot 1 (3n)].
    cudaStream_t s_in = nullptr, s_out = nullptr;
    double* io = nullptr;
    cudaEvent_t ev_in_ready = nullptr;   // rho0 staged (s_in)
    cudaEvent_t ev_in_free = nullptr;    // the init kernels have read the staging array (stream)
    cudaEvent_t ev_mom[2] = {nullptr, nullptr};   // moments of slot k written (stream)
    cudaEvent_t ev_out[2] = {nullptr, nullptr};   // slot k copied to the host (s_out)
    int slot = 0;
};

namespace {

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

inline size_t tsize(const lbm_params& p) { return p.precision == LBM_FP64 ? sizeof(double) : sizeof(float); }

dim3 generic_grid(const lbm_params& p)
{
    return dim3((p.nx + GTX - 1) / GTX, (p.ny + GTY - 1) / GTY);
}

struct Layout {
    size_t f0, f1, rho, vx, vy, vsnap, parts, ticket, dstats, status, total;
};

Layout layout_of(const lbm_params& p)
{
    const size_t n = (size_t)p.nx * p.ny;
    const dim3 g = generic_grid(p);
    Layout L;
    size_t o = 0;
    L.f0 = o; o = align256(o + 9 * n * tsize(p));
    L.f1 = o; o = align256(o + 9 * n * tsize(p));
    L.rho = o; o = align256(o + n * sizeof(double));
    L.vx = o; o = align256(o + n * sizeof(double));
    L.vy = o; o = align256(o + n * sizeof(double));
    L.vsnap = o; o = align256(o + n * sizeof(double2));
    L.parts = o; o = align256(o + (size_t)g.x * g.y * sizeof(Partial));
    L.ticket = o; o = align256(o + sizeof(unsigned));
    L.dstats = o; o = align256(o + sizeof(DevStats));
    L.status = o; o = align256(o + sizeof(unsigned));
    L.total = o;
    return L;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    std::fprintf(stderr, "liblbm: CUDA error %s\n", cudaGetErrorString(e));
    return LBM_E_CUDA;
}

#define LBM_CUDA(call)                                 \
    do {                                               \
        int s_ = cuda_status(call);                    \
        if (s_ != LBM_OK) return s_;                   \
    } while (0)

template <typename T, typename C, int COLL, int FORC>
void launch_generic(lbm_ctx* c, const void* fin, void* fout)
{
    k_step_generic<T, C, COLL, FORC><<<generic_grid(c->p), GTX * GTY, 0, c->stream>>>(
        (const T*)fin, (T*)fout, c->p.nx, c->p.ny, make_coef<C>(c->p), c->status);
}

template <typename T, typename C>
void launch_generic_scheme(lbm_ctx* c, const void* fin, void* fout)
{
    const lbm_params& p = c->p;
    if (p.collision == LBM_MRT) launch_generic<T, C, MRT, GUO>(c, fin, fout);
    else if (p.forcing == LBM_GUO) launch_generic<T, C, BGK, GUO>(c, fin, fout);
    else if (p.forcing == LBM_EDM) launch_generic<T, C, BGK, EDM>(c, fin, fout);
    else if (p.forcing == LBM_LI) launch_generic<T, C, BGK, LI>(c, fin, fout);
    else launch_generic<T, C, BGK, SC>(c, fin, fout);
}

// Without autotuning: the strip kernel where it applies -- for FP32 lattices
// at least 1024 wide the 256-thread, two-stage carried configuration (the
// fastest measured on large lattices), otherwise the first strip
// configuration -- unless its strips and row chunks (at least 16 rows each)
// cannot give every SM a CTA, as on small lattices, where the generic
// kernel's 32 x 8 tiles spread wider; else the generic kernel.
int default_config(const lbm_params& p)
{
    if (!lbm_strip_supported(&p)) return 0;
    int cfg = 1;
    if (p.precision == LBM_FP32_DEV && p.nx >= 1024) {
        const int n = lbm_strip_config_count(p.precision);
        for (int i = 0; i < n; ++i) {
            const StripConfig sc = lbm_strip_config(p.precision, i);
            if (sc.threads == 256 && sc.stages == 2) { cfg = i + 1; break; }
        }
    }
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
            nsm = 1;
    }
    const StripConfig sc = lbm_strip_config(p.precision, cfg - 1);
    const long long width = 4LL * sc.threads;
    const long long strips = (p.nx + width - 1) / width;
    if (strips * std::max(1, p.ny / 16) < nsm) return 0;
    return cfg;
}

int n_configs(const lbm_params& p) { return 1 + (lbm_strip_supported(&p) ? lbm_strip_config_count(p.precision) : 0); }

// One fused step from fin to fout with kernel configuration cfg.
int launch_step(lbm_ctx* c, int cfg, const void* fin, void* fout, long long first_wait = kStageWaitPolls)
{
    if (cfg >= 1) {
        const int s = lbm_strip_launch(&c->p, cfg - 1, fin, fout, c->status, c->stream, first_wait);
        if (s != LBM_OK) return s;
    } else if (c->p.precision == LBM_FP64) {
        launch_generic_scheme<double, double>(c, fin, fout);
    } else {
        launch_generic_scheme<float, float>(c, fin, fout);
    }
    LBM_CUDA(cudaGetLastError());
    return LBM_OK;
}

int step_once(lbm_ctx* c)
{
    const long long first_wait = c->inject_timeout ? 0 : kStageWaitPolls;
    c->inject_timeout = false;
    const int s = launch_step(c, c->config, c->f[c->cur], c->f[c->cur ^ 1], first_wait);
    if (s != LBM_OK) return s;
    c->cur ^= 1;
    c->steps += 1;
    return LBM_OK;
}

template <typename T, typename C>
void launch_observe(lbm_ctx* c, int mode, double* rho, double* vx, double* vy)
{
    k_observe<T, C><<<generic_grid(c->p), GTX * GTY, 0, c->stream>>>(
        (const T*)c->f[c->cur], c->p.nx, c->p.ny, make_coef<C>(c->p), mode, rho, vx, vy,
        reinterpret_cast<VSnap<C>*>(c->vsnap), c->parts, c->dstats, c->status);
}

// Observation of the current state: with the strip walk where the strip
// kernel applies (one launch, reduction included), else the generic tiled
// kernel followed (with OBS_REDUCE) by the one-CTA final reduction.
int observe_into(lbm_ctx* c, int mode, double* rho, double* vx, double* vy)
{
    if (lbm_strip_supported(&c->p))
        return observe_strip_launch(&c->p, c->f[c->cur], mode, rho, vx, vy, c->vsnap, c->parts, c->ticket,
                                    c->dstats, c->status, c->stream);
    if (c->p.precision == LBM_FP64) launch_observe<double, double>(c, mode, rho, vx, vy);
    else launch_observe<float, float>(c, mode, rho, vx, vy);
    LBM_CUDA(cudaGetLastError());
    if (mode & OBS_REDUCE) {
        k_reduce_final<<<1, 256, 0, c->stream>>>(c->parts, c->nparts, c->p.nx, c->dstats);
        LBM_CUDA(cudaGetLastError());
    }
    return LBM_OK;
}

// The moment fields (mode OBS_FIELDS) into the given device arrays.
int observe_fields_into(lbm_ctx* c, double* rho, double* vx, double* vy)
{
    return observe_into(c, OBS_FIELDS, rho, vx, vy);
}

// The copy streams, events and device arrays of the asynchronous host I/O.
int ensure_io(lbm_ctx* c)
{
    if (c->io) return LBM_OK;
    // each piece is made once, so a call after a failed set-up completes it
    const size_t n = (size_t)c->p.nx * c->p.ny;
    if (!c->s_in) LBM_CUDA(cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking));
    if (!c->s_out) LBM_CUDA(cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking));
    cudaEvent_t* evs[6] = {&c->ev_in_ready, &c->ev_in_free, &c->ev_mom[0], &c->ev_mom[1], &c->ev_out[0], &c->ev_out[1]};
    for (cudaEvent_t* e : evs)
        if (!*e) LBM_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    LBM_CUDA(cudaMalloc(&c->io, 7 * n * sizeof(double)));
    return LBM_OK;
}

void release_io(lbm_ctx* c)
{
    if (c->s_in) cudaStreamSynchronize(c->s_in);
    if (c->s_out) cudaStreamSynchronize(c->s_out);
    cudaEvent_t evs[6] = {c->ev_in_ready, c->ev_in_free, c->ev_mom[0], c->ev_mom[1], c->ev_out[0], c->ev_out[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (c->s_in) cudaStreamDestroy(c->s_in);
    if (c->s_out) cudaStreamDestroy(c->s_out);
    if (c->io) cudaFree(c->io);
}

int observe(lbm_ctx* c, int mode) { return observe_into(c, mode, c->rho, c->vx, c->vy); }

int status_code(unsigned bits)
{
    if (bits & ST_NONFINITE) return LBM_E_NONFINITE;
    if (bits & ST_EOS) return LBM_E_EOS_DOMAIN;
    if (bits & ST_TIMEOUT) return LBM_E_TIMEOUT;
    if (bits & ST_ALIGN) return LBM_E_CUDA;
    return LBM_OK;
}

// The deviation reference exactly as the kernels see it (rounded to float on
// the FP32 path), so that stored deviations and rho = rho_ref + sum g agree.
double rho_ref_eff(const lbm_params& p)
{
    return p.precision == LBM_FP64 ? 0.0 : double(float(p.rho_ref));
}

template <typename T>
void launch_init_rest(lbm_ctx* c, const double* rho0)
{
    if constexpr (sizeof(T) == sizeof(float)) {
        // the FP64 v_x field doubles as the float deviation scratch (n floats fit in n doubles)
        float* dev = reinterpret_cast<float*>(c->vx);
        const size_t n = (size_t)c->p.nx * c->p.ny;
        k_init_dev_f32<<<1024, 256, 0, c->stream>>>(rho0, dev, n, rho_ref_eff(c->p));
        k_init_rest_f32<<<1024, 256, 0, c->stream>>>(dev, (float*)c->f[c->cur], c->p.nx, c->p.ny);
    } else {
        k_init_rest<T><<<1024, 256, 0, c->stream>>>(rho0, (T*)c->f[c->cur], c->p.nx, c->p.ny, rho_ref_eff(c->p));
    }
}

template <typename T>
void launch_plane(lbm_ctx* c, int a, int to_stored)
{
    k_plane_convert<T><<<1024, 256, 0, c->stream>>>((T*)c->f[c->cur], c->rho, a, c->p.nx, c->p.ny,
                                                      rho_ref_eff(c->p), to_stored);
}

int reset_state(lbm_ctx* c)
{
    c->steps = 0;
    c->have_snap = false;
    LBM_CUDA(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    return LBM_OK;
}

uint64_t fnv1a(const unsigned char* d, size_t n, uint64_t h = 1469598103934665603ull)
{
    for (size_t i = 0; i < n; ++i) { h ^= d[i]; h *= 1099511628211ull; }
    return h;
}

const char kMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};

struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    lbm_params p;
    int64_t steps;
    uint64_t payload_bytes, checksum;
};

}  // namespace

extern "C" {

const char* lbm_strerror(int s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_E_INVALID: return "invalid argument";
    case LBM_E_CUDA: return "CUDA error";
    case LBM_E_NONFINITE: return "non-finite value in the lattice";
    case LBM_E_EOS_DOMAIN: return "density outside the EOS domain (psi undefined)";
    case LBM_E_TIMEOUT: return "device-side wait timed out";
    case LBM_E_NOT_CONVERGED: return "not converged within max_steps";
    case LBM_E_IO: return "checkpoint I/O error";
    case LBM_E_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

int lbm_version(void) { return (1 << 16) | 0; }

int lbm_workspace_bytes(const lbm_params* p, size_t* bytes)
{
    if (!p || !bytes) return LBM_E_INVALID;
    const int v = lbm_validate_params(p);
    if (v != LBM_OK) return v;
    *bytes = layout_of(*p).total;
    return LBM_OK;
}

int lbm_create(const lbm_params* p, void* cuda_stream, void* workspace_dev, size_t workspace_bytes,
               lbm_ctx** out)
{
    if (!p || !out) return LBM_E_INVALID;
    *out = nullptr;
    int v = lbm_validate_params(p);
    if (v != LBM_OK) return v;
    const Layout L = layout_of(*p);
    if (workspace_dev && (workspace_bytes < L.total || ((uintptr_t)workspace_dev & 255))) return LBM_E_INVALID;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_E_INVALID;
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    c->owns = workspace_dev == nullptr;
    c->ws_bytes = L.total;
    if (c->owns) {
        cudaError_t e = cudaMalloc(&c->ws, L.total);
        if (e != cudaSuccess) { delete c; return cuda_status(e); }
    } else {
        c->ws = workspace_dev;
    }
    char* b = (char*)c->ws;
    c->f[0] = b + L.f0;
    c->f[1] = b + L.f1;
    c->rho = (double*)(b + L.rho);
    c->vx = (double*)(b + L.vx);
    c->vy = (double*)(b + L.vy);
    c->vsnap = (double2*)(b + L.vsnap);
    c->parts = (Partial*)(b + L.parts);
    c->ticket = (unsigned*)(b + L.ticket);
    const dim3 g = generic_grid(*p);
    c->nparts = int(g.x * g.y);
    c->dstats = (DevStats*)(b + L.dstats);
    c->status = (unsigned*)(b + L.status);
    c->cur = 0;
    c->config = default_config(*p);
    cudaError_t e = cudaMallocHost(&c->hstats, sizeof(DevStats));
    if (e != cudaSuccess) {
        if (c->owns) cudaFree(c->ws);
        delete c;
        return cuda_status(e);
    }
    if (cudaMemsetAsync(c->ws, 0, L.total, c->stream) != cudaSuccess) {
        lbm_destroy(c);
        return LBM_E_CUDA;
    }
    reset_state(c);
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    release_io(c);
    if (c->owns && c->ws) cudaFree(c->ws);
    if (c->hstats) cudaFreeHost(c->hstats);
    delete c;
}

int lbm_init_density_dev(lbm_ctx* c, const double* rho0_dev)
{
    if (!c || !rho0_dev) return LBM_E_INVALID;
    c->cur = 0;
    if (c->p.precision == LBM_FP64) launch_init_rest<double>(c, rho0_dev);
    else launch_init_rest<float>(c, rho0_dev);
    LBM_CUDA(cudaGetLastError());
    return reset_state(c);
}

int lbm_init_density(lbm_ctx* c, const double* rho0_host)
{
    if (!c || !rho0_host) return LBM_E_INVALID;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    LBM_CUDA(cudaMemcpyAsync(c->rho, rho0_host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    return lbm_init_density_dev(c, c->rho);
}

int lbm_init_density_async(lbm_ctx* c, const double* rho0_host)
{
    if (!c || !rho0_host) return LBM_E_INVALID;
    int s = ensure_io(c);
    if (s != LBM_OK) return s;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    // the staging array is free once the previous asynchronous init has read it
    LBM_CUDA(cudaStreamWaitEvent(c->s_in, c->ev_in_free, 0));
    LBM_CUDA(cudaMemcpyAsync(c->io, rho0_host, n * sizeof(double), cudaMemcpyHostToDevice, c->s_in));
    LBM_CUDA(cudaEventRecord(c->ev_in_ready, c->s_in));
    LBM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in_ready, 0));
    if ((s = lbm_init_density_dev(c, c->io)) != LBM_OK) return s;
    LBM_CUDA(cudaEventRecord(c->ev_in_free, c->stream));
    return LBM_OK;
}

int lbm_read_moments_async(lbm_ctx* c, double* rho_host, double* vx_host, double* vy_host)
{
    if (!c) return LBM_E_INVALID;
    int s = ensure_io(c);
    if (s != LBM_OK) return s;
    const size_t n = (size_t)c->p.nx * c->p.ny, nb = n * sizeof(double);
    const int k = c->slot;
    double* m = c->io + n + (size_t)k * 3 * n;
    // the slot's arrays are free once its previous copies to the host are done
    LBM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_out[k], 0));
    if ((s = observe_fields_into(c, m, m + n, m + 2 * n)) != LBM_OK) return s;
    LBM_CUDA(cudaEventRecord(c->ev_mom[k], c->stream));
    LBM_CUDA(cudaStreamWaitEvent(c->s_out, c->ev_mom[k], 0));
    if (rho_host) LBM_CUDA(cudaMemcpyAsync(rho_host, m, nb, cudaMemcpyDeviceToHost, c->s_out));
    if (vx_host) LBM_CUDA(cudaMemcpyAsync(vx_host, m + n, nb, cudaMemcpyDeviceToHost, c->s_out));
    if (vy_host) LBM_CUDA(cudaMemcpyAsync(vy_host, m + 2 * n, nb, cudaMemcpyDeviceToHost, c->s_out));
    LBM_CUDA(cudaEventRecord(c->ev_out[k], c->s_out));
    c->slot = k ^ 1;
    return LBM_OK;
}

int lbm_wait_io(lbm_ctx* c)
{
    if (!c) return LBM_E_INVALID;
    if (c->s_in) LBM_CUDA(cudaStreamSynchronize(c->s_in));
    if (c->s_out) LBM_CUDA(cudaStreamSynchronize(c->s_out));
    return LBM_OK;
}

int lbm_init_preset(lbm_ctx* c, int kind, double size, double width, double rho_l, double rho_v,
                    int32_t cell, uint64_t seed, double noise_amp)
{
    if (!c) return LBM_E_INVALID;
    if (rho_l <= 0 || rho_v <= 0) {
        const int s = lbm_maxwell(c->p.T_over_Tc, &rho_v, &rho_l);
        if (s != LBM_OK) return s;
    }
    std::vector<double> rho0;
    const int s = lbm_preset_field(c->p.nx, c->p.ny, kind, size, width, rho_l, rho_v, cell, seed,
                                   noise_amp, rho0);
    if (s != LBM_OK) return s;
    const int r = lbm_init_density(c, rho0.data());
    if (r != LBM_OK) return r;
    LBM_CUDA(cudaStreamSynchronize(c->stream));   // rho0 is a local host vector
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t nsteps)
{
    if (!c || nsteps < 0) return LBM_E_INVALID;
    for (int64_t i = 0; i < nsteps; ++i) {
        const int s = step_once(c);
        if (s != LBM_OK) return s;
    }
    return LBM_OK;
}

int lbm_stats(lbm_ctx* c, int snapshot, lbm_stats_t* out)
{
    if (!c || !out) return LBM_E_INVALID;
    int mode = OBS_REDUCE;
    if (c->have_snap) mode |= OBS_SNAP_CMP;
    if (snapshot) mode |= OBS_SNAP_STORE;
    int s = observe(c, mode);
    if (s != LBM_OK) return s;
    LBM_CUDA(cudaMemcpyAsync(c->hstats, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    const DevStats& d = *c->hstats;
    out->mass = d.mass;
    out->max_v = d.max_v;
    out->max_dv = c->have_snap ? d.max_dv : -1.0;
    out->rho_min = d.rho_min;
    out->rho_max = d.rho_max;
    out->rho_center = d.rho_center;
    out->rho_corner = d.rho_corner;
    out->rho_row_mid = d.rho_row_mid;
    out->rho_row0 = d.rho_row0;
    out->steps = c->steps;
    out->status = status_code(d.status);
    out->reserved = 0;
    if (snapshot) c->have_snap = true;
    return LBM_OK;
}

int lbm_run_to_steady(lbm_ctx* c, double tol, int64_t check_every, int64_t max_steps, int64_t* steps_done)
{
    if (!c || !(tol > 0) || check_every <= 0 || max_steps < 0) return LBM_E_INVALID;
    int64_t done = 0;
    if (steps_done) *steps_done = 0;
    lbm_stats_t st;
    int s = lbm_stats(c, 1, &st);
    if (s != LBM_OK) return s;
    if (st.status != LBM_OK) return st.status;
    while (done < max_steps) {
        const int64_t k = (max_steps - done < check_every) ? max_steps - done : check_every;
        s = lbm_step(c, k);
        if (s != LBM_OK) return s;
        done += k;
        if (steps_done) *steps_done = done;
        s = lbm_stats(c, 1, &st);
        if (s != LBM_OK) return s;
        if (st.status != LBM_OK) return st.status;
        if (k == check_every && st.max_dv >= 0 && st.max_dv < tol) return LBM_OK;
    }
    return LBM_E_NOT_CONVERGED;
}

int lbm_read_moments(lbm_ctx* c, double* rho_host, double* vx_host, double* vy_host)
{
    if (!c) return LBM_E_INVALID;
    int s = observe(c, OBS_FIELDS);
    if (s != LBM_OK) return s;
    const size_t nb = (size_t)c->p.nx * c->p.ny * sizeof(double);
    if (rho_host) LBM_CUDA(cudaMemcpyAsync(rho_host, c->rho, nb, cudaMemcpyDeviceToHost, c->stream));
    if (vx_host) LBM_CUDA(cudaMemcpyAsync(vx_host, c->vx, nb, cudaMemcpyDeviceToHost, c->stream));
    if (vy_host) LBM_CUDA(cudaMemcpyAsync(vy_host, c->vy, nb, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_read_populations(lbm_ctx* c, double* f_host)
{
    if (!c || !f_host) return LBM_E_INVALID;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    for (int a = 0; a < 9; ++a) {
        if (c->p.precision == LBM_FP64) launch_plane<double>(c, a, 0);
        else launch_plane<float>(c, a, 0);
        LBM_CUDA(cudaGetLastError());
        LBM_CUDA(cudaMemcpyAsync(f_host + a * n, c->rho, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_write_populations(lbm_ctx* c, const double* f_host)
{
    if (!c || !f_host) return LBM_E_INVALID;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    c->cur = 0;
    for (int a = 0; a < 9; ++a) {
        LBM_CUDA(cudaMemcpyAsync(c->rho, f_host + a * n, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if (c->p.precision == LBM_FP64) launch_plane<double>(c, a, 1);
        else launch_plane<float>(c, a, 1);
        LBM_CUDA(cudaGetLastError());
    }
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return reset_state(c);
}

int lbm_copy_rows(lbm_ctx* c, int y0, int nrows, void* buf_dev, int to_lattice)
{
    if (!c || !buf_dev || nrows < 0 || y0 < 0 || (long long)y0 + nrows > c->p.ny) return LBM_E_INVALID;
    const size_t es = tsize(c->p), n = (size_t)c->p.nx * c->p.ny, rows = (size_t)nrows * c->p.nx;
    unsigned char* f = static_cast<unsigned char*>(c->f[c->cur]);
    unsigned char* b = static_cast<unsigned char*>(buf_dev);
    for (int a = 0; a < 9 && nrows > 0; ++a) {
        unsigned char* lat = f + es * (a * n + (size_t)y0 * c->p.nx);
        unsigned char* buf = b + es * (a * rows);
        LBM_CUDA(cudaMemcpyAsync(to_lattice ? lat : buf, to_lattice ? buf : lat, es * rows, cudaMemcpyDeviceToDevice,
                                 c->stream));
    }
    return LBM_OK;
}

int lbm_save(lbm_ctx* c, const char* path)
{
    if (!c || !path) return LBM_E_INVALID;
    const size_t bytes = 9 * (size_t)c->p.nx * c->p.ny * tsize(c->p);
    std::vector<unsigned char> buf(bytes);
    LBM_CUDA(cudaMemcpyAsync(buf.data(), c->f[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.header_bytes = sizeof(CkptHeader);
    h.p = c->p;
    h.steps = c->steps;
    h.payload_bytes = bytes;
    h.checksum = fnv1a(buf.data(), bytes);
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return LBM_E_IO;
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(buf.data(), 1, bytes, fp) == bytes;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : LBM_E_IO;
}

int lbm_load(lbm_ctx* c, const char* path)
{
    if (!c || !path) return LBM_E_INVALID;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return LBM_E_IO;
    CkptHeader h;
    const size_t bytes = 9 * (size_t)c->p.nx * c->p.ny * tsize(c->p);
    std::vector<unsigned char> buf(bytes);
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::memcmp(h.magic, kMagic, 8) == 0 &&
              h.version == 1 && h.header_bytes == sizeof(CkptHeader) &&
              std::memcmp(&h.p, &c->p, sizeof(lbm_params)) == 0 && h.payload_bytes == bytes &&
              std::fread(buf.data(), 1, bytes, fp) == bytes && fnv1a(buf.data(), bytes) == h.checksum;
    std::fclose(fp);
    if (!ok) return LBM_E_IO;
    c->cur = 0;
    LBM_CUDA(cudaMemcpyAsync(c->f[0], buf.data(), bytes, cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    const int s = reset_state(c);
    c->steps = h.steps;
    return s;
}

int lbm_inject_stage_timeout(lbm_ctx* c)
{
    if (!c) return LBM_E_INVALID;
    if (c->config < 1) return LBM_E_UNSUPPORTED;   // the generic kernel has no staged copies
    c->inject_timeout = true;
    return LBM_OK;
}

int lbm_get_variant(lbm_ctx* c, int* variant)
{
    if (!c || !variant) return LBM_E_INVALID;
    *variant = c->config >= 1 ? 1 : 0;
    return LBM_OK;
}

int lbm_set_variant(lbm_ctx* c, int variant)
{
    if (!c || variant < -1 || variant > 1) return LBM_E_INVALID;
    if (variant == 1 && !lbm_strip_supported(&c->p)) return LBM_E_UNSUPPORTED;
    c->config = variant == -1 ? default_config(c->p) : variant;
    return LBM_OK;
}

int lbm_config_count(const lbm_params* p, int* count)
{
    if (!p || !count || lbm_validate_params(p) != LBM_OK) return LBM_E_INVALID;
    *count = n_configs(*p);
    return LBM_OK;
}

int lbm_config_describe(const lbm_params* p, int config, int* threads, int* stages, int* nodes_per_thread)
{
    if (!p || lbm_validate_params(p) != LBM_OK || config < 0 || config >= n_configs(*p)) return LBM_E_INVALID;
    int th = GTX * GTY, st = 0, npt = 1;
    if (config >= 1) {
        const StripConfig sc = lbm_strip_config(p->precision, config - 1);
        th = sc.threads;
        st = sc.stages;
        npt = 4;
    }
    if (threads) *threads = th;
    if (stages) *stages = st;
    if (nodes_per_thread) *nodes_per_thread = npt;
    return LBM_OK;
}

int lbm_get_config(lbm_ctx* c, int* config)
{
    if (!c || !config) return LBM_E_INVALID;
    *config = c->config;
    return LBM_OK;
}

int lbm_set_config(lbm_ctx* c, int config)
{
    if (!c || config < 0 || config >= n_configs(c->p)) return LBM_E_INVALID;
    c->config = config;
    return LBM_OK;
}

int lbm_autotune(lbm_ctx* c, int trial_steps, int* config, double* ms_per_step)
{
    if (!c || trial_steps < 1) return LBM_E_INVALID;
    cudaEvent_t e0, e1;
    LBM_CUDA(cudaEventCreate(&e0));
    LBM_CUDA(cudaEventCreate(&e1));
    int best = c->config;
    float best_ms = 3.4e38f;
    int status = LBM_OK;
    const void* fin = c->f[c->cur];
    void* spare = c->f[c->cur ^ 1];
    for (int cfg = 0; cfg < n_configs(c->p) && status == LBM_OK; ++cfg) {
        // Trials read the current state and write the spare buffer: the
        // lattice state is unchanged.  One untimed launch sets up the kernel.
        status = launch_step(c, cfg, fin, spare);
        if (status != LBM_OK) break;
        if ((status = cuda_status(cudaEventRecord(e0, c->stream))) != LBM_OK) break;
        for (int i = 0; i < trial_steps && status == LBM_OK; ++i) status = launch_step(c, cfg, fin, spare);
        if (status != LBM_OK) break;
        if ((status = cuda_status(cudaEventRecord(e1, c->stream))) != LBM_OK) break;
        if ((status = cuda_status(cudaEventSynchronize(e1))) != LBM_OK) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= trial_steps;
        if (ms < best_ms) { best_ms = ms; best = cfg; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != LBM_OK) return status;
    c->config = best;
    if (config) *config = best;
    if (ms_per_step) *ms_per_step = best_ms;
    return LBM_OK;
}

}  // extern "C"
