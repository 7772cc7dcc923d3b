"""lbm_stats_noalloc: the lattice observables for callers that cannot
allocate device memory (for example code inside an application whose memory
pool owns the GPU, or a loop that must not stall on cudaMalloc/cudaFree).

The entry point is called through the C ABI on a population buffer the
caller owns, twice in a row (the fixed scratch array keeps the first call's
contents), and must agree with lbm_stats on the same lattice state.  This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


def stored_layout(f, rho_ref, dtype):
    """Post-streaming populations f_a(x) -> the library's stored buffer
    f_a(x + e_a) - w_a rho_ref (pull convention), as a numpy array."""
    out = np.empty_like(f)
    for a, (ex, ey) in enumerate(E):
        out[a] = np.roll(f[a], (-ey, -ex), axis=(0, 1)) - W[a] * rho_ref
    return out.astype(dtype)


def noalloc(lbm, params, buf, stream):
    out = lbm.lbm_stats_t()
    st = lbm.lbm_stats_noalloc(ctypes.byref(params), ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(stream.cuda_stream),
            ctypes.byref(out))
    return st, out.as_dict()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_noalloc_stats_match_lbm_stats(lbm, precision, rtol):
    import torch
    nx, ny = 200, 120
    p = lbm.make_params(nx, ny, 0.8, 0.9, -0.304, 1.0, "mrt", "guo", precision, s_e=0.8, s_eps=0.8, s_q=1.1)
    with lbm.Lattice(p) as lat:
        lat.init_preset("droplet", 30.0, seed=11)
        lat.step(40)
        ref = lat.stats()
        f = lat.read_populations()
    host = stored_layout(f, p.rho_ref if precision == "fp32" else 0.0,
                         np.float64 if precision == "fp64" else np.float32)
    buf = torch.from_numpy(host).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    free = []
    for call in range(2):
        st, got = noalloc(lbm, p, buf, stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert st == lbm.OK, (call, lbm.lbm_strerror(st))
        assert got["status"] == ref["status"] == 0
        for k in ("mass", "max_v", "rho_min", "rho_max", "rho_center", "rho_corner", "rho_row_mid", "rho_row0"):
            assert got[k] == pytest.approx(ref[k], rel=rtol), (call, k)
        assert got["max_dv"] == -1.0
    # after the first call's one-time set-up, a call takes no device memory
    assert free[1] == free[0]


def test_noalloc_rejects_lattices_beyond_its_scratch(lbm):
    import torch
    p = lbm.make_params(4096, 4104, 0.8, 0.9, -0.304, precision="fp32")   # 128 x 513 tiles > 65536
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    st, _ = noalloc(lbm, p, buf, torch.cuda.current_stream())
    assert st == lbm.E_UNSUPPORTED


def test_noalloc_follows_the_current_cuda_context(lbm):
    """The scratch array's device address belongs to a CUDA context (each
    context loads its own copy of the library's device code).  A caller that
    runs its own contexts -- one reason it cannot allocate through the
    runtime -- must get correct results in each: the same lattice observed in
    the device's primary context, in a context of its own, in the primary
    context again, and in a second own context created after the first was
    destroyed.  Run in a fresh interpreter that drives the contexts through
    the driver API (no torch)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = textwrap.dedent("""
        import ctypes, sys
        import numpy as np
        sys.path.insert(0, %r)
        from paper_1412_5170_gb300 import lbm, synth
        cu = ctypes.CDLL("libcuda.so.1")
        def ok(r, what):
            assert r == 0, (what, r)
        ok(cu.cuInit(0), "cuInit")
        dev = ctypes.c_int()
        ok(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
        nx, ny = 96, 64
        p = lbm.make_params(nx, ny, 0.8, 0.9, -0.304, 1.0, "bgk", "guo", "fp64")
        rv, rl = lbm.maxwell(0.8)
        rho0 = synth.density_field(nx, ny, "droplet", rl, rv, 20.0, seed=3)
        E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
        W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
        # stored layout of the state at rest f_a = w_a rho0: f*_a(x) = w_a rho0(x + e_a)
        host = np.ascontiguousarray(np.stack([W[a] * np.roll(rho0, (-ey, -ex), axis=(0, 1))
                                              for a, (ex, ey) in enumerate(E)]))
        def observe(ctx):
            ok(cu.cuCtxPushCurrent_v2(ctx), "push")
            d = ctypes.c_uint64()
            ok(cu.cuMemAlloc_v2(ctypes.byref(d), ctypes.c_size_t(host.nbytes)), "alloc")
            ok(cu.cuMemcpyHtoD_v2(d, host.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(host.nbytes)), "copy")
            out = lbm.lbm_stats_t()
            st = lbm.lbm_stats_noalloc(ctypes.byref(p), ctypes.c_void_p(d.value), None, ctypes.byref(out))
            ok(cu.cuMemFree_v2(d), "free")
            popped = ctypes.c_void_p()
            ok(cu.cuCtxPopCurrent_v2(ctypes.byref(popped)), "pop")
            assert st == 0, lbm.lbm_strerror(st)
            return out.as_dict()
        prim = ctypes.c_void_p()
        ok(cu.cuDevicePrimaryCtxRetain(ctypes.byref(prim), dev), "retain")
        own = ctypes.c_void_p()
        ok(cu.cuCtxCreate_v2(ctypes.byref(own), 0, dev), "create")
        ok(cu.cuCtxPopCurrent_v2(ctypes.byref(ctypes.c_void_p())), "pop created")
        runs = [observe(prim), observe(own), observe(prim)]
        ok(cu.cuCtxDestroy_v2(own), "destroy")
        own2 = ctypes.c_void_p()
        ok(cu.cuCtxCreate_v2(ctypes.byref(own2), 0, dev), "create 2")
        ok(cu.cuCtxPopCurrent_v2(ctypes.byref(ctypes.c_void_p())), "pop created 2")
        runs.append(observe(own2))
        ok(cu.cuCtxDestroy_v2(own2), "destroy 2")
        ok(cu.cuDevicePrimaryCtxRelease_v2(dev), "release")
        assert abs(runs[0]["mass"] - rho0.sum()) < 1e-12 * rho0.sum(), (runs[0]["mass"], rho0.sum())
        for r in runs[1:]:
            assert r == runs[0], (r, runs[0])
        print("contexts ok")
    """ % root)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "contexts ok" in r.stdout, r.stdout + r.stderr
