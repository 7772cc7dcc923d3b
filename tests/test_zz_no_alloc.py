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
    for call in range(2):
        st, got = noalloc(lbm, p, buf, stream)
        assert st == lbm.OK, (call, lbm.lbm_strerror(st))
        assert got["status"] == ref["status"] == 0
        for k in ("mass", "max_v", "rho_min", "rho_max", "rho_center", "rho_corner", "rho_row_mid", "rho_row0"):
            assert got[k] == pytest.approx(ref[k], rel=rtol), (call, k)
        assert got["max_dv"] == -1.0


def test_noalloc_rejects_lattices_beyond_its_scratch(lbm):
    import torch
    p = lbm.make_params(4096, 4104, 0.8, 0.9, -0.304, precision="fp32")   # 128 x 513 tiles > 65536
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    st, _ = noalloc(lbm, p, buf, torch.cuda.current_stream())
    assert st == lbm.E_UNSUPPORTED
