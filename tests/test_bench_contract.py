"""bench.py's reference arm (the FP64 oracle on the host) prints one JSON line
with the contract's keys; it runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["steps"] == 3 and d["value"] > 0
    assert d["config"]["workload"].startswith("droplet array 4096x4096")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def _bench():
    import importlib
    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_coexistence_tail_of_a_geometric_approach_is_exact():
    """A probe approaching its limit L as p_k = L + c r^k: from its last two
    changes the tail estimate is exactly what is still to come, |p_k - L|,
    for a monotone (0 < r < 1) approach; an alternating one (r < 0) is bounded
    by its last change."""
    b = _bench()
    L, c = 0.25, 1e-3
    for r in (0.5, 0.9, 0.99):
        p = [L + c * r ** k for k in range(6)]
        d, dp = p[5] - p[4], p[4] - p[3]
        # exact up to the rounding of the differences (cancellation near L)
        assert abs(b.coex_tail(d, dp) - abs(p[5] - L)) <= 1e-8 * abs(p[5] - L)
    p = [L + c * (-0.6) ** k for k in range(6)]
    d, dp = p[5] - p[4], p[4] - p[3]
    assert b.coex_tail(d, dp) == abs(d) >= abs(p[5] - L)


def test_coexistence_tail_refuses_until_the_changes_shrink():
    b = _bench()
    inf = float("inf")
    assert b.coex_tail(1e-6, float("nan")) == inf     # one change known
    assert b.coex_tail(2e-6, 1e-6) == inf             # growing
    assert b.coex_tail(1e-6, 1e-6) == inf             # not shrinking
    assert b.coex_tail(1e-6, 0.0) == inf              # a move after a standstill
    assert b.coex_tail(0.0, 1e-6) == 0.0              # did not move


def test_coexistence_measure_takes_the_larger_probe_and_rule():
    """The criterion's quantity: the probes' relative change since the
    previous check, and with rule "tail" at least their relative tails from
    this check's pair of changes and from the pair before."""
    b = _bench()
    nan = float("nan")
    unknown = ((nan, nan), (nan, nan))
    prev, cur = (0.4, 0.01), (0.4 + 4e-7, 0.01 + 2e-8)
    m, hist = b.coex_measure(prev, cur, unknown, "change")
    d = (cur[0] - prev[0], cur[1] - prev[1])
    assert hist == ((d[0], nan), (d[1], nan)) or (hist[0][0] == d[0] and hist[1][0] == d[1])
    assert m == max(abs(d[0]) / cur[0], abs(d[1]) / cur[1])
    assert abs(m - 2e-8 / (0.01 + 2e-8)) < 1e-6 * m       # the vapour probe's
    assert b.coex_measure(prev, cur, unknown, "tail")[0] == float("inf")
    # both probes shrinking geometrically (0.5 and 0.99 per check): the vapour
    # probe's tail is 99 of its last changes, and 99 of the one before
    # (100 of the last) from the previous pair, the larger
    hist = ((d[0] / 0.5, d[0] / 0.25), (d[1] / 0.99, d[1] / 0.99 ** 2))
    m, _ = b.coex_measure(prev, cur, hist, "tail")
    assert abs(m - 100 * abs(d[1]) / cur[1]) < 1e-8 * m
    # one sign flip of the last change does not hide a slow approach before it
    hist = ((-d[0], -d[0] / 0.5), (-d[1], -d[1] / 0.99))
    m, _ = b.coex_measure(prev, cur, hist, "tail")
    assert m >= 99 * abs(d[1]) / cur[1] * 0.99
