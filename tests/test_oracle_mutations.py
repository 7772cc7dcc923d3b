"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU,
in a temporary directory), compiles it, and runs the CPU pin tests against it
in a subprocess with ORACLE_SO pointing at the broken library: the run must
fail.

Not listed: Eq. 23's printed index pair (F_i v_j + v_j F_i).  Contracted with
the symmetric tensor (e_i e_j - c_s^2 d_ij) it equals (F_i v_j + v_i F_j), so
that reading is not a mistake and no pin can (or should) tell them apart.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")
PINS = ["tests/test_oracle_node.py", "tests/test_oracle_force.py", "tests/test_oracle_thermo.py",
        "tests/test_oracle_lattice.py"]

MUTATIONS = {
    "force_A_sign": ("Fx[y * nx + x] = -A * sumU[0]", "Fx[y * nx + x] = A * sumU[0]"),
    "force_d2q9_weights": ("const double wforce[9] = {0.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0 / 3,\n"
                           "                              1.0 / 12, 1.0 / 12, 1.0 / 12, 1.0 / 12};",
                           "const double wforce[9] = {0.0, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,\n"
                           "                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};"),
    "guo_isotropic_sign": ("(e[i] * e[j] - cs2 * delta)", "(e[i] * e[j] + cs2 * delta)"),
    "guo_second_order_dropped": ("S[a] = W[a] * prefactor * (first + second);",
                                 "S[a] = W[a] * prefactor * first;"),
    "guo_prefactor_dropped": ("orc_guo_source(1.0 - 1.0 / (2.0 * tau), Fx, Fy, vx, vy, S);",
                              "orc_guo_source(1.0, Fx, Fy, vx, vy, S);"),
    "guo_velocity_full_force": ("double vx = ux + Fx / (2.0 * rho), vy = uy + Fy / (2.0 * rho);\n"
                                "            orc_feq(rho, vx, vy, feq);",
                                "double vx = ux + Fx / rho, vy = uy + Fy / rho;\n"
                                "            orc_feq(rho, vx, vy, feq);"),
    "eos_dropped_cubic": ("double num = 1.0 + eta + eta * eta - eta * eta * eta;",
                          "double num = 1.0 + eta + eta * eta;"),
    "eos_attraction_sign": ("- a * rho * rho);", "+ a * rho * rho);"),
    "streaming_reversed": ("int xd = wrap(x + EX[a], nx), yd = wrap(y + EY[a], ny);",
                           "int xd = wrap(x - EX[a], nx), yd = wrap(y - EY[a], ny);"),
    "edm_relax_to_shifted": ("fstar[a] = f[a] - (f[a] - feq[a]) / tau + (feq_shift[a] - feq[a]);",
                             "fstar[a] = f[a] - (f[a] - feq_shift[a]) / tau + (feq_shift[a] - feq[a]);"),
    "sc_missing_tau": ("orc_feq(rho, ux + tau * Fx / rho, uy + tau * Fy / rho, feq);",
                       "orc_feq(rho, ux + Fx / rho, uy + Fy / rho, feq);"),
    "mrt_eps_row": ("M[2 * 9 + a] = 4.0 - 21.0 / 2.0 * e2", "M[2 * 9 + a] = 4.0 - 19.0 / 2.0 * e2"),
    "mrt_source_half": ("(1.0 - lam[k] / 2.0) * Sm[k]", "(1.0 - lam[k]) * Sm[k]"),
    "feq_u2_coefficient": ("- u2 / (2.0 * cs2));", "- u2 / cs2);"),
    "li_shift_sign": ("vx + c * Fx, vy + c * Fy, S);", "vx - c * Fx, vy - c * Fy, S);"),
    "li_psi_not_squared": ("double c = p->sigma / ((tau - 0.5) * psi * psi);",
                           "double c = p->sigma / ((tau - 0.5) * psi);"),
    "li_viscosity_denominator": ("double c = p->sigma / ((tau - 0.5) * psi * psi);",
                                 "double c = p->sigma / ((tau - 0.5) / 3.0 * psi * psi);"),
}


def _build(tmp_path, name, src_text):
    c = tmp_path / (name + ".c")
    c.write_text(src_text)
    so = tmp_path / (name + ".so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    return str(so)


def _pins_pass(so):
    env = dict(os.environ, ORACLE_SO=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode == 0, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    text = open(SRC).read()
    old, new = MUTATIONS[name]
    assert text.count(old) >= 1, "mutation anchor not found: %s" % name
    ok, out = _pins_pass(_build(tmp_path, name, text.replace(old, new)))
    assert not ok, "pins did not catch %s:\n%s" % (name, out)
