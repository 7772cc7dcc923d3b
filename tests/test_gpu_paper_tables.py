"""The paper's static-bubble tables reproduced by the FP64 GPU path (itself
held to 1e-12 of the oracle): a gas bubble of R = 23 in a 100 x 100 periodic
liquid at T/Tc = 0.6, BGK, run 30 000 steps; rho_g at the centre node,
rho_l at the corner node, Us_max = max |v| (readings 10-11).

* Table 3 (Sec. 4.2.1, K = 0.5): its A column is Kupershtokh's own weight
  A_K, so Eq. 6 takes A = 2 A_K (reading 4); with that the printed rho_g,
  rho_l and Us_max are met to 0.1 %, 0.02 % and 2 %.
* Table 4 (Sec. 4.3.2, eps = 1.68, A = -0.84, K = 1, Guo): rho_g within 3 %
  (1.3-2.4 % low; the printed values sit between A = -0.84 and -0.86),
  rho_l within 0.6 % (0.45-0.58 % low), Us_max within 10 %.  At tau = 0.7 the spurious
  currents (Us ~ 0.12) push an interface node past the EOS domain (psi^2 <
  0), which the library reports; the densities still match.
* Table 5 (Li et al.'s model, sigma = 0.105): rho_g within 2 % at tau = 0.8
  and 1, 10 % at tau = 1.5; its rise with tau is reproduced.
* Table 7 (Sec. 4.4.2, MRT, "the same parameters as Table 4"): with Table 4's
  eps = 1.68 the MRT bubble keeps the BGK gas density (0.0043 against the
  printed 0.0021 -- at leading order the relaxation rates do not move the
  coexistence densities); the printed values follow eps = 1.4 (A = -0.7):
  rho_g within 7 % (0.1 %, 3.7 %, 6.5 % at tau_nu = 0.7, 1, 1.5 with the
  rates 0.8 / 0.8 / 1.1, which the paper does not state), rho_l within
  0.2 %, and rho_g falls with tau_nu as printed.  Us_max is not compared: it
  follows the unstated rates.
"""
import json
import os

import pytest

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def bubble(lbm, forcing, tau, A, K, sigma=0.0, steps=30000, collision="bgk"):
    p = lbm.make_params(100, 100, 0.6, tau, A, K, collision, forcing, "fp64", sigma=sigma,
                        s_e=0.8, s_eps=0.8, s_q=1.1)
    with lbm.Lattice(p) as lat:
        lat.init_preset("bubble", 23.0, seed=1)
        lat.autotune(3)   # the fastest kernel for this small lattice (the state does not advance)
        lat.step(steps)
        st = lat.stats()
    return st


@pytest.mark.parametrize("row", GOLD["table3"]["rows"], ids=lambda r: "%s-tau%g" % (r["forcing"], r["tau"]))
def test_table3_bubble_guo_and_edm(lbm, row):
    st = bubble(lbm, row["forcing"], row["tau"], 2 * row["A"], 0.5)
    assert st["status"] == 0
    assert st["rho_center"] == pytest.approx(row["rho_g"], rel=1e-3)
    assert st["rho_corner"] == pytest.approx(row["rho_l"], rel=2e-4)
    assert st["max_v"] == pytest.approx(row["us_max"], rel=0.02)


@pytest.mark.parametrize("row", GOLD["table4"]["rows"], ids=lambda r: "tau%g" % r["tau"])
def test_table4_kupershtokh_tau_sweep(lbm, row):
    st = bubble(lbm, "guo", row["tau"], -0.84, 1.0)
    assert st["status"] == (lbm.E_EOS_DOMAIN if row["tau"] == 0.7 else 0)
    assert st["rho_center"] == pytest.approx(row["rho_g"], rel=0.03)
    assert st["rho_corner"] == pytest.approx(row["rho_l"], rel=6e-3)
    assert st["max_v"] == pytest.approx(row["us_max"], rel=0.1)


def test_table5_li_tau_sweep(lbm):
    t5 = GOLD["table5"]
    rg = []
    for row in t5["rows"]:
        st = bubble(lbm, "li", row["tau"], 0.0, 1.0, sigma=t5["sigma"])
        assert st["status"] == 0
        rel = 0.02 if row["tau"] <= 1.0 else 0.1
        assert st["rho_center"] == pytest.approx(row["rho_g"], rel=rel)
        assert st["rho_corner"] == pytest.approx(row["rho_l"], rel=5e-3)
        assert st["max_v"] == pytest.approx(row["us_max"], rel=0.15)
        rg.append(st["rho_center"])
    assert rg[0] < rg[1] < rg[2]   # gas density rises with tau (Sec. 4.3.2)


def test_table7_mrt_bubble_follows_eps_1_4(lbm):
    rows = GOLD["table7"]["rows"]
    rg = []
    for row in rows:
        st = bubble(lbm, "guo", row["tau_nu"], -0.7, 1.0, collision="mrt")
        assert st["status"] == 0
        assert st["rho_center"] == pytest.approx(row["rho_g"], rel=0.07)
        assert st["rho_corner"] == pytest.approx(row["rho_l"], rel=2e-3)
        rg.append(st["rho_center"])
    assert rg[0] > rg[1] > rg[2]
    # Table 4's eps = 1.68 gives the BGK gas density again, twice the printed one
    st = bubble(lbm, "guo", 1.0, -0.84, 1.0, collision="mrt")
    assert st["rho_center"] > 1.8 * rows[1]["rho_g"]
