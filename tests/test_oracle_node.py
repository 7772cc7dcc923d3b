"""Pins of the oracle's node-level arithmetic: equilibrium (Eq. 2), Guo source
(Eq. 23), the three forcing schemes (Eqs. 20-23) and MRT (Eqs. 34-36), checked
against the moment identities that define them and against exact identities
the paper states."""
import itertools

import numpy as np
import pytest

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
RNG = np.random.default_rng(1412)


def moments(f):
    f = np.asarray(f)
    m0 = f.sum()
    m1 = (f[:, None] * E).sum(0)
    m2 = np.einsum("a,ai,aj->ij", f, E, E)
    return m0, m1, m2


def random_states(n=20):
    for _ in range(n):
        rho = RNG.uniform(0.002, 0.45)
        u = RNG.uniform(-0.1, 0.1, 2)
        F = RNG.uniform(-1e-3, 1e-3, 2) * rho
        yield rho, u, F


def test_feq_moments(orc):
    """Eq. 2 is the D2Q9 equilibrium: sum f = rho, sum f e = rho u,
    sum f e e = rho u u + rho c_s^2 I with c_s^2 = 1/3."""
    for rho, u, _ in random_states():
        m0, m1, m2 = moments(orc.feq(rho, *u))
        assert m0 == pytest.approx(rho, rel=1e-15)
        np.testing.assert_allclose(m1, rho * u, rtol=0, atol=1e-16)
        np.testing.assert_allclose(m2, rho * np.outer(u, u) + rho / 3 * np.eye(2), rtol=0, atol=2e-16)


def test_guo_source_moments(orc):
    """Eq. 23: sum F_a = 0, sum F_a e = (1 - 1/2tau) F,
    sum F_a e e = (1 - 1/2tau)(v F + F v)."""
    for rho, v, F in random_states():
        tau = RNG.uniform(0.55, 1.5)
        pre = 1 - 1 / (2 * tau)
        m0, m1, m2 = moments(orc.guo_source(pre, *F, *v))
        assert abs(m0) < 1e-19
        np.testing.assert_allclose(m1, pre * F, rtol=1e-13, atol=1e-20)
        np.testing.assert_allclose(m2, pre * (np.outer(v, F) + np.outer(F, v)), rtol=1e-12, atol=1e-20)


SCHEMES = [("bgk", "guo"), ("bgk", "edm"), ("bgk", "sc"), ("mrt", "guo")]


@pytest.mark.parametrize("coll,forc", SCHEMES)
def test_collision_conserves_mass_and_adds_force(orc, coll, forc):
    """Every scheme: sum f* = rho and sum f* e = rho u + F (Eqs. 21-25:
    the force enters the momentum balance exactly once per step)."""
    for rho, u, F in random_states():
        tau = RNG.uniform(0.55, 1.5)
        p = orc.params(4, 4, 0.7, tau, -0.152, 1.0, coll, forc, s_e=0.8, s_eps=0.8, s_q=1.1)
        f = orc.feq(rho, *u) * (1 + RNG.uniform(-0.05, 0.05, 9))
        rho_f, j, _ = moments(f)
        uf = j / rho_f
        fs = orc.collide_node(p, f, rho_f, *uf, *F)
        m0, m1, _ = moments(fs)
        assert m0 == pytest.approx(rho_f, rel=1e-13)
        np.testing.assert_allclose(m1, j + F, rtol=0, atol=1e-13 * rho_f)


def test_sc_equals_edm_at_tau_one(orc):
    """Sec. 4.2.1: the SC and EDM schemes give identical results at tau = 1
    (both reduce to f* = f^eq(rho, u + F/rho))."""
    for rho, u, F in random_states():
        f = orc.feq(rho, *u) * (1 + RNG.uniform(-0.05, 0.05, 9))
        r, j, _ = moments(f)
        a = orc.collide_node(orc.params(4, 4, 0.7, 1.0, -0.1, 1, "bgk", "sc"), f, r, *(j / r), *F)
        b = orc.collide_node(orc.params(4, 4, 0.7, 1.0, -0.1, 1, "bgk", "edm"), f, r, *(j / r), *F)
        np.testing.assert_allclose(a, b, rtol=0, atol=2e-16)
        np.testing.assert_allclose(a, orc.feq(r, *(j / r + F / r)), rtol=0, atol=2e-16)


def test_mrt_with_equal_rates_is_bgk(orc):
    """Eq. 34 with Lambda = I/tau is the LBGK equation with Guo's source (Eq. 23)."""
    for rho, u, F in random_states():
        tau = RNG.uniform(0.55, 1.5)
        f = orc.feq(rho, *u) * (1 + RNG.uniform(-0.05, 0.05, 9))
        r, j, _ = moments(f)
        s = 1 / tau
        a = orc.collide_node(orc.params(4, 4, .7, tau, -.1, 1, "mrt", "guo", s_e=s, s_eps=s, s_q=s),
                             f, r, *(j / r), *F)
        b = orc.collide_node(orc.params(4, 4, .7, tau, -.1, 1, "bgk", "guo"), f, r, *(j / r), *F)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-16)


def test_mrt_matrix_rows(orc):
    """The transform of Eq. 34: rows 1, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy are
    mutually orthogonal, the conserved rows give rho and j, and the inverse is exact."""
    M = orc.mrt_matrix()
    G = M @ M.T
    np.testing.assert_allclose(G - np.diag(np.diag(G)), 0, atol=0)
    np.testing.assert_allclose(np.diag(G), [9, 36, 36, 6, 12, 6, 12, 4, 4])
    np.testing.assert_array_equal(M[3], E[:, 0])
    np.testing.assert_array_equal(M[5], E[:, 1])
    np.testing.assert_allclose(orc.invert9(M) @ M, np.eye(9), atol=1e-15)


def test_mrt_equilibrium_moments_closed_form(orc):
    """m^eq = M f^eq(rho, v) has the textbook D2Q9 closed form
    (rho, rho(-2 + 3v^2), rho(1 - 3v^2), rho vx, -rho vx, rho vy, -rho vy,
    rho(vx^2 - vy^2), rho vx vy) -- checks the e and eps rows' polynomials."""
    M = orc.mrt_matrix()
    for rho, v, _ in random_states():
        v2 = v @ v
        want = [rho, rho * (-2 + 3 * v2), rho * (1 - 3 * v2), rho * v[0], -rho * v[0],
                rho * v[1], -rho * v[1], rho * (v[0] ** 2 - v[1] ** 2), rho * v[0] * v[1]]
        np.testing.assert_allclose(M @ orc.feq(rho, *v), want, rtol=1e-13, atol=1e-17)


def test_mrt_nonconserved_rates_matter_only_off_equilibrium(orc):
    """At equilibrium with F = 0 every MRT rate choice returns f unchanged."""
    f = orc.feq(0.3, 0.02, -0.01)
    r, j, _ = moments(f)
    for se, sq in itertools.product((0.8, 1.3), (1.1, 1.7)):
        p = orc.params(4, 4, .7, 0.8, -.1, 1, "mrt", "guo", s_e=se, s_eps=se, s_q=sq)
        np.testing.assert_allclose(orc.collide_node(p, f, r, *(j / r), 0.0, 0.0), f, atol=1e-16)


def test_li_collision_moments(orc):
    """Eq. 31 at one node: the collision conserves mass, adds F to the
    momentum exactly once, and its second moment carries, beyond Guo's,
    the shift (1 - 1/2tau) * 2 sigma F F / ((tau - 1/2) psi^2) that sets
    Eq. 32's eps (the sigma term is what distinguishes Li et al.'s model)."""
    for rho, u, F in random_states():
        tau = RNG.uniform(0.6, 1.5)
        psi = RNG.uniform(0.05, 0.4)
        sigma = 0.105
        f = orc.feq(rho, *u) * (1 + RNG.uniform(-0.05, 0.05, 9))
        rho_f, j, _ = moments(f)
        uf = j / rho_f
        li = orc.collide_node(orc.params(4, 4, 0.7, tau, 0.0, 1.0, "bgk", "li", sigma=sigma), f, rho_f, *uf, *F, psi)
        guo = orc.collide_node(orc.params(4, 4, 0.7, tau, 0.0, 1.0, "bgk", "guo"), f, rho_f, *uf, *F)
        m0, m1, m2 = moments(li)
        g0, g1, g2 = moments(guo)
        assert m0 == pytest.approx(rho_f, rel=1e-14)
        np.testing.assert_allclose(m1, j + F, rtol=1e-12, atol=1e-18)
        shift = (1 - 1 / (2 * tau)) * 2 * sigma * np.outer(F, F) / ((tau - 0.5) * psi ** 2)
        np.testing.assert_allclose(m2 - g2, shift, rtol=1e-6, atol=1e-16)   # a difference of O(0.1) moments
