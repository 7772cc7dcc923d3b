"""Pins of the oracle's interaction force (Eq. 6 with U = G psi^2/2, G = -1,
weights w(1) = 1/3, w(2) = 1/12 of Eq. 4) against its Taylor expansion
(Eq. 10), exact stencil symmetries and the periodic-sum identity."""
import numpy as np
import pytest


def test_uniform_psi_gives_zero_force(orc):
    psi = np.full((7, 9), 0.37)
    Fx, Fy = orc.force(psi, -0.3)
    assert np.abs(Fx).max() == 0.0 and np.abs(Fy).max() == 0.0


def test_force_sums_to_zero_on_periodic_lattice(orc):
    """The stencil of Eq. 6 is antisymmetric under e -> -e, so on a periodic lattice
    sum_x F(x) = 0: total momentum is conserved."""
    rng = np.random.default_rng(7)
    psi = rng.uniform(0.05, 0.4, (11, 13))
    for A in (-0.84, -0.152, 0.0, 0.4):
        Fx, Fy = orc.force(psi, A)
        scale = np.abs(Fx).max()
        assert abs(Fx.sum()) < 1e-14 * scale * psi.size
        assert abs(Fy.sum()) < 1e-14 * scale * psi.size


def _eq10_plane_wave(orc, N, A, direction):
    """Max residual of the stencil force against the three Taylor terms of Eq. 10
    (G = -1, c = 1, e2 = 1) for psi = g(s) = p0 + d sin(k s), s = n . x.

    With n the integer lattice direction, grad psi = n g', grad^2 psi = |n|^2 g''
    and grad(grad^2 psi) = n |n|^2 g''', so Eq. 10 reads
        F = n [ g g' + (1/6) |n|^2 g g''' + (A/2) |n|^2 g'' g' ].
    """
    nx_, ny_ = direction
    k = 2 * np.pi / N
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    s = nx_ * x + ny_ * y
    p0, d = 0.3, 0.05
    g = p0 + d * np.sin(k * s)
    g1 = d * k * np.cos(k * s)
    g2 = -d * k * k * np.sin(k * s)
    g3 = -d * k ** 3 * np.cos(k * s)
    n2 = nx_ * nx_ + ny_ * ny_
    bracket = g * g1 + g * n2 * g3 / 6.0 + (A / 2.0) * n2 * g2 * g1
    Fx, Fy = orc.force(g, A)
    return max(np.abs(Fx - nx_ * bracket).max(), np.abs(Fy - ny_ * bracket).max())


@pytest.mark.parametrize("direction", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("A", [-0.84, -0.26, 0.5])
def test_force_matches_eq10_to_fifth_order(orc, direction, A):
    """Eq. 10: F3 = -G c^2 [psi grad psi + (e2 c^2/6) psi grad(grad^2 psi)
    + (A e2 c^2/2)(grad^2 psi) grad psi] + O(d^5).  With the right weights and the
    sign of A as written in Eq. 6 the residual falls by 2^5 per refinement; a
    wrong A sign, or D2Q9 weights in place of w(1) = 1/3, w(2) = 1/12, leaves a
    residual of third order or lower."""
    r = [_eq10_plane_wave(orc, N, A, direction) for N in (32, 64, 128)]
    rate1, rate2 = r[0] / r[1], r[1] / r[2]
    assert rate1 > 28 and rate2 > 28, (r, rate1, rate2)
    assert r[2] < 1e-9
