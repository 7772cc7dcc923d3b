"""Independent 50-digit stepper for tiny lattices (test helper, not the oracle).

Written separately from ``oracle/lbm_oracle.c`` and structured differently on
purpose: nodes are dictionary entries, streaming is a push to x + e_a, the
equilibrium is evaluated from its moment form and MRT inverts M with mpmath.
Agreement with the C oracle on 4x4 and 5x3 lattices to ~1e-14 rules out
indexing, orientation and streaming mistakes in either.
"""
from mpmath import mp, mpf, sqrt

mp.dps = 50
EV = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WT = [mpf(4) / 9] + [mpf(1) / 9] * 4 + [mpf(1) / 36] * 4
WF = [mpf(0)] + [mpf(1) / 3] * 4 + [mpf(1) / 12] * 4   # w(|e|^2) of Eq. 4
CS2 = mpf(1) / 3


def tc():
    return mpf("0.18727") / mpf("0.4963") / 4


def pressure(r, T, K):
    return K * (r * T * (1 + r + r ** 2 - r ** 3) / (1 - r) ** 3 - r ** 2)


def feq(r, u):
    out = []
    for (ex, ey), w in zip(EV, WT):
        eu = ex * u[0] + ey * u[1]
        out.append(w * r * (1 + eu / CS2 + eu * eu / (2 * CS2 ** 2) - (u[0] ** 2 + u[1] ** 2) / (2 * CS2)))
    return out


def guo(pre, F, v):
    out = []
    for (ex, ey), w in zip(EV, WT):
        eF = ex * F[0] + ey * F[1]
        ev = ex * v[0] + ey * v[1]
        vF = v[0] * F[0] + v[1] * F[1]
        # (F_i v_j + v_i F_j)(e_i e_j - cs2 d_ij)/(2 cs2^2) = (2 eF ev - 2 cs2 vF)/(2 cs2^2)
        out.append(w * pre * (eF / CS2 + (eF * ev - CS2 * vF) / CS2 ** 2))
    return out


def mrt_M():
    rows = []
    polys = [lambda ex, ey: 1, lambda ex, ey: -4 + 3 * (ex * ex + ey * ey),
             lambda ex, ey: 4 - mpf(21) / 2 * (ex * ex + ey * ey) + mpf(9) / 2 * (ex * ex + ey * ey) ** 2,
             lambda ex, ey: ex, lambda ex, ey: (-5 + 3 * (ex * ex + ey * ey)) * ex,
             lambda ex, ey: ey, lambda ex, ey: (-5 + 3 * (ex * ex + ey * ey)) * ey,
             lambda ex, ey: ex * ex - ey * ey, lambda ex, ey: ex * ey]
    for pf in polys:
        rows.append([mpf(pf(ex, ey)) for ex, ey in EV])
    return mp.matrix(rows)


def step(f, nx, ny, prm):
    """f: dict {(a, x, y): mpf} of post-streaming populations; returns the next f."""
    T = mpf(prm["T_over_Tc"]) * tc()
    K, tau, A = mpf(prm["K"]), mpf(prm["tau"]), mpf(prm["A"])
    G = mpf(-1)
    rho, mom, psi = {}, {}, {}
    for x in range(nx):
        for y in range(ny):
            r = sum(f[(a, x, y)] for a in range(9))
            jx = sum(f[(a, x, y)] * EV[a][0] for a in range(9))
            jy = sum(f[(a, x, y)] * EV[a][1] for a in range(9))
            rho[(x, y)], mom[(x, y)] = r, (jx, jy)
            psi[(x, y)] = sqrt(2 * (r / 3 - pressure(r, T, K)))
    out = {}
    M = mrt_M() if prm["collision"] == "mrt" else None
    Minv = M ** -1 if M is not None else None
    for x in range(nx):
        for y in range(ny):
            Fx = Fy = mpf(0)
            for a in range(1, 9):
                nb = ((x + EV[a][0]) % nx, (y + EV[a][1]) % ny)
                U = G * psi[nb] ** 2 / 2
                term = -A * WF[a] * U - (1 - A) * G * psi[(x, y)] * WF[a] * psi[nb]
                Fx += term * EV[a][0]
                Fy += term * EV[a][1]
            r = rho[(x, y)]
            u = (mom[(x, y)][0] / r, mom[(x, y)][1] / r)
            F = (Fx, Fy)
            fl = [f[(a, x, y)] for a in range(9)]
            v = (u[0] + F[0] / (2 * r), u[1] + F[1] / (2 * r))
            if prm["collision"] == "mrt":
                lam = [1, prm["s_e"], prm["s_eps"], 1, prm["s_q"], 1, prm["s_q"], 1 / tau, 1 / tau]
                lam = [mpf(s) for s in lam]
                m = M * mp.matrix(fl)
                meq = M * mp.matrix(feq(r, v))
                S = M * mp.matrix(guo(mpf(1), F, v))
                ms = mp.matrix([m[k] - lam[k] * (m[k] - meq[k]) + (1 - lam[k] / 2) * S[k] for k in range(9)])
                fs = list(Minv * ms)
            elif prm["forcing"] == "guo":
                fe, src = feq(r, v), guo(1 - 1 / (2 * tau), F, v)
                fs = [fl[a] - (fl[a] - fe[a]) / tau + src[a] for a in range(9)]
            elif prm["forcing"] == "li":
                # Eq. 31: Guo's source with v' = v + sigma F / ((tau - 1/2) psi^2)
                c = mpf(prm["sigma"]) / ((tau - mpf(1) / 2) * psi[(x, y)] ** 2)
                vp = (v[0] + c * F[0], v[1] + c * F[1])
                fe, src = feq(r, v), guo(1 - 1 / (2 * tau), F, vp)
                fs = [fl[a] - (fl[a] - fe[a]) / tau + src[a] for a in range(9)]
            elif prm["forcing"] == "edm":
                fe = feq(r, u)
                fe2 = feq(r, (u[0] + F[0] / r, u[1] + F[1] / r))
                fs = [fl[a] - (fl[a] - fe[a]) / tau + fe2[a] - fe[a] for a in range(9)]
            else:
                fe = feq(r, (u[0] + tau * F[0] / r, u[1] + tau * F[1] / r))
                fs = [fl[a] - (fl[a] - fe[a]) / tau for a in range(9)]
            for a in range(9):
                out[(a, (x + EV[a][0]) % nx, (y + EV[a][1]) % ny)] = fs[a]
    return out
