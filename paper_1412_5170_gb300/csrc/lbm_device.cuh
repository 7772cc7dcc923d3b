// lbm_device.cuh -- per-node arithmetic of the pseudo-potential D2Q9 update
// (Hu, Li & Uddin, arXiv:1412.5170), shared by every liblbm kernel.
//
// All functions work on population *deviations* g_a = f_a - w_a rho_ref with
// a compile-time compute type C.  The FP64 path uses rho_ref = 0 (so g = f);
// the FP32 path stores g in float so that vapour densities (~1e-3 of the
// liquid's) keep their significant digits.  Every formula below is linear in
// the w_a rho_ref shift, which therefore cancels exactly.
#pragma once
#include <cstdint>

namespace lbm {

enum : int { BGK = 0, MRT = 1 };
enum : int { GUO = 0, EDM = 1, SC = 2 };
enum : unsigned { ST_NONFINITE = 1u, ST_EOS = 2u, ST_TIMEOUT = 4u };

// D2Q9 velocities (Sec. 2): 0 rest, 1-4 axes, 5-8 diagonals.
__host__ __device__ constexpr int ex(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int ey(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }
template <typename C>
__host__ __device__ constexpr C wt(int a) { return a == 0 ? C(4) / C(9) : (a < 5 ? C(1) / C(9) : C(1) / C(36)); }

// Division, reciprocal and square root in the compute type: CUDA's fast
// single-precision intrinsics for float (a few ulp, far below the FP32
// path's tolerances), IEEE operations for double.
__device__ __forceinline__ float cdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double cdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float csqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double csqrt(double a) { return sqrt(a); }

// Per-lattice constants in the compute type.
template <typename C>
struct Coef {
    C T;          // absolute temperature (T/Tc) * Tc
    C K;          // EOS scale (Eq. 30)
    C half_A;     // A/2      (Eq. 6 potential term with U = -psi^2/2)
    C one_m_A;    // 1 - A    (Eq. 6 effective-density term)
    C omega;      // 1/tau
    C tau;
    C guo_pre;    // 1 - 1/(2 tau)  (Eq. 23)
    C s_e, s_eps, s_q;  // MRT rates (Eq. 35); s_nu = omega
    C rho_ref;    // deviation reference (0 for FP64)
};

// psi from the K-scaled Carnahan-Starling EOS (Eqs. 29-30, a = 1, b = 4,
// R = 1, so eta = b rho / 4 = rho) through Eq. 7 with G = -1:
//   psi^2 = 2 (rho/3 - p).  Out-of-domain densities set ST_EOS and give 0.
template <typename C>
__device__ __forceinline__ C psi_of_rho(C rho, const Coef<C>& k, unsigned& bad)
{
    const C eta = rho;
    const C one_m = C(1) - eta;
    const C num = C(1) + eta * (C(1) + eta * (C(1) - eta));
    const C den = one_m * one_m * one_m;
    const C p = k.K * (rho * k.T * cdiv(num, den) - rho * rho);
    const C s = C(2) * (rho * (C(1) / C(3)) - p);
    const bool ok = (rho > C(0)) && (rho < C(1)) && (s >= C(0));
    if (!ok) bad |= ST_EOS;
    return ok ? csqrt(s) : C(0);
}

// Kupershtokh's hybrid force (Eq. 6) with G = -1, U = -psi^2/2 and the
// nearest-neighbour weights w(1) = 1/3, w(2) = 1/12 (Eq. 4):
//   F = (A/2) sum_a w_a psi^2(x+e_a) e_a + (1 - A) psi(x) sum_a w_a psi(x+e_a) e_a.
// Neighbour psi values by compass point (E = +x, N = +y).
template <typename C>
struct Stencil { C c, e, n, w, s, ne, nw, sw, se; };

template <typename C>
__device__ __forceinline__ void force(const Stencil<C>& q, const Coef<C>& k, C& Fx, C& Fy)
{
    const C w1 = C(1) / C(3), w2 = C(1) / C(12);
    const C sx1 = w1 * (q.e - q.w) + w2 * ((q.ne - q.sw) + (q.se - q.nw));
    const C sy1 = w1 * (q.n - q.s) + w2 * ((q.ne - q.sw) + (q.nw - q.se));
    const C e2 = q.e * q.e, w2s = q.w * q.w, n2 = q.n * q.n, s2 = q.s * q.s;
    const C ne2 = q.ne * q.ne, nw2 = q.nw * q.nw, sw2 = q.sw * q.sw, se2 = q.se * q.se;
    const C sx2 = w1 * (e2 - w2s) + w2 * ((ne2 - sw2) + (se2 - nw2));
    const C sy2 = w1 * (n2 - s2) + w2 * ((ne2 - sw2) + (nw2 - se2));
    Fx = k.half_A * sx2 + k.one_m_A * q.c * sx1;
    Fy = k.half_A * sy2 + k.one_m_A * q.c * sy1;
}

// Moments of the deviations (Eq. 3): drho = sum g (rho = rho_ref + drho),
// j = sum g e (the w_a rho_ref shift has zero first moment).
template <typename C>
__device__ __forceinline__ void moments(const C g[9], C& drho, C& jx, C& jy)
{
    drho = ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
    jx = (g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]));
    jy = (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
}

// Deviation equilibrium (Eq. 2 minus w_a rho_ref):
//   w_a [drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)]
template <typename C>
__device__ __forceinline__ C feq_dev(int a, C drho, C rho, C ux, C uy, C usq15)
{
    const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
    return wt<C>(a) * (drho + rho * (C(3) * eu + C(4.5) * eu * eu - usq15));
}

// Collision of one node.  In: g (pulled deviations at time t), F.  Out: g
// becomes the post-collision deviations; vx, vy receive v = u + F/(2 rho).
template <typename C, int COLL, int FORC>
__device__ __forceinline__ void collide(C g[9], C Fx, C Fy, const Coef<C>& k, C& vx, C& vy, C& rho_out)
{
    C drho, jx, jy;
    moments(g, drho, jx, jy);
    const C rho = k.rho_ref + drho;
    const C inv_rho = cdiv(C(1), rho);
    const C ux = jx * inv_rho, uy = jy * inv_rho;
    vx = ux + C(0.5) * Fx * inv_rho;
    vy = uy + C(0.5) * Fy * inv_rho;
    rho_out = rho;

    if constexpr (COLL == BGK && FORC == GUO) {
        // Eqs. 1, 2, 23: relax to f^eq(rho, v), add Guo's source.
        const C usq = C(1.5) * (vx * vx + vy * vy);
        const C vF3 = C(3) * (vx * Fx + vy * Fy);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const C eF = C(ex(a)) * Fx + C(ey(a)) * Fy;
            const C ev = C(ex(a)) * vx + C(ey(a)) * vy;
            const C S = wt<C>(a) * k.guo_pre * (C(3) * eF + C(9) * ev * eF - vF3);
            const C fe = feq_dev<C>(a, drho, rho, vx, vy, usq);
            g[a] = g[a] + k.omega * (fe - g[a]) + S;
        }
    } else if constexpr (COLL == BGK && FORC == EDM) {
        // Eqs. 1, 22: relax to f^eq(rho, u), add f^eq(rho, u + du) - f^eq(rho, u),
        // du = F/rho, written out as the exact difference of the two quadratics.
        const C usq = C(1.5) * (ux * ux + uy * uy);
        const C dux = Fx * inv_rho, duy = Fy * inv_rho;
        const C dq = C(1.5) * (dux * (C(2) * ux + dux) + duy * (C(2) * uy + duy));
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
            const C edu = C(ex(a)) * dux + C(ey(a)) * duy;
            const C diff = wt<C>(a) * rho * (C(3) * edu + C(4.5) * edu * (C(2) * eu + edu) - dq);
            const C fe = feq_dev<C>(a, drho, rho, ux, uy, usq);
            g[a] = g[a] + k.omega * (fe - g[a]) + diff;
        }
    } else if constexpr (COLL == BGK && FORC == SC) {
        // Eqs. 20-21: relax to f^eq(rho, u + tau F / rho); no source term.
        const C uex = ux + k.tau * Fx * inv_rho, uey = uy + k.tau * Fy * inv_rho;
        const C usq = C(1.5) * (uex * uex + uey * uey);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const C fe = feq_dev<C>(a, drho, rho, uex, uey, usq);
            g[a] = g[a] + k.omega * (fe - g[a]);
        }
    } else {
        static_assert(COLL == MRT && FORC == GUO, "MRT supports Guo forcing only");
        // Eq. 34 in the orthogonal D2Q9 moment basis (rho, e, eps, jx, qx, jy,
        // qy, pxx, pxy), with m, m^eq and S = M (Guo source / (1 - 1/2tau)) in
        // closed form.  Deviations shift m by -rho_ref (1, -2, 1, 0, ..., 0).
        const C m1 = -C(4) * g[0] - ((g[1] + g[3]) + (g[2] + g[4])) + C(2) * ((g[5] + g[7]) + (g[6] + g[8]));
        const C m2 = C(4) * g[0] - C(2) * ((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
        const C m4 = -C(2) * (g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]));
        const C m6 = -C(2) * (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
        const C m7 = (g[1] + g[3]) - (g[2] + g[4]);
        const C m8 = (g[5] + g[7]) - (g[6] + g[8]);
        const C v2 = vx * vx + vy * vy;
        const C rv2 = C(3) * rho * v2;
        const C eq1 = -C(2) * drho + rv2;        // rho(-2 + 3v^2) + 2 rho_ref
        const C eq2 = drho - rv2;                // rho(1 - 3v^2) - rho_ref
        const C eq4 = -rho * vx, eq6 = -rho * vy;
        const C eq7 = rho * (vx * vx - vy * vy), eq8 = rho * vx * vy;
        const C vF = vx * Fx + vy * Fy;
        const C S1 = C(6) * vF, S2 = -C(6) * vF, S4 = -Fx, S6 = -Fy;
        const C S7 = C(2) * (vx * Fx - vy * Fy), S8 = vx * Fy + vy * Fx;
        const C s_nu = k.omega;
        // m* = m - s (m - m^eq) + (1 - s/2) S; rho and j come out as drho, j + F.
        const C a0 = drho;
        const C a1 = m1 - k.s_e * (m1 - eq1) + (C(1) - C(0.5) * k.s_e) * S1;
        const C a2 = m2 - k.s_eps * (m2 - eq2) + (C(1) - C(0.5) * k.s_eps) * S2;
        const C a3 = jx + Fx;
        const C a4 = m4 - k.s_q * (m4 - eq4) + (C(1) - C(0.5) * k.s_q) * S4;
        const C a5 = jy + Fy;
        const C a6 = m6 - k.s_q * (m6 - eq6) + (C(1) - C(0.5) * k.s_q) * S6;
        const C a7 = m7 - s_nu * (m7 - eq7) + (C(1) - C(0.5) * s_nu) * S7;
        const C a8 = m8 - s_nu * (m8 - eq8) + (C(1) - C(0.5) * s_nu) * S8;
        // f* = M^-1 m* with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
        const C b0 = a0 * (C(1) / C(9)), b1 = a1 * (C(1) / C(36)), b2 = a2 * (C(1) / C(36));
        const C b3 = a3 * (C(1) / C(6)), b4 = a4 * (C(1) / C(12));
        const C b5 = a5 * (C(1) / C(6)), b6 = a6 * (C(1) / C(12));
        const C b7 = a7 * C(0.25), b8 = a8 * C(0.25);
        const C axis = b0 - b1 - C(2) * b2;      // common part of e1..e4
        const C diag = b0 + C(2) * b1 + b2;      // common part of e5..e8
        const C px = b3 - C(2) * b4, py = b5 - C(2) * b6;
        const C dx = b3 + b4, dy = b5 + b6;
        g[0] = b0 - C(4) * b1 + C(4) * b2;
        g[1] = axis + px + b7;
        g[3] = axis - px + b7;
        g[2] = axis + py - b7;
        g[4] = axis - py - b7;
        g[5] = diag + dx + dy + b8;
        g[6] = diag - dx + dy - b8;
        g[7] = diag - dx - dy + b8;
        g[8] = diag + dx - dy - b8;
    }
    // Every scheme conserves mass (sum f* = rho).  Close the rest population
    // on it so that rounding in the equilibrium weights (4/9, 1/9, 1/36 and
    // the 1/9 of M^-1 are inexact in binary) cannot bias the mass step after
    // step; the residual is one unbiased rounding of g[0].
    g[0] = drho - (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8])));
}

// Status bits of a node after collision: non-finite output.
template <typename C>
__device__ __forceinline__ unsigned finite_bits(const C g[9])
{
    C s = C(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) s += g[a];
    return isfinite(s) ? 0u : ST_NONFINITE;
}

}  // namespace lbm
