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
enum : int { GUO = 0, EDM = 1, SC = 2, LI = 3 };
enum : unsigned { ST_NONFINITE = 1u, ST_EOS = 2u, ST_TIMEOUT = 4u, ST_ALIGN = 8u };

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
// Square root of a >= 0 (0 maps to 0).
__device__ __forceinline__ float csqrt(float a) { return a > 0.f ? a * rsqrtf(a) : 0.f; }
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
    C li_c;       // sigma / (tau - 1/2): Li et al.'s v' = v + li_c F / psi^2 (Eq. 31)
    // MRT relaxation of moment m with rate s, equilibrium m^eq and source S,
    // already divided by the squared norm n of its row of M (M^-1 = M^T / n):
    //   (m - s (m - m^eq) + (1 - s/2) S) / n = r0 m + r1 m^eq + r2 S
    // rows: 0 = e (s_e, n 36), 1 = eps (s_eps, 36), 2 = q (s_q, 12), 3 = nu (1/tau, 4)
    C r0[4], r1[4], r2[4];
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

// Both terms share the neighbour sum, so F = sum_a w_a e_a phi(x+e_a) with
// phi(n) = psi(n) [(A/2) psi(n) + (1 - A) psi(x)].
template <typename C>
__device__ __forceinline__ void force(const Stencil<C>& q, const Coef<C>& k, C& Fx, C& Fy)
{
    const C w1 = C(1) / C(3), w2 = C(1) / C(12);
    const C cc = k.one_m_A * q.c;
    const C pe = q.e * (k.half_A * q.e + cc), pw = q.w * (k.half_A * q.w + cc);
    const C pn = q.n * (k.half_A * q.n + cc), ps = q.s * (k.half_A * q.s + cc);
    const C pne = q.ne * (k.half_A * q.ne + cc), psw = q.sw * (k.half_A * q.sw + cc);
    const C pse = q.se * (k.half_A * q.se + cc), pnw = q.nw * (k.half_A * q.nw + cc);
    const C d1 = pne - psw, d2 = pse - pnw;
    Fx = w1 * (pe - pw) + w2 * (d1 + d2);
    Fy = w1 * (pn - ps) + w2 * (d1 - d2);
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

// Collision of one node.  In: g (pulled deviations at time t), F, psi at the
// node (used by Li et al.'s model only).  Out: g becomes the post-collision
// deviations; vx, vy receive v = u + F/(2 rho).
template <typename C, int COLL, int FORC>
__device__ __forceinline__ void collide(C g[9], C Fx, C Fy, const Coef<C>& k, C& vx, C& vy, C& rho_out, C psi)
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
    } else if constexpr (COLL == BGK && FORC == LI) {
        // Eq. 31 (Li et al.): as Guo, with v' = v + sigma F / ((tau - 1/2) psi^2)
        // in the second-order part of the source; F is Eq. 4's (A = 0).
        const C c = cdiv(k.li_c, psi * psi);
        const C wx = vx + c * Fx, wy = vy + c * Fy;
        const C usq = C(1.5) * (vx * vx + vy * vy);
        const C wF3 = C(3) * (wx * Fx + wy * Fy);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const C eF = C(ex(a)) * Fx + C(ey(a)) * Fy;
            const C ew = C(ex(a)) * wx + C(ey(a)) * wy;
            const C S = wt<C>(a) * k.guo_pre * (C(3) * eF + C(9) * ew * eF - wF3);
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
        // qy, pxx, pxy) with m, m^eq and S = M (Guo source / (1 - 1/2tau)) in
        // closed form; each relaxed moment comes out already scaled by 1/n of
        // its row, ready for f* = M^T (m* / n).  Deviations shift m by
        // -rho_ref (1, -2, 1, 0, ..., 0), which the equilibria absorb.
        const C Sa = g[1] + g[3], Sb = g[2] + g[4], Sc = g[5] + g[7], Sd = g[6] + g[8];
        const C axis = Sa + Sb, diag = Sc + Sd;
        const C D1 = g[1] - g[3], D2 = g[2] - g[4], D57 = g[5] - g[7], D86 = g[8] - g[6];
        const C m1 = C(2) * diag - axis - C(4) * g[0];
        const C m2 = diag - C(2) * axis + C(4) * g[0];
        const C m4 = (D57 + D86) - C(2) * D1;
        const C m6 = (D57 - D86) - C(2) * D2;
        const C m7 = Sa - Sb, m8 = Sc - Sd;
        const C vx2 = vx * vx, vy2 = vy * vy;
        const C rv2 = C(3) * rho * (vx2 + vy2);
        const C vF6 = C(6) * (vx * Fx + vy * Fy);
        const C b1 = k.r0[0] * m1 + k.r1[0] * (rv2 - C(2) * drho) + k.r2[0] * vF6;
        const C b2 = k.r0[1] * m2 + k.r1[1] * (drho - rv2) - k.r2[1] * vF6;
        const C b4 = k.r0[2] * m4 - k.r1[2] * (rho * vx) - k.r2[2] * Fx;
        const C b6 = k.r0[2] * m6 - k.r1[2] * (rho * vy) - k.r2[2] * Fy;
        const C b7 = k.r0[3] * m7 + k.r1[3] * (rho * (vx2 - vy2)) + k.r2[3] * (C(2) * (vx * Fx - vy * Fy));
        const C b8 = k.r0[3] * m8 + k.r1[3] * (rho * vx * vy) + k.r2[3] * (vx * Fy + vy * Fx);
        const C b0 = drho * (C(1) / C(9));
        const C b3 = (jx + Fx) * (C(1) / C(6)), b5 = (jy + Fy) * (C(1) / C(6));
        const C ax = b0 - b1 - C(2) * b2;      // common part of e1..e4
        const C dg = b0 + C(2) * b1 + b2;      // common part of e5..e8
        const C px = b3 - C(2) * b4, py = b5 - C(2) * b6;
        const C dx = b3 + b4, dy = b5 + b6;
        g[1] = ax + px + b7;
        g[3] = ax - px + b7;
        g[2] = ax + py - b7;
        g[4] = ax - py - b7;
        g[5] = dg + (dx + dy) + b8;
        g[7] = dg - (dx + dy) + b8;
        g[6] = dg - (dx - dy) - b8;
        g[8] = dg + (dx - dy) - b8;
        // row 0 of M^-1 = M^T / n: f0 = m0/9 - 4 m_e/36 + 4 m_eps/36 (FP64;
        // the FP32 path closes g[0] on the mass below)
        if constexpr (sizeof(C) != sizeof(float)) g[0] = b0 - C(4) * b1 + C(4) * b2;
    }
    // Every scheme conserves mass (sum f* = rho).  In FP32 the rest population
    // is closed on it, so that rounding in the equilibrium weights (4/9, 1/9,
    // 1/36 and the 1/9 of M^-1 are inexact in binary) cannot bias the mass
    // step after step; the residual is one unbiased rounding of g[0].  In FP64
    // that bias is about 1e-16 of the mass per step and g[0] keeps its own
    // formula: closing it would conserve mass better than any FP64 evaluation
    // of Eqs. 23 and 34 written out term by term, and drift from one by about
    // 1e-15 of rho per step.
    if constexpr (sizeof(C) == sizeof(float))
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
