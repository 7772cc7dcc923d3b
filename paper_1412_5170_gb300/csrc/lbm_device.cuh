// lbm_device.cuh -- per-node arithmetic of the pseudo-potential D2Q9 update
// (Hu, Li & Uddin, arXiv:1412.5170), shared by every liblbm kernel.
//
// All functions work on population *deviations* g_a = f_a - w_a rho_ref with
// a compile-time compute type C.  The FP64 path uses rho_ref = 0 (so g = f);
// the FP32 path stores g in float so that vapour densities (~1e-3 of the
// liquid's) keep their significant digits.  Every formula below is linear in
// the w_a rho_ref shift, which therefore cancels exactly.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

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

// ---------------------------------------------------------------------------
// FP32 arithmetic without biased constants.
//
// Near T/Tc = 0.5 with a small EOS scale K the vapour density of the model is
// very sensitive to the effective temperature: a change of the pressure by
// about 1e-8 rho moves rho_v by ~1e-4 of itself.  Float cannot hold 1/3, 1/12,
// 1/6 (each rounds up by 3.0e-8 of itself) nor the D2Q9 weights 4/9, 1/9,
// 1/36 (up by 7.45e-9), and a rounded constant scales the same term at every
// node and every step by the same factor -- the force, the kinetic pressure
// rho/3, the momentum source -- which is such a pressure change.  The FP32
// step therefore applies every such constant either as an exact integer
// (36 w_a = 16, 4, 1; the MRT row norms divide 36) or as an unevaluated sum
// hi + lo of two floats (hi = float(c), lo = float(c - hi)) through one fused
// multiply-add, and refines the hardware's approximate division and square
// root by one Newton step.  What is left are roundings whose sign varies
// from node to node.  Measured on the host copy of this arithmetic (64^2
// droplet, T/Tc = 0.5, K = 1/16, 30 000 steps) the vapour density moves from
// 1e-4 to a few 1e-6 of the FP64 oracle's.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fma_rn(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
// a / b, 1 / b and sqrt(s) to about one ulp without the special-case
// branches of the correctly rounded operations: the hardware approximation
// followed by one Newton correction -- for the quotient q = a y (y ~ 1/b)
// the residual r = a - b q, exact in one fused multiply-add, gives q + r y
// (Markstein's correction); for the root r = s y (y ~ 1/sqrt(s)) Heron's
// step r + (s - r^2) y/2.  The operands here are normal floats (densities in
// (0, 1), their EOS terms, psi^2 > 0).  The host build (tests) uses the IEEE
// operations.
__device__ __forceinline__ float div_nr(float a, float b)
{
#ifdef __CUDA_ARCH__
    const float y = __fdividef(1.0f, b);
    const float q = a * y;
    return fma_rn(fma_rn(-b, q, a), y, q);
#else
    return a / b;
#endif
}
__device__ __forceinline__ float rcp_nr(float b)
{
#ifdef __CUDA_ARCH__
    const float y = __fdividef(1.0f, b);
    return fma_rn(fma_rn(-b, y, 1.0f), y, y);
#else
    return 1.0f / b;
#endif
}
__device__ __forceinline__ float sqrt_nr(float s)   // s > 0
{
#ifdef __CUDA_ARCH__
    const float y = rsqrtf(s);
    const float r = s * y;
    return fma_rn(fma_rn(-r, r, s), 0.5f * y, r);
#else
    return std::sqrt(s);
#endif
}
// The bits of a float as an unsigned integer.
__device__ __forceinline__ unsigned float_bits(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    unsigned u;
    std::memcpy(&u, &x, sizeof u);
    return u;
#endif
}
// x c for a constant c = hi + lo held as two floats.
__device__ __forceinline__ float mul_split(float x, float hi, float lo) { return fma_rn(x, hi, x * lo); }
constexpr float kTwoThirdsHi = 0x1.555556p-1f, kTwoThirdsLo = -0x1.555556p-26f;   // 2/3
constexpr float kTwelfthHi = 0x1.555556p-4f, kTwelfthLo = -0x1.555556p-29f;       // 1/12
constexpr float k36thHi = 0x1.c71c72p-6f, k36thLo = -0x1.c71c72p-33f;             // 1/36
constexpr float kNinthHi = 0x1.c71c72p-4f, kNinthLo = -0x1.c71c72p-31f;           // 1/9
constexpr float kSixthHi = 0x1.555556p-3f, kSixthLo = -0x1.555556p-28f;           // 1/6
// 36 w_a: the D2Q9 weights as exact integers.
__host__ __device__ constexpr float w36(int a) { return a == 0 ? 16.f : (a < 5 ? 4.f : 1.f); }

// Per-lattice constants in the compute type.
template <typename C>
struct Coef {
    C T;          // absolute temperature (T/Tc) * Tc
    C K;          // EOS scale (Eq. 30)
    C half_A;     // A/2      (Eq. 6 potential term with U = -psi^2/2)
    C one_m_A;    // 1 - A    (Eq. 6 effective-density term)
    C omega;      // 1/tau
    C tau;
    C guo_pre;    // 1 - 1/(2 tau)  (Eq. 23); FP32: 1 - omega/2 exactly
    C s_e, s_eps, s_q;  // MRT rates (Eq. 35); s_nu = omega
    C rho_ref;    // deviation reference (0 for FP64)
    C li_c;       // sigma / (tau - 1/2): Li et al.'s v' = v + li_c F / psi^2 (Eq. 31)
    // MRT relaxation of moment m with rate s, equilibrium m^eq and source S,
    // already divided by the squared norm n of its row of M (M^-1 = M^T / n):
    //   (m - s (m - m^eq) + (1 - s/2) S) / n = r0 m + r1 m^eq + r2 S
    // rows: 0 = e (s_e, n 36), 1 = eps (s_eps, 36), 2 = q (s_q, 12), 3 = nu (1/tau, 4)
    // (FP64 path; the FP32 path relaxes with the rates themselves)
    C r0[4], r1[4], r2[4];
    // FP32 path only (see "FP32 arithmetic without biased constants"):
    C A;          // Eq. 6 weight
    C tau_lo;     // tau + tau_lo = 1/omega (Shan-Chen shift: omega tau F = F exactly)
    C h_e, h_eps, h_q;   // 1 - s/2 of the MRT rates s_e, s_eps, s_q (Eq. 34's source factor), in float
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
    if constexpr (sizeof(C) == sizeof(float)) {
        // psi^2 = 2 rho/3 - 2 K rho (T q - rho), q the CS quotient: 2/3 as
        // hi + lo, q Newton-refined, and T q - rho (a small difference in the
        // liquid) in one fused multiply-add
        const float q = div_nr(num, den);
        const float s = fma_rn(-2.f * k.K * rho, fma_rn(k.T, q, -rho), mul_split(rho, kTwoThirdsHi, kTwoThirdsLo));
        // 0 < rho < 1 in one unsigned compare of the bits (negative values,
        // zero and NaN fall outside)
        const bool in = float_bits(rho) - 1u < float_bits(1.0f) - 1u;
        if (!(in && s >= 0.f)) bad |= ST_EOS;
        return (in && s > 0.f) ? sqrt_nr(s) : 0.f;
    } else {
        const C p = k.K * (rho * k.T * cdiv(num, den) - rho * rho);
        const C s = C(2) * (rho * (C(1) / C(3)) - p);
        const bool ok = (rho > C(0)) && (rho < C(1)) && (s >= C(0));
        if (!ok) bad |= ST_EOS;
        return ok ? csqrt(s) : C(0);
    }
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
    if constexpr (sizeof(C) == sizeof(float)) {
        // The same sum regrouped so that no rounded coefficient scales the
        // leading term: F = psi(x) sum w psi(x+e) e + A sum w e psi(x+e)
        // (psi(x+e)/2 - psi(x)), and per opposite pair (n, n')
        //   phi(n) - phi(n') = (psi_n - psi_n') [psi(x) + A ((psi_n + psi_n')/2 - psi(x))],
        // whose difference is exact and whose A term is of higher order;
        // then F = (1/12) [4 (axis pair) + (diagonal pairs)].
        const float c = q.c;
        const float dx = (q.e - q.w) * fma_rn(k.A, 0.5f * (q.e + q.w) - c, c);
        const float dy = (q.n - q.s) * fma_rn(k.A, 0.5f * (q.n + q.s) - c, c);
        const float d1 = (q.ne - q.sw) * fma_rn(k.A, 0.5f * (q.ne + q.sw) - c, c);
        const float d2 = (q.se - q.nw) * fma_rn(k.A, 0.5f * (q.se + q.nw) - c, c);
        Fx = mul_split(4.f * dx + (d1 + d2), kTwelfthHi, kTwelfthLo);
        Fy = mul_split(4.f * dy + (d1 - d2), kTwelfthHi, kTwelfthLo);
    } else {
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
}

// Moments of the deviations (Eq. 3): drho = sum g (rho = rho_ref + drho),
// j = sum g e (the w_a rho_ref shift has zero first moment).
template <typename C>
__device__ __forceinline__ void momentum(const C g[9], C& jx, C& jy)
{
    jx = (g[1] - g[3]) + ((g[5] - g[7]) + (g[8] - g[6]));
    jy = (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
}
template <typename C>
__device__ __forceinline__ void moments(const C g[9], C& drho, C& jx, C& jy)
{
    drho = ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
    momentum(g, jx, jy);
}
// Sum of the eight moving deviations, the tree the FP32 step's density and
// mass closure share.
__device__ __forceinline__ float moving_sum(const float g[9])
{
    return ((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
}

// Deviation equilibrium (Eq. 2 minus w_a rho_ref):
//   w_a [drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)]
template <typename C>
__device__ __forceinline__ C feq_dev(int a, C drho, C rho, C ux, C uy, C usq15)
{
    const C eu = C(ex(a)) * ux + C(ey(a)) * uy;
    return wt<C>(a) * (drho + rho * (C(3) * eu + C(4.5) * eu * eu - usq15));
}

// FP32 collision, every scheme.  The D2Q9 weights enter as the integers
// w36 = 36 w_a, and every product that carries a term of the size of rho
// (the equilibria, Guo's and the exact-difference sources, the MRT moments of
// rho, e, eps and j) is scaled by 1/36 (1/9, 1/6) held as hi + lo; the
// momentum a step adds is then F exactly up to rounding (omega and
// 1 - omega/2 are exact floats, see make_coef).  The moments, velocities and
// relaxations are those of the FP64 collision below (same equations, same
// readings); only the placement of the constants differs.  The reciprocal
// 1/rho is Newton-refined: the exact-difference and Shan-Chen schemes take
// their momentum source through it.
template <int COLL, int FORC>
__device__ __forceinline__ void collide_f32(float g[9], float Fx, float Fy, const Coef<float>& k, float& vx,
                                            float& vy, float& rho_out, float psi)
{
    // density: the rest deviation plus the moving ones' sum, which the mass
    // closure at the end reuses (sum9, the psi pass's density, adds in the
    // same order in FP32)
    const float g0_old = g[0];
    const float s_old = moving_sum(g);
    const float drho = g0_old + s_old;
    float jx, jy;
    momentum(g, jx, jy);
    const float rho = k.rho_ref + drho;
    const float inv_rho = rcp_nr(rho);
    const float ux = jx * inv_rho, uy = jy * inv_rho;
    // v = u + F/(2 rho).  (Written as (j + F/2)/rho, algebraically the same,
    // a narrow FP32 slab's total momentum wandered 50 times further from
    // zero -- 6e-5 against 1e-6 over 1e5 steps -- and the slab drifted.)
    vx = ux + 0.5f * Fx * inv_rho;
    vy = uy + 0.5f * Fy * inv_rho;
    rho_out = rho;
    if constexpr (COLL == BGK && (FORC == GUO || FORC == LI)) {
        // Eqs. 1, 2, 23 (Li et al.: Eq. 31, v' in the source's second-order
        // term): omega f^eq + S = w36 (omega X + (1 - omega/2) Y) / 36, with
        // X = (f^eq - w rho_ref)/w and Y = S / (w (1 - omega/2)); then
        // f* = f + [(omega f^eq + S) - omega f], the bracket in one rounding.
        float wx = vx, wy = vy;
        if constexpr (FORC == LI) {
            const float c = cdiv(k.li_c, psi * psi);
            wx = vx + c * Fx;
            wy = vy + c * Fy;
        }
        const float usq = 1.5f * (vx * vx + vy * vy);
        const float wF3 = 3.f * (wx * Fx + wy * Fy);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const float eF = float(ex(a)) * Fx + float(ey(a)) * Fy;
            const float ev = float(ex(a)) * vx + float(ey(a)) * vy;
            const float ew = float(ex(a)) * wx + float(ey(a)) * wy;
            const float X = drho + rho * (3.f * ev + 4.5f * ev * ev - usq);
            const float Y = 3.f * eF + 9.f * ew * eF - wF3;
            const float Z = w36(a) * fma_rn(k.omega, X, k.guo_pre * Y);
            g[a] = g[a] + fma_rn(-k.omega, g[a], mul_split(Z, k36thHi, k36thLo));
        }
    } else if constexpr (COLL == BGK && FORC == EDM) {
        // Eqs. 1, 22: omega f^eq(u) + [f^eq(u + du) - f^eq(u)] = w36 (omega X + D) / 36
        const float usq = 1.5f * (ux * ux + uy * uy);
        const float dux = Fx * inv_rho, duy = Fy * inv_rho;
        const float dq = 1.5f * (dux * (2.f * ux + dux) + duy * (2.f * uy + duy));
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const float eu = float(ex(a)) * ux + float(ey(a)) * uy;
            const float edu = float(ex(a)) * dux + float(ey(a)) * duy;
            const float X = drho + rho * (3.f * eu + 4.5f * eu * eu - usq);
            const float D = rho * (3.f * edu + 4.5f * edu * (2.f * eu + edu) - dq);
            const float Z = w36(a) * fma_rn(k.omega, X, D);
            g[a] = g[a] + fma_rn(-k.omega, g[a], mul_split(Z, k36thHi, k36thLo));
        }
    } else if constexpr (COLL == BGK && FORC == SC) {
        // Eqs. 20-21, the shift tau F / rho with tau = 1/omega as hi + lo
        const float tx = Fx * inv_rho, ty = Fy * inv_rho;
        const float uex = ux + mul_split(tx, k.tau, k.tau_lo), uey = uy + mul_split(ty, k.tau, k.tau_lo);
        const float usq = 1.5f * (uex * uex + uey * uey);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const float eu = float(ex(a)) * uex + float(ey(a)) * uey;
            const float X = w36(a) * (drho + rho * (3.f * eu + 4.5f * eu * eu - usq));
            g[a] = g[a] + k.omega * (mul_split(X, k36thHi, k36thLo) - g[a]);
        }
    } else {
        static_assert(COLL == MRT && FORC == GUO, "MRT supports Guo forcing only");
        // Eq. 34 in the orthogonal basis (rho, e, eps, jx, qx, jy, qy, pxx,
        // pxy): m* = m - s (m - m^eq) + (1 - s/2) S per moment, the conserved
        // ones m0* = drho and j* = j + F (s_rho = s_j = 1), each divided by
        // its row norm n (M^-1 = M^T / n).  The norms 9, 36 and 6 of the
        // moments of the size of rho (rho, e, eps, j) are applied as hi + lo;
        // q (n = 12) and the stresses (n = 4, exact) carry only velocity and
        // force terms.
        const float Sa = g[1] + g[3], Sb = g[2] + g[4], Sc = g[5] + g[7], Sd = g[6] + g[8];
        const float axis = Sa + Sb, diag = Sc + Sd;
        const float D1 = g[1] - g[3], D2 = g[2] - g[4], D57 = g[5] - g[7], D86 = g[8] - g[6];
        const float m1 = 2.f * diag - axis - 4.f * g[0];
        const float m2 = diag - 2.f * axis + 4.f * g[0];
        const float m4 = (D57 + D86) - 2.f * D1;
        const float m6 = (D57 - D86) - 2.f * D2;
        const float m7 = Sa - Sb, m8 = Sc - Sd;
        const float vx2 = vx * vx, vy2 = vy * vy;
        const float rv2 = 3.f * rho * (vx2 + vy2);
        const float vF6 = 6.f * (vx * Fx + vy * Fy);
        const float se = k.s_e, sp = k.s_eps, sq = k.s_q, sn = k.omega;
        const float b0 = mul_split(drho, kNinthHi, kNinthLo);
        // the factors 1 - s/2 come precomputed (k.h_*, and 1 - omega/2 = k.guo_pre), the
        // same floats the expressions would give, so that no node spends an instruction on them
        const float b1 = mul_split((m1 - se * (m1 - (rv2 - 2.f * drho))) + k.h_e * vF6, k36thHi, k36thLo);
        const float b2 = mul_split((m2 - sp * (m2 - (drho - rv2))) - k.h_eps * vF6, k36thHi, k36thLo);
        const float b3 = mul_split(jx + Fx, kSixthHi, kSixthLo), b5 = mul_split(jy + Fy, kSixthHi, kSixthLo);
        const float b4 = ((m4 - sq * (m4 + rho * vx)) - k.h_q * Fx) * (1.f / 12.f);
        const float b6 = ((m6 - sq * (m6 + rho * vy)) - k.h_q * Fy) * (1.f / 12.f);
        const float b7 = 0.25f * ((m7 - sn * (m7 - rho * (vx2 - vy2))) + k.guo_pre * (2.f * (vx * Fx - vy * Fy)));
        const float b8 = 0.25f * ((m8 - sn * (m8 - rho * vx * vy)) + k.guo_pre * (vx * Fy + vy * Fx));
        const float ax = b0 - b1 - 2.f * b2;      // common part of e1..e4
        const float dg = b0 + 2.f * b1 + b2;      // common part of e5..e8
        const float px = b3 - 2.f * b4, py = b5 - 2.f * b6;
        const float dx = b3 + b4, dy = b5 + b6;
        g[1] = ax + px + b7;
        g[3] = ax - px + b7;
        g[2] = ax + py - b7;
        g[4] = ax - py - b7;
        g[5] = dg + (dx + dy) + b8;
        g[7] = dg - (dx + dy) + b8;
        g[6] = dg - (dx - dy) - b8;
        g[8] = dg + (dx - dy) - b8;
    }
    // Every scheme conserves mass (sum f* = rho).  The rest population takes
    // up what the other eight gave or took: g0 + (s_old - s_new), the two
    // sums over the same tree.  Its rounding is then of the size of this
    // step's change, and nil where the node no longer changes -- whereas
    // closing g0 on the moment drho (drho - s_new) leaves the roundings of the
    // two large sums in every step, the same at every node of a uniform
    // region: a flat FP32 slab of 8 x 127 nodes then gained mass at 1.6e-4
    // of itself per 8e4 steps and its vapour density drifted by 2e-4 (7e-6
    // and 3e-5 with this form; both measured on the host copy of this code).
    g[0] = g0_old + (s_old - moving_sum(g));
}

// FP64 collision (the compute type C is double), every scheme.
template <typename C, int COLL, int FORC>
__device__ __forceinline__ void collide_f64(C g[9], C Fx, C Fy, const Coef<C>& k, C& vx, C& vy, C& rho_out, C psi)
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
        // row 0 of M^-1 = M^T / n: f0 = m0/9 - 4 m_e/36 + 4 m_eps/36
        g[0] = b0 - C(4) * b1 + C(4) * b2;
    }
    // The rest population keeps its own formula here (the FP32 collision
    // closes it on the mass instead): in FP64 the weights' rounding biases the
    // mass by about 1e-16 per step, and closing g[0] would conserve mass better
    // than any FP64 evaluation of Eqs. 23 and 34 written out term by term,
    // drifting from one by about 1e-15 of rho per step.
}

// Collision of one node.  In: g (pulled deviations at time t), F, psi at the
// node (used by Li et al.'s model only).  Out: g becomes the post-collision
// deviations; vx, vy receive v = u + F/(2 rho).
template <typename C, int COLL, int FORC>
__device__ __forceinline__ void collide(C g[9], C Fx, C Fy, const Coef<C>& k, C& vx, C& vy, C& rho_out, C psi)
{
    if constexpr (sizeof(C) == sizeof(float)) collide_f32<COLL, FORC>(g, Fx, Fy, k, vx, vy, rho_out, psi);
    else collide_f64<C, COLL, FORC>(g, Fx, Fy, k, vx, vy, rho_out, psi);
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
