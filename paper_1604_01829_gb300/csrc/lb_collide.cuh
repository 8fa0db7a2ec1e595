// Collision of one node (Sec. 1.1 of Ustach & Faller, arXiv:1604.01829),
// shared by the fused collide-and-stream kernels.
#pragma once

#include "lb_internal.h"

namespace lbk {

// ---------------------------------------------------------------- collision
// Post-collision populations of one node, in place. Force F = uniform + spread
// bead force; u = (j + F/2) / rho (Guo forcing); MRT in the orthogonal
// D3Q19 moment basis 1, c, c^2-1, 3cx^2-c^2, cy^2-cz^2, cxcy, cycz, czcx,
// (3c^2-5)c, (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz, 3c^4-6c^2+1,
// (2c^2-3)(3cx^2-c^2), (2c^2-3)(cy^2-cz^2), with norms b_k = sum w e_k^2.
template <typename R, bool DEV, int COLL, bool NOISE>
__device__ __forceinline__ void collide(R (&f)[19], R Fx, R Fy, R Fz, const CollParams<R> &a, uint2 key,
                                        uint32_t instance, uint32_t node, uint32_t step) {
    const R s1 = f[1] + f[2], d1 = f[1] - f[2];
    const R s3 = f[3] + f[4], d3 = f[3] - f[4];
    const R s5 = f[5] + f[6], d5 = f[5] - f[6];
    const R s7 = f[7] + f[8], d7 = f[7] - f[8];
    const R s9 = f[9] + f[10], d9 = f[9] - f[10];
    const R s11 = f[11] + f[12], d11 = f[11] - f[12];
    const R s13 = f[13] + f[14], d13 = f[13] - f[14];
    const R s15 = f[15] + f[16], d15 = f[15] - f[16];
    const R s17 = f[17] + f[18], d17 = f[17] - f[18];
    const R Sax = s1 + s3 + s5;
    const R Sxy = s7 + s9, Sxz = s11 + s13, Syz = s15 + s17;
    const R Sd = Sxy + Sxz + Syz;
    const R m0 = f[0] + Sax + Sd;                      // rho, or rho - rho0 for deviations
    const R rho = DEV ? a.rho0 + m0 : m0;
    const R jx = d1 + d7 + d9 + d11 + d13;
    const R jy = d3 + d7 - d9 + d15 + d17;
    const R jz = d5 + d11 - d13 + d15 - d17;
    R ir;
    if constexpr (sizeof(R) == 4) ir = __fdividef(1.0f, rho); else ir = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * ir;
    const R uy = (jy + R(0.5) * Fy) * ir;
    const R uz = (jz + R(0.5) * Fz) * ir;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R uu = ux * ux + uy * uy + uz * uz;
    constexpr R w0 = R(1.0 / 3.0), w1 = R(1.0 / 18.0), w2 = R(1.0 / 36.0);

    if (COLL == 0) {
        // BGK: f* = f - (f - f_eq)/tau + (1 - 1/(2 tau)) w [3(c-u) + 9 (c.u) c].F
        const R om = a.omega, h = R(1) - R(0.5) * om;
        const R base = DEV ? m0 : rho;                 // w rho (or w (rho - rho0)) coefficient of '1'
        const R k2 = R(1.5) * uu;
        // rest population
        f[0] = f[0] - om * (f[0] - w0 * (base - rho * k2)) + h * w0 * (R(-3) * uF);
        auto pair = [&](int i, R cu, R cF, R w) {
            const R e = w * (base + rho * (R(4.5) * cu * cu - k2));
            const R o = w * rho * R(3) * cu;
            const R se = w * (R(9) * cu * cF - R(3) * uF);
            const R so = w * R(3) * cF;
            f[i] = f[i] - om * (f[i] - (e + o)) + h * (se + so);
            f[i + 1] = f[i + 1] - om * (f[i + 1] - (e - o)) + h * (se - so);
        };
        pair(1, ux, Fx, w1);
        pair(3, uy, Fy, w1);
        pair(5, uz, Fz, w1);
        pair(7, ux + uy, Fx + Fy, w2);
        pair(9, ux - uy, Fx - Fy, w2);
        pair(11, ux + uz, Fx + Fz, w2);
        pair(13, ux - uz, Fx - Fz, w2);
        pair(15, uy + uz, Fy + Fz, w2);
        pair(17, uy - uz, Fy - Fz, w2);
        return;
    }

    // MRT: non-conserved moments
    const R A5 = R(2) * s1 - s3 - s5, B5 = Sxy + Sxz - R(2) * Syz;
    const R A6 = s3 - s5, B6 = Sxy - Sxz;
    const R m4 = Sd - f[0];
    const R m5 = A5 + B5, m17 = B5 - A5;
    const R m6 = A6 + B6, m18 = B6 - A6;
    const R m7 = s7 - s9, m8 = s15 - s17, m9 = s11 - s13;
    const R m10 = R(-2) * d1 + d7 + d9 + d11 + d13;
    const R m11 = R(-2) * d3 + d7 - d9 + d15 + d17;
    const R m12 = R(-2) * d5 + d11 - d13 + d15 - d17;
    const R m13 = d7 + d9 - d11 - d13;
    const R m14 = -d7 + d9 + d15 + d17;
    const R m15 = d11 - d13 - d15 + d17;
    const R m16 = f[0] - R(2) * Sax + Sd;

    // Post-collision moments, each already multiplied by c_k = w_diag / b_k
    // (the host folds c_k into the rates): A_k = c_k ((1 - g_k) m_eq + g_k m
    // + (1 + g_k)/2 S_k + noise). Equilibrium stress moments rho u u and Guo
    // source moments (uF + Fu); ghost modes have zero equilibrium and source.
    const R ruu_x = rho * ux, ruu_y = rho * uy, ruu_z = rho * uz;
    const R e4 = ruu_x * ux + ruu_y * uy + ruu_z * uz;
    const R exx = ruu_x * ux, eyy = ruu_y * uy, ezz = ruu_z * uz;
    const R e5 = R(2) * exx - eyy - ezz, e6 = eyy - ezz;
    const R e7 = ruu_x * uy, e8 = ruu_y * uz, e9 = ruu_z * ux;
    const R uFx = ux * Fx, uFy = uy * Fy, uFz = uz * Fz;
    R q4 = a.ke[0] * e4 + a.km[0] * m4 + a.ks[0] * (R(2) * uF);
    R q5 = a.ke[1] * e5 + a.km[1] * m5 + a.ks[1] * (R(2) * (R(2) * uFx - uFy - uFz));
    R q6 = a.ke[2] * e6 + a.km[2] * m6 + a.ks[2] * (R(2) * (uFy - uFz));
    R q7 = a.ke[3] * e7 + a.km[3] * m7 + a.ks[3] * (ux * Fy + uy * Fx);
    R q8 = a.ke[4] * e8 + a.km[4] * m8 + a.ks[4] * (uy * Fz + uz * Fy);
    R q9 = a.ke[5] * e9 + a.km[5] * m9 + a.ks[5] * (uz * Fx + ux * Fz);
    R q10 = a.kg[0] * m10, q11 = a.kg[1] * m11, q12 = a.kg[2] * m12;
    R q13 = a.kg[3] * m13, q14 = a.kg[4] * m14, q15 = a.kg[5] * m15;
    R q16 = a.kg[6] * m16, q17 = a.kg[7] * m17, q18 = a.kg[8] * m18;

    if (NOISE) {
        // 15 non-conserved modes, variance 3 rho kT b_k (1 - g_k^2); kn_k holds
        // c_k sqrt(3 kT b_k (1 - g_k^2)) sqrt(12) (times 2^-32 in FP32). The
        // variates are 16-bit: two Philox calls give 16 half-words, mode 4 + j
        // takes half-word j (high half of word j/2 for even j, else the low
        // half), xi = sqrt(12) ((h + 1/2) 2^-16 - 1/2). In FP32 the half-word
        // and a 1/2 below it become the mantissa of y = 1 + (h + 1/2) 2^-16 in
        // [1, 2), and (y - 3/2) 2^32 = xi 2^32 / sqrt(12) is exact in one FMA
        // (no integer-to-float conversion).
        const uint4 r0 = philox4x32_10(make_uint4(node, step, instance, 0u), key);
        const uint4 r1 = philox4x32_10(make_uint4(node, step, instance, 1u), key);
        R sr;
        if constexpr (sizeof(R) == 4) asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sr) : "f"(rho));
        else sr = sqrt(rho);
        auto hi = [&](R &q, int k, uint32_t v) {
            if constexpr (sizeof(R) == 8) q += (sr * a.kn[k]) * centred16_d(v >> 16);
            else q = fmaf(sr * a.kn[k], fmaf(__uint_as_float(((v >> 9) & 0x7FFF80u) | 0x3F800040u), 0x1p32f, -0x1.8p32f), q);
        };
        auto lo = [&](R &q, int k, uint32_t v) {
            if constexpr (sizeof(R) == 8) q += (sr * a.kn[k]) * centred16_d(v & 0xFFFFu);
            else q = fmaf(sr * a.kn[k], fmaf(__uint_as_float(((v << 7) & 0x7FFF80u) | 0x3F800040u), 0x1p32f, -0x1.8p32f), q);
        };
        hi(q4, 0, r0.x); lo(q5, 1, r0.x); hi(q6, 2, r0.y); lo(q7, 3, r0.y);
        hi(q8, 4, r0.z); lo(q9, 5, r0.z); hi(q10, 6, r0.w); lo(q11, 7, r0.w);
        hi(q12, 8, r1.x); lo(q13, 9, r1.x); hi(q14, 10, r1.y); lo(q15, 11, r1.y);
        hi(q16, 12, r1.z); lo(q17, 13, r1.z); hi(q18, 14, r1.w);
    }

    // back to populations: f*_i = w_i sum_k e_k(c_i) m*_k / b_k; with the
    // c_k folded in, diagonal links are E +- O, axis links 2 (E +- O), rest 12 E
    constexpr R c0 = R(1.0 / 36.0), c1 = R(1.0 / 12.0);
    const R q0 = c0 * m0;
    const R q1 = c1 * (jx + Fx), q2 = c1 * (jy + Fy), q3 = c1 * (jz + Fz);
    f[0] = R(12) * (q0 - q4 + q16);
    const R U = q0 - R(2) * q16, V = q17 - q5, Wv = q6 - q18;
    {
        const R E = U - R(2) * V, O = q1 - R(2) * q10;
        f[1] = R(2) * (E + O); f[2] = R(2) * (E - O);
    }
    {
        const R E = U + V + Wv, O = q2 - R(2) * q11;
        f[3] = R(2) * (E + O); f[4] = R(2) * (E - O);
    }
    {
        const R E = U + V - Wv, O = q3 - R(2) * q12;
        f[5] = R(2) * (E + O); f[6] = R(2) * (E - O);
    }
    const R Ed = q0 + q4 + q16;
    const R S5 = q5 + q17, S6 = q6 + q18;
    const R T1 = Ed + S5 + S6, T2 = Ed + S5 - S6, T3 = Ed - R(2) * S5;
    const R P = q1 + q10, Q = q2 + q11, Rr = q3 + q12;
    {
        const R O = P + Q + q13 - q14;
        f[7] = T1 + q7 + O; f[8] = T1 + q7 - O;
    }
    {
        const R O = P - Q + q13 + q14;
        f[9] = T1 - q7 + O; f[10] = T1 - q7 - O;
    }
    {
        const R O = P + Rr - q13 + q15;
        f[11] = T2 + q9 + O; f[12] = T2 + q9 - O;
    }
    {
        const R O = P - Rr - q13 - q15;
        f[13] = T2 - q9 + O; f[14] = T2 - q9 - O;
    }
    {
        const R O = Q + Rr + q14 - q15;
        f[15] = T3 + q8 + O; f[16] = T3 + q8 - O;
    }
    {
        const R O = Q - Rr + q14 + q15;
        f[17] = T3 - q8 + O; f[18] = T3 - q8 - O;
    }
}

template <int COLL, bool NOISE>
__device__ __forceinline__ void collide_fp32(float (&f)[19], float Fx, float Fy, float Fz,
                                             const CollParams<float> &a, const FluidArgs &fa, uint32_t node,
                                             uint32_t step) {
    collide<float, true, COLL, NOISE>(f, Fx, Fy, Fz, a, make_uint2(fa.key0, fa.key1), fa.instance, node, step);
}

}  // namespace lbk
