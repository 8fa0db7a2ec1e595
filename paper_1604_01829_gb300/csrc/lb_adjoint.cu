// Hand-written adjoint of the deterministic LB + raspberry step.
//
// Objective: J = (1/W) sum over the last W steps of V_axis of one body, the
// steady velocity of a colloid pulled by a constant force, whose drag is
// xi = F_ext / J (Eq. (stokesflow) read for a driven colloid, Sec. 2.3 of
// Ustach & Faller, arXiv:1604.01829). The driver returns dJ/dgamma (bead
// friction of Eq. (latticeboltzmannfriction)) and dJ/ds_b for every
// body-frame bead offset. Bodies must be fixed or translation-only (the
// orientation held), the fluid deterministic (kT = 0).
//
// Reverse pass per step n (natural-layout adjoint arrays, 19 + 3 per node):
//   bodies: second half kick reversed (lam F_tot, lam V', lam X');
//   fluid: streaming reversed as a pull from the downstream nodes (halfway
//     bounce-back swaps the link), then the collision reversed in moment
//     space (lam m* = M^-T lam*, relaxation, equilibrium and Guo source
//     derivatives, u = (j + F/2)/rho), giving lam f_n and lam F_node;
//   coupling: eight lanes per bead recompute u_b and F_b, then add the
//     spread and interpolation terms into lam f_n and lam F_prev with
//     atomics, accumulate dJ/dgamma and dJ/ds_b (trilinear weights are
//     differentiated piecewise);
//   bodies: kick-drift reversed.
// States come from a two-level checkpointing schedule: the forward sweep
// stores one snapshot every K steps; the reverse sweep re-runs each segment
// from its snapshot, taping every step of it, and walks it backwards. K
// follows from the number of checkpoint slots (c slots: K = ceil(T / c),
// memory c snapshots + K taped steps, one extra forward sweep).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lb_couple.cuh"
#include "lb_ctx.h"

namespace lbk {

template <typename R>
struct AdjParams {
    R rho0;
    R A[6];     // 1 - g_k, modes 4-9
    R H[6];     // (1 + g_k)/2, modes 4-9
    R G[15];    // g_k, modes 4-18
};

struct BodyAdj {
    double lX[3], lV[3], lFl[3];   // adjoints of X, V, F_last after the step being reversed
    double lXp[3], lVp[3], lFt[3]; // adjoints of X', V', F_tot within it
};

struct AdjArgs {
    Geom g;
    const void *fn;             // taped population buffer before step n (AA layout)
    bool odd;                   // parity of n
    const void *Fprev;          // taped spread force read by step n ([3][N], storage precision)
    const void *Fnew;           // taped spread force written by step n
    const double *gforce;       // uniform force density (3)
    const void *lam_in;         // adjoint of f_{n+1}, natural layout [19][N]
    void *lam_out;              // adjoint of f_n
    const void *lFp_in;         // adjoint of F_prev_{n+1} (= of F_new_n), [3][N]
    void *lFn;                  // adjoint of F_node of step n (work array)
    void *lFp_out;              // adjoint of F_prev_n
    AdjParams<double> pd;
    AdjParams<float> pf;
};

namespace {

// ------------------------------------------------------------ collision adjoint
template <typename R, bool DEV>
__device__ __forceinline__ void collide_adjoint(R (&lam)[19], const R (&f)[19], R Fx, R Fy, R Fz,
                                                const AdjParams<R> &P, R &lFx, R &lFy, R &lFz) {
    // forward quantities
    R m0 = f[0], jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        m0 += f[i];
        if (cx(i)) jx += cx(i) * f[i];
        if (cy(i)) jy += cy(i) * f[i];
        if (cz(i)) jz += cz(i) * f[i];
    }
    const R rho = DEV ? P.rho0 + m0 : m0;
    const R ir = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * ir, uy = (jy + R(0.5) * Fy) * ir, uz = (jz + R(0.5) * Fz) * ir;

    // lam m*_k = (1/b_k) sum_i w_i e_k(c_i) lam*_i: moments of g_i = w_i lam*_i
    R g[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) g[i] = R(wq(i)) * lam[i];
    const R s1 = g[1] + g[2], d1 = g[1] - g[2], s3 = g[3] + g[4], d3 = g[3] - g[4];
    const R s5 = g[5] + g[6], d5 = g[5] - g[6], s7 = g[7] + g[8], d7 = g[7] - g[8];
    const R s9 = g[9] + g[10], d9 = g[9] - g[10], s11 = g[11] + g[12], d11 = g[11] - g[12];
    const R s13 = g[13] + g[14], d13 = g[13] - g[14], s15 = g[15] + g[16], d15 = g[15] - g[16];
    const R s17 = g[17] + g[18], d17 = g[17] - g[18];
    const R Sax = s1 + s3 + s5, Sxy = s7 + s9, Sxz = s11 + s13, Syz = s15 + s17, Sd = Sxy + Sxz + Syz;
    const R A5 = R(2) * s1 - s3 - s5, B5 = Sxy + Sxz - R(2) * Syz, A6 = s3 - s5, B6 = Sxy - Sxz;
    const R L0 = g[0] + Sax + Sd;
    const R L1 = R(3) * (d1 + d7 + d9 + d11 + d13);
    const R L2 = R(3) * (d3 + d7 - d9 + d15 + d17);
    const R L3 = R(3) * (d5 + d11 - d13 + d15 - d17);
    const R L4 = R(1.5) * (Sd - g[0]);
    const R L5 = R(0.75) * (A5 + B5), L6 = R(2.25) * (A6 + B6);
    const R L7 = R(9) * (s7 - s9), L8 = R(9) * (s15 - s17), L9 = R(9) * (s11 - s13);
    const R L10 = R(1.5) * (R(-2) * d1 + d7 + d9 + d11 + d13);
    const R L11 = R(1.5) * (R(-2) * d3 + d7 - d9 + d15 + d17);
    const R L12 = R(1.5) * (R(-2) * d5 + d11 - d13 + d15 - d17);
    const R L13 = R(4.5) * (d7 + d9 - d11 - d13);
    const R L14 = R(4.5) * (-d7 + d9 + d15 + d17);
    const R L15 = R(4.5) * (d11 - d13 - d15 + d17);
    const R L16 = R(0.5) * (g[0] - R(2) * Sax + Sd);
    const R L17 = R(0.75) * (B5 - A5), L18 = R(2.25) * (B6 - A6);

    // relaxation: lam m_k = g_k lam m*_k
    const R a4 = P.G[0] * L4, a5 = P.G[1] * L5, a6 = P.G[2] * L6, a7 = P.G[3] * L7, a8 = P.G[4] * L8;
    const R a9 = P.G[5] * L9, a10 = P.G[6] * L10, a11 = P.G[7] * L11, a12 = P.G[8] * L12;
    const R a13 = P.G[9] * L13, a14 = P.G[10] * L14, a15 = P.G[11] * L15, a16 = P.G[12] * L16;
    const R a17 = P.G[13] * L17, a18 = P.G[14] * L18;

    // equilibrium stress rho u u and Guo source (uF + Fu) of modes 4-9
    R lux = 0, luy = 0, luz = 0, lrho = 0;
    lFx = 0; lFy = 0; lFz = 0;
    {
        const R l = L4, A = P.A[0], H = P.H[0];
        lux += l * (R(2) * A * rho * ux + R(2) * H * Fx);
        luy += l * (R(2) * A * rho * uy + R(2) * H * Fy);
        luz += l * (R(2) * A * rho * uz + R(2) * H * Fz);
        lrho += l * A * (ux * ux + uy * uy + uz * uz);
        lFx += l * R(2) * H * ux; lFy += l * R(2) * H * uy; lFz += l * R(2) * H * uz;
    }
    {
        const R l = L5, A = P.A[1], H = P.H[1];
        lux += l * (R(4) * A * rho * ux + R(4) * H * Fx);
        luy += l * (R(-2) * A * rho * uy - R(2) * H * Fy);
        luz += l * (R(-2) * A * rho * uz - R(2) * H * Fz);
        lrho += l * A * (R(2) * ux * ux - uy * uy - uz * uz);
        lFx += l * R(4) * H * ux; lFy -= l * R(2) * H * uy; lFz -= l * R(2) * H * uz;
    }
    {
        const R l = L6, A = P.A[2], H = P.H[2];
        luy += l * (R(2) * A * rho * uy + R(2) * H * Fy);
        luz += l * (R(-2) * A * rho * uz - R(2) * H * Fz);
        lrho += l * A * (uy * uy - uz * uz);
        lFy += l * R(2) * H * uy; lFz -= l * R(2) * H * uz;
    }
    {
        const R l = L7, A = P.A[3], H = P.H[3];
        lux += l * (A * rho * uy + H * Fy);
        luy += l * (A * rho * ux + H * Fx);
        lrho += l * A * ux * uy;
        lFx += l * H * uy; lFy += l * H * ux;
    }
    {
        const R l = L8, A = P.A[4], H = P.H[4];
        luy += l * (A * rho * uz + H * Fz);
        luz += l * (A * rho * uy + H * Fy);
        lrho += l * A * uy * uz;
        lFy += l * H * uz; lFz += l * H * uy;
    }
    {
        const R l = L9, A = P.A[5], H = P.H[5];
        luz += l * (A * rho * ux + H * Fx);
        lux += l * (A * rho * uz + H * Fz);
        lrho += l * A * uz * ux;
        lFz += l * H * ux; lFx += l * H * uz;
    }
    // conserved: m*_0 = rho, m*_a = j_a + F_a
    lrho += L0;
    R ljx = L1, ljy = L2, ljz = L3;
    lFx += L1; lFy += L2; lFz += L3;
    // u = (j + F/2) / rho
    ljx += lux * ir; ljy += luy * ir; ljz += luz * ir;
    lFx += R(0.5) * lux * ir; lFy += R(0.5) * luy * ir; lFz += R(0.5) * luz * ir;
    lrho -= (lux * ux + luy * uy + luz * uz) * ir;

    // lam f_i = sum_k e_k(c_i) lam m_k, lam m_0 = lam rho, lam m_a = lam j_a
    const R q0 = lrho;
    lam[0] = q0 - a4 + a16;
    {
        const R E = q0 + R(2) * a5 - R(2) * a16 - R(2) * a17, O = ljx - R(2) * a10;
        lam[1] = E + O; lam[2] = E - O;
    }
    {
        const R E = q0 - a5 + a6 - R(2) * a16 + a17 - a18, O = ljy - R(2) * a11;
        lam[3] = E + O; lam[4] = E - O;
    }
    {
        const R E = q0 - a5 - a6 - R(2) * a16 + a17 + a18, O = ljz - R(2) * a12;
        lam[5] = E + O; lam[6] = E - O;
    }
    const R Ed = q0 + a4 + a16;
    {
        const R E = Ed + a5 + a6 + a7 + a17 + a18, O = ljx + ljy + a10 + a11 + a13 - a14;
        lam[7] = E + O; lam[8] = E - O;
    }
    {
        const R E = Ed + a5 + a6 - a7 + a17 + a18, O = ljx - ljy + a10 - a11 + a13 + a14;
        lam[9] = E + O; lam[10] = E - O;
    }
    {
        const R E = Ed + a5 - a6 + a9 + a17 - a18, O = ljx + ljz + a10 + a12 - a13 + a15;
        lam[11] = E + O; lam[12] = E - O;
    }
    {
        const R E = Ed + a5 - a6 - a9 + a17 - a18, O = ljx - ljz + a10 - a12 - a13 - a15;
        lam[13] = E + O; lam[14] = E - O;
    }
    {
        const R E = Ed - R(2) * a5 + a8 - R(2) * a17, O = ljy + ljz + a11 + a12 + a14 - a15;
        lam[15] = E + O; lam[16] = E - O;
    }
    {
        const R E = Ed - R(2) * a5 - a8 - R(2) * a17, O = ljy - ljz + a11 - a12 + a14 + a15;
        lam[17] = E + O; lam[18] = E - O;
    }
}

// One thread per node: pull the adjoint of the post-collision populations
// from the downstream nodes, reverse the collision.
template <typename T>
__global__ void __launch_bounds__(128) k_adj_collide(const AdjArgs a) {
    using R = T;
    constexpr bool DEV = sizeof(T) == 4;
    const Geom &g = a.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const long long N = g.N;
    const long long n = nidx(g, x, y, z);
    const T *lin = static_cast<const T *>(a.lam_in);
    T *lout = static_cast<T *>(a.lam_out);
    T *lFn = static_cast<T *>(a.lFn);
    const T *lFpin = static_cast<const T *>(a.lFp_in);
    if (is_wall(g, x, y, z)) {
#pragma unroll
        for (int i = 0; i < 19; ++i) lout[i * N + n] = T(0);
        for (int c = 0; c < 3; ++c) lFn[c * N + n] = T(0);
        return;
    }
    R lam[19], f[19];
    const T *fn = static_cast<const T *>(a.fn);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int xd = wrapm(x + cx(i), g.nx), yd = wrapm(y + cy(i), g.ny), zd = wrapm(z + cz(i), g.nz);
        lam[i] = is_wall(g, xd, yd, zd) ? lin[opp(i) * N + n] : lin[i * N + nidx(g, xd, yd, zd)];
        f[i] = (R)load_pre(fn, g, x, y, z, n, i, a.odd);
    }
    const T *Fnew = static_cast<const T *>(a.Fnew);
    const R Fx = (R)(a.gforce[0] + (double)Fnew[n]), Fy = (R)(a.gforce[1] + (double)Fnew[N + n]);
    const R Fz = (R)(a.gforce[2] + (double)Fnew[2 * N + n]);
    R lFx, lFy, lFz;
    if constexpr (DEV) collide_adjoint<R, true>(lam, f, Fx, Fy, Fz, a.pf, lFx, lFy, lFz);
    else collide_adjoint<R, false>(lam, f, Fx, Fy, Fz, a.pd, lFx, lFy, lFz);
#pragma unroll
    for (int i = 0; i < 19; ++i) lout[i * N + n] = lam[i];
    // F_node = g + F_new: its adjoint adds to that of F_new (which F_prev_{n+1} also is)
    lFn[n] = lFpin[n] + lFx;
    lFn[N + n] = lFpin[N + n] + lFy;
    lFn[2 * N + n] = lFpin[2 * N + n] + lFz;
}

template <typename T>
__global__ void k_zero(T *p, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = T(0);
}

struct AdjCouple {
    Geom g;
    const void *fn;
    bool odd;
    double rho0, gamma;
    const double *gforce;
    const void *Fprev;
    const void *lFn;            // adjoint of F_node of step n
    void *lam_f;                // adjoint of f_n (accumulated)
    void *lFp;                  // adjoint of F_prev_n (accumulated)
    const double *s;
    const int *bead_body;
    const Body *bodies;         // taped bodies before step n
    BodyAdj *adj;
    double *dJds;
    double *lgam;
    int nbeads;
};

// eight lanes per bead, as the forward coupling
template <typename T>
__global__ void __launch_bounds__(128) k_adj_couple(const AdjCouple a) {
    using R = T;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t >> 3, c = t & 7;
    const bool active = k < a.nbeads;
    const Geom &g = a.g;
    const T *fn = static_cast<const T *>(a.fn);
    const int body = active ? a.bead_body[k] : 0;
    const Body &B = a.bodies[body];
    // kinematics of the step (translation-only or fixed bodies)
    double Xp[3], Vp[3], Rm[9], wl[3];
    for (int q = 0; q < 3; ++q) {
        if (B.fixed == 2) {
            Vp[q] = B.V[q] + 0.5 * B.F_last[q] / B.mass;
            Xp[q] = B.X[q] + Vp[q];
        } else {
            Vp[q] = B.V[q];
            Xp[q] = B.X[q];
        }
    }
    quat_to_R(B.q, Rm);
    const double w0[3] = {B.fixed == 2 ? 0.0 : B.w[0], B.fixed == 2 ? 0.0 : B.w[1], B.fixed == 2 ? 0.0 : B.w[2]};
    for (int q = 0; q < 3; ++q) wl[q] = Rm[3 * q] * w0[0] + Rm[3 * q + 1] * w0[1] + Rm[3 * q + 2] * w0[2];
    double s[3] = {0, 0, 0};
    if (active) { s[0] = a.s[3 * k]; s[1] = a.s[3 * k + 1]; s[2] = a.s[3 * k + 2]; }
    double rel[3], r[3], v[3], wxr[3];
    for (int q = 0; q < 3; ++q) rel[q] = Rm[3 * q] * s[0] + Rm[3 * q + 1] * s[1] + Rm[3 * q + 2] * s[2];
    for (int q = 0; q < 3; ++q) r[q] = Xp[q] + rel[q];
    cross3(wl, rel, wxr);
    for (int q = 0; q < 3; ++q) v[q] = Vp[q] + wxr[q];

    const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    const int n3[3] = {g.nx, g.ny, g.nz};
    int xyz[3];
    double tw[3], wt = 1.0;
    for (int q = 0; q < 3; ++q) {
        const double tq = r[q] - 0.5, fl = floor(tq), fr = tq - fl;
        int b0 = (int)fl % n3[q];
        if (b0 < 0) b0 += n3[q];
        xyz[q] = o[q] ? (b0 + 1 == n3[q] ? 0 : b0 + 1) : b0;
        tw[q] = o[q] ? fr : 1.0 - fr;
        wt *= tw[q];
    }
    const long long n = nidx(g, xyz[0], xyz[1], xyz[2]);
    const bool fluid = active && !is_wall(g, xyz[0], xyz[1], xyz[2]);
    double uc[3] = {0, 0, 0}, rho = 1.0;
    if (fluid) {
        R rr, j[3];
        node_rho_j<R>(fn, g, xyz[0], xyz[1], xyz[2], n, a.odd, (R)a.rho0, rr, j);
        rho = (double)rr;
        for (int q = 0; q < 3; ++q)
            uc[q] = ((double)j[q] + 0.5 * (a.gforce[q] + (double)static_cast<const T *>(a.Fprev)[q * g.N + n])) / rho;
    }
    double ub[3], lsum[3] = {0, 0, 0};
    const T *lFn = static_cast<const T *>(a.lFn);
    double lFc[3] = {0, 0, 0};
    if (fluid)
        for (int q = 0; q < 3; ++q) lFc[q] = (double)lFn[q * g.N + n];
    for (int q = 0; q < 3; ++q) {
        ub[q] = fluid ? wt * uc[q] : 0.0;
        lsum[q] = fluid ? wt * lFc[q] : 0.0;
    }
    for (int off = 1; off < 8; off <<= 1)
        for (int q = 0; q < 3; ++q) {
            ub[q] += __shfl_xor_sync(0xffffffffu, ub[q], off, 8);
            lsum[q] += __shfl_xor_sync(0xffffffffu, lsum[q], off, 8);
        }
    // F_b = -gamma (v - u_b); lam F_b = lam F_tot - sum_c w_c lam F_node(c)
    const BodyAdj &BA = a.adj[body];
    double Fb[3], lFb[3], lv[3], lub[3], lg = 0.0;
    for (int q = 0; q < 3; ++q) {
        Fb[q] = -a.gamma * (v[q] - ub[q]);
        lFb[q] = BA.lFt[q] - lsum[q];
        lv[q] = -a.gamma * lFb[q];
        lub[q] = a.gamma * lFb[q];
        lg += -(v[q] - ub[q]) * lFb[q];
    }
    // this lane's node: interpolation and spread terms
    double lw = 0.0;
    if (fluid) {
        double luc[3];
        for (int q = 0; q < 3; ++q) {
            lw += -Fb[q] * lFc[q] + uc[q] * lub[q];
            luc[q] = wt * lub[q];
        }
        const double lrho = -(luc[0] * uc[0] + luc[1] * uc[1] + luc[2] * uc[2]) / rho;
        const double lj[3] = {luc[0] / rho, luc[1] / rho, luc[2] / rho};
        T *lf = static_cast<T *>(a.lam_f);
        T *lFp = static_cast<T *>(a.lFp);
        // the pre-collision population of the node, in natural layout
#pragma unroll
        for (int i = 0; i < 19; ++i)
            atomicAdd(&lf[i * g.N + n], (T)(lrho + cx(i) * lj[0] + cy(i) * lj[1] + cz(i) * lj[2]));
        for (int q = 0; q < 3; ++q) atomicAdd(&lFp[q * g.N + n], (T)(0.5 * luc[q] / rho));
    }
    // trilinear weight: d w / d r_q = (o_q ? 1 : -1) prod_{q' != q} tw_q'
    double lr[3];
    lr[0] = lw * (o[0] ? 1.0 : -1.0) * tw[1] * tw[2];
    lr[1] = lw * (o[1] ? 1.0 : -1.0) * tw[0] * tw[2];
    lr[2] = lw * (o[2] ? 1.0 : -1.0) * tw[0] * tw[1];
    if (!fluid) lr[0] = lr[1] = lr[2] = 0.0;
    for (int off = 1; off < 8; off <<= 1)
        for (int q = 0; q < 3; ++q) lr[q] += __shfl_xor_sync(0xffffffffu, lr[q], off, 8);
    if (active && c == 0) {
        atomicAdd(a.lgam, lg);
        double lrel[3], lxw[3];
        cross3(lv, wl, lxw);
        for (int q = 0; q < 3; ++q) lrel[q] = lr[q] + lxw[q];
        for (int q = 0; q < 3; ++q)
            a.dJds[3 * k + q] += Rm[q] * lrel[0] + Rm[3 + q] * lrel[1] + Rm[6 + q] * lrel[2];
        BodyAdj *BAw = a.adj + body;
        for (int q = 0; q < 3; ++q) {
            atomicAdd(&BAw->lXp[q], lr[q]);
            atomicAdd(&BAw->lVp[q], lv[q]);
        }
    }
}

// second half kick reversed (plus the objective's contribution)
__global__ void k_adj_body_pre(const Body *bodies, BodyAdj *adj, int nb, int jb, int axis, double jw) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const Body &B = bodies[b];
    BodyAdj &A = adj[b];
    if (b == jb) A.lV[axis] += jw;
    for (int q = 0; q < 3; ++q) {
        A.lXp[q] = A.lX[q];
        A.lFt[q] = A.lFl[q];
        A.lVp[q] = 0.0;
        if (B.fixed == 2) {
            A.lVp[q] = A.lV[q];
            A.lFt[q] += A.lV[q] / (2.0 * B.mass);
        }
    }
}

// kick and drift reversed
__global__ void k_adj_body_post(const Body *bodies, BodyAdj *adj, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const Body &B = bodies[b];
    BodyAdj &A = adj[b];
    for (int q = 0; q < 3; ++q) {
        if (B.fixed == 2) {
            const double lvt = A.lVp[q] + A.lXp[q];
            A.lX[q] = A.lXp[q];
            A.lV[q] = lvt;
            A.lFl[q] = lvt / (2.0 * B.mass);
        } else {
            A.lX[q] = A.lV[q] = A.lFl[q] = 0.0;
        }
    }
}

__global__ void k_record_v(const Body *bodies, int jb, int axis, double *out, int idx) {
    out[idx] = bodies[jb].V[axis];
}

}  // namespace
}  // namespace lbk

using lbk::BodyAdj;

namespace {

struct Snapshot {
    void *f = nullptr;
    void *F[2] = {nullptr, nullptr};
    int *tiles[2] = {nullptr, nullptr};
    int *tlist[2] = {nullptr, nullptr};   // list entries, then the count
    Body *bodies = nullptr;
    long long step = 0;
};

struct Tape {
    void *f = nullptr;        // populations before the step
    void *Fprev = nullptr;    // spread force the step reads
    void *Fnew = nullptr;     // spread force the step writes
    Body *bodies = nullptr;   // bodies before the step
    long long step = 0;
};

template <typename P>
cudaError_t amalloc(std::vector<void *> &pool, P **p, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)p, bytes < 16 ? 16 : bytes);
    if (e == cudaSuccess) pool.push_back((void *)*p);
    return e;
}

}  // namespace

extern "C" lb_status lb_adjoint_drag(lb_handle h, int nsteps, int window, int body, int axis, int checkpoints,
                                     double *J, double *dJ_dgamma, double *dJ_dbeads) {
    if (!h) return LB_ERR_ARG;
    if (nsteps < 1 || window < 1 || window > nsteps || axis < 0 || axis > 2 || !J || !dJ_dgamma)
        return lbk::ctx_fail(h, LB_ERR_ARG, "need nsteps >= window >= 1, axis 0-2, J and dJ_dgamma");
    if (h->p.kT > 0.0) return lbk::ctx_fail(h, LB_ERR_ARG, "the adjoint needs a deterministic fluid (kT = 0)");
    if (h->p.md_substeps > 1) return lbk::ctx_fail(h, LB_ERR_STATE, "the adjoint covers one MD step per LB step");
    if (h->g.chan || h->wall.on)
        return lbk::ctx_fail(h, LB_ERR_STATE, "the adjoint covers periodic boxes and pores, not moving or bead walls");
    const int nb = (int)h->hb.size(), nbeads = (int)h->hbody_of.size();
    if (body < 0 || body >= nb || nbeads == 0) return lbk::ctx_fail(h, LB_ERR_ARG, "bad body id");
    for (const Body &b : h->hb)
        if (b.fixed != 1 && b.fixed != 2)
            return lbk::ctx_fail(h, LB_ERR_ARG, "the adjoint needs fixed (1) or translation-only (2) bodies");
    lb_status st = lbk::ctx_upload(h);
    if (st == LB_OK) st = lbk::ctx_apply_external(h);
    if (st != LB_OK) return st;
    cudaStream_t s = h->stream;
    const long long N = h->g.N;
    const size_t es = h->fp32 ? 4 : 8;
    const size_t fbytes = es * 19 * (size_t)N, Fbytes = es * 3 * (size_t)N;
    const size_t tbytes = sizeof(int) * (size_t)h->ntx * h->nty * h->ntz, bbytes = sizeof(Body) * nb;
    const size_t lbytes = sizeof(int) * (size_t)h->list_cap;
    int c = checkpoints > 0 ? checkpoints : (int)std::ceil(std::sqrt((double)nsteps));
    if (c > nsteps) c = nsteps;
    const int K = (nsteps + c - 1) / c;
    const int nseg = (nsteps + K - 1) / K;

    std::vector<void *> pool;
    auto cleanup = [&]() { for (void *p : pool) cudaFree(p); };
#define ACUDA(call)                                                                             \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            cleanup();                                                                          \
            if (e_ == cudaErrorMemoryAllocation) { cudaGetLastError(); return lbk::ctx_fail(h, LB_ERR_OOM, "adjoint: device memory"); } \
            return lbk::ctx_fail(h, LB_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
        }                                                                                       \
    } while (0)

    std::vector<Snapshot> snaps(nseg + 1);   // +1: the final state
    for (auto &S : snaps) {
        ACUDA(amalloc(pool, &S.f, fbytes));
        for (int k = 0; k < 2; ++k) {
            ACUDA(amalloc(pool, &S.F[k], Fbytes));
            ACUDA(amalloc(pool, &S.tiles[k], tbytes));
            ACUDA(amalloc(pool, &S.tlist[k], lbytes + sizeof(int)));
        }
        ACUDA(amalloc(pool, &S.bodies, bbytes));
    }
    std::vector<Tape> tape(K);
    for (auto &T : tape) {
        ACUDA(amalloc(pool, &T.f, fbytes));
        ACUDA(amalloc(pool, &T.Fprev, Fbytes));
        ACUDA(amalloc(pool, &T.Fnew, Fbytes));
        ACUDA(amalloc(pool, &T.bodies, bbytes));
    }
    void *lam[2], *lFp[2], *lFn;
    for (int k = 0; k < 2; ++k) {
        ACUDA(amalloc(pool, &lam[k], fbytes));
        ACUDA(amalloc(pool, &lFp[k], es * 3 * (size_t)N));
    }
    ACUDA(amalloc(pool, &lFn, es * 3 * (size_t)N));
    BodyAdj *adj;
    double *dJds, *lgam, *vhist;
    ACUDA(amalloc(pool, &adj, sizeof(BodyAdj) * nb));
    ACUDA(amalloc(pool, &dJds, sizeof(double) * 3 * nbeads));
    ACUDA(amalloc(pool, &lgam, sizeof(double)));
    ACUDA(amalloc(pool, &vhist, sizeof(double) * nsteps));

    auto save = [&](Snapshot &S) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(S.f, h->f, fbytes, cudaMemcpyDeviceToDevice, s);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaMemcpyAsync(S.F[k], h->Fbuf[k], Fbytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(S.tiles[k], h->tiles[k], tbytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(S.tlist[k], h->tlist[k], lbytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((char *)S.tlist[k] + lbytes, h->tcount[k], sizeof(int), cudaMemcpyDeviceToDevice, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(S.bodies, h->db, bbytes, cudaMemcpyDeviceToDevice, s);
        S.step = h->step;
        return e;
    };
    auto restore = [&](const Snapshot &S) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(h->f, S.f, fbytes, cudaMemcpyDeviceToDevice, s);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaMemcpyAsync(h->Fbuf[k], S.F[k], Fbytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->tiles[k], S.tiles[k], tbytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->tlist[k], S.tlist[k], lbytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->tcount[k], (char *)S.tlist[k] + lbytes, sizeof(int), cudaMemcpyDeviceToDevice, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->db, S.bodies, bbytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) {
            h->step = S.step;
            static thread_local unsigned long long sv;
            sv = (unsigned long long)S.step;
            e = cudaMemcpyAsync(h->step_dev, &sv, sizeof(sv), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        return e;
    };

    // ---------------------------------------------------------------- forward
    const long long n0 = h->step;
    for (int sg = 0; sg < nseg; ++sg) {
        ACUDA(save(snaps[sg]));
        const int a0 = sg * K, a1 = std::min(nsteps, a0 + K);
        for (int n = a0; n < a1; ++n) {
            if ((st = lb_step(h, 1)) != LB_OK) { cleanup(); return st; }
            lbk::k_record_v<<<1, 1, 0, s>>>(h->db, body, axis, vhist, n);
            ACUDA(cudaGetLastError());
        }
    }
    ACUDA(save(snaps[nseg]));
    std::vector<double> vh(nsteps);
    ACUDA(cudaMemcpyAsync(vh.data(), vhist, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, s));
    ACUDA(cudaStreamSynchronize(s));
    double Jv = 0.0;
    for (int n = nsteps - window; n < nsteps; ++n) Jv += vh[n];
    *J = Jv / window;

    // ---------------------------------------------------------------- reverse
    lbk::AdjArgs aa{};
    aa.g = h->g;
    aa.gforce = h->gforce;
    {
        static const int modes[6] = {4, 5, 6, 7, 8, 9};
        auto rate = [&](int k) {
            if (h->p.collision == 0) return 1.0 - 1.0 / h->p.tau;   // BGK = MRT with equal rates
            return k == 4 ? h->p.gamma_bulk : (k <= 9 ? h->p.gamma_shear : (k <= 15 ? h->p.gamma_odd : h->p.gamma_even));
        };
        aa.pd.rho0 = h->p.rho0;
        for (int q = 0; q < 6; ++q) {
            aa.pd.A[q] = 1.0 - rate(modes[q]);
            aa.pd.H[q] = 0.5 * (1.0 + rate(modes[q]));
        }
        for (int k = 4; k <= 18; ++k) aa.pd.G[k - 4] = rate(k);
        aa.pf.rho0 = (float)aa.pd.rho0;
        for (int q = 0; q < 6; ++q) { aa.pf.A[q] = (float)aa.pd.A[q]; aa.pf.H[q] = (float)aa.pd.H[q]; }
        for (int q = 0; q < 15; ++q) aa.pf.G[q] = (float)aa.pd.G[q];
    }
    const long long nl = 19 * N, n3 = 3 * N;
    auto zero = [&](void *p, long long n) {
        if (h->fp32) lbk::k_zero<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((float *)p, n);
        else lbk::k_zero<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double *)p, n);
    };
    zero(lam[0], nl);
    zero(lFp[0], n3);
    ACUDA(cudaMemsetAsync(adj, 0, sizeof(BodyAdj) * nb, s));
    ACUDA(cudaMemsetAsync(dJds, 0, sizeof(double) * 3 * nbeads, s));
    ACUDA(cudaMemsetAsync(lgam, 0, sizeof(double), s));
    int cur = 0;
    const dim3 block = h->block;
    const dim3 grid((h->g.nx + block.x - 1) / block.x, (h->g.ny + block.y - 1) / block.y, h->g.nz);
    for (int sg = nseg - 1; sg >= 0; --sg) {
        ACUDA(restore(snaps[sg]));
        const int a0 = sg * K, a1 = std::min(nsteps, a0 + K);
        for (int n = a0; n < a1; ++n) {
            Tape &T = tape[n - a0];
            const int prev = (int)(((n0 + n) & 1) ^ 1), curb = (int)((n0 + n) & 1);
            ACUDA(cudaMemcpyAsync(T.f, h->f, fbytes, cudaMemcpyDeviceToDevice, s));
            ACUDA(cudaMemcpyAsync(T.Fprev, h->Fbuf[prev], Fbytes, cudaMemcpyDeviceToDevice, s));
            ACUDA(cudaMemcpyAsync(T.bodies, h->db, bbytes, cudaMemcpyDeviceToDevice, s));
            T.step = h->step;
            if ((st = lb_step(h, 1)) != LB_OK) { cleanup(); return st; }
            ACUDA(cudaMemcpyAsync(T.Fnew, h->Fbuf[curb], Fbytes, cudaMemcpyDeviceToDevice, s));
        }
        for (int n = a1 - 1; n >= a0; --n) {
            const Tape &T = tape[n - a0];
            const double jw = n >= nsteps - window ? 1.0 / window : 0.0;
            lbk::k_adj_body_pre<<<(nb + 63) / 64, 64, 0, s>>>(T.bodies, adj, nb, jw != 0.0 ? body : -1, axis, jw);
            ACUDA(cudaGetLastError());
            aa.fn = T.f;
            aa.odd = (T.step & 1) != 0;
            aa.Fprev = T.Fprev;
            aa.Fnew = T.Fnew;
            aa.lam_in = lam[cur];
            aa.lam_out = lam[cur ^ 1];
            aa.lFp_in = lFp[cur];
            aa.lFn = lFn;
            aa.lFp_out = lFp[cur ^ 1];
            if (h->fp32) lbk::k_adj_collide<float><<<grid, block, 0, s>>>(aa);
            else lbk::k_adj_collide<double><<<grid, block, 0, s>>>(aa);
            ACUDA(cudaGetLastError());
            zero(lFp[cur ^ 1], n3);
            lbk::AdjCouple ac{};
            ac.g = h->g;
            ac.fn = T.f;
            ac.odd = aa.odd;
            ac.rho0 = h->p.rho0;
            ac.gamma = h->p.gamma_bead;
            ac.gforce = h->gforce;
            ac.Fprev = T.Fprev;
            ac.lFn = lFn;
            ac.lam_f = lam[cur ^ 1];
            ac.lFp = lFp[cur ^ 1];
            ac.s = h->ds;
            ac.bead_body = h->dbody_of;
            ac.bodies = T.bodies;
            ac.adj = adj;
            ac.dJds = dJds;
            ac.lgam = lgam;
            ac.nbeads = nbeads;
            const unsigned cg = (unsigned)((8LL * nbeads + 127) / 128);
            if (h->fp32) lbk::k_adj_couple<float><<<cg, 128, 0, s>>>(ac);
            else lbk::k_adj_couple<double><<<cg, 128, 0, s>>>(ac);
            ACUDA(cudaGetLastError());
            lbk::k_adj_body_post<<<(nb + 63) / 64, 64, 0, s>>>(T.bodies, adj, nb);
            ACUDA(cudaGetLastError());
            cur ^= 1;
        }
    }
    ACUDA(cudaMemcpyAsync(dJ_dgamma, lgam, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dJ_dbeads) ACUDA(cudaMemcpyAsync(dJ_dbeads, dJds, sizeof(double) * 3 * nbeads, cudaMemcpyDeviceToHost, s));
    // leave the handle where the forward sweep ended
    ACUDA(restore(snaps[nseg]));
    ACUDA(cudaStreamSynchronize(s));
    cleanup();
#undef ACUDA
    return LB_OK;
}
