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
#include <chrono>
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
    // the step's kinematics as the FP32 coupling forms them (set by the body
    // kernel that opens each reversed step): rotation, velocity and lab omega
    // after the kick and drift, X - 1/2 split into floor and fraction
    float Rf[9], Vf[3], wlf[3], Xf[3];
    int Xi[3];
};

struct AdjArgs {
    Geom g;
    const void *fn;             // taped population buffer before step n (AA layout)
    bool odd;                   // parity of n
    const void *Fprev;          // taped spread force read by step n ([3][N], storage precision)
    const void *Fnew;           // taped spread force written by step n
    const double *gforce;       // uniform force density (3)
    const float *gforce_f;      // the same in FP32 (FP32 storage)
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
    // the adjoint of F_prev of this step starts at zero (the coupling's
    // reverse adds into it after this kernel)
    T *lFpo = static_cast<T *>(a.lFp_out);
    lFpo[n] = T(0);
    lFpo[N + n] = T(0);
    lFpo[2 * N + n] = T(0);
    if (is_wall(g, x, y, z)) {
#pragma unroll
        for (int i = 0; i < 19; ++i) lout[i * N + n] = T(0);
        for (int c = 0; c < 3; ++c) lFn[c * N + n] = T(0);
        return;
    }
    R lam[19], f[19];
    const T *fn = static_cast<const T *>(a.fn);
    if (g.pore_axis < 0 && !g.chan) {
        // periodic box: neighbours from per-axis wrapped offsets, no wall tests
        const int nx = g.nx, nxy = g.nx * g.ny;
        const int xo[3] = {(x == 0 ? nx : x) - 1, x, x + 1 == nx ? 0 : x + 1};
        const int yo[3] = {((y == 0 ? g.ny : y) - 1) * nx, y * nx, (y + 1 == g.ny ? 0 : y + 1) * nx};
        const int zo[3] = {((z == 0 ? g.nz : z) - 1) * nxy, z * nxy, (z + 1 == g.nz ? 0 : z + 1) * nxy};
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const long long dn = xo[1 + cx(i)] + yo[1 + cy(i)] + zo[1 + cz(i)];   // downstream x + c_i
            lam[i] = lin[i * N + dn];
            if (!a.odd || i == 0) f[i] = fn[i * N + n];
            else f[i] = fn[opp(i) * N + (long long)(xo[1 - cx(i)] + yo[1 - cy(i)] + zo[1 - cz(i)])];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int xd = wrapm(x + cx(i), g.nx), yd = wrapm(y + cy(i), g.ny), zd = wrapm(z + cz(i), g.nz);
            lam[i] = is_wall(g, xd, yd, zd) ? lin[opp(i) * N + n] : lin[i * N + nidx(g, xd, yd, zd)];
            f[i] = (R)load_pre(fn, g, x, y, z, n, i, a.odd);
        }
    }
    const T *Fnew = static_cast<const T *>(a.Fnew);
    R Fx, Fy, Fz;
    if constexpr (DEV) {          // as the FP32 forward collision forms it
        Fx = a.gforce_f[0] + Fnew[n];
        Fy = a.gforce_f[1] + Fnew[N + n];
        Fz = a.gforce_f[2] + Fnew[2 * N + n];
    } else {
        Fx = (R)(a.gforce[0] + (double)Fnew[n]);
        Fy = (R)(a.gforce[1] + (double)Fnew[N + n]);
        Fz = (R)(a.gforce[2] + (double)Fnew[2 * N + n]);
    }
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

// Eight lanes per bead, as the forward coupling. The per-lane arithmetic is
// in Q, the storage precision: FP32 storage works in FP32 as the forward
// FP32 coupling does (GB300's FP64 pipe is narrow, and in FP64 this kernel
// is bound by it), with the bead position split into the FP64 floor of
// X - 1/2 and a small FP32 remainder so that it keeps its resolution in any
// box; the body-level sums (dJ/dgamma, dJ/ds, the body adjoints) are
// accumulated in FP64.
template <typename T>
__global__ void __launch_bounds__(128) k_adj_couple(const AdjCouple a) {
    using R = T;
    using Q = T;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t >> 3, c = t & 7;
    const bool active = k < a.nbeads;
    const Geom &g = a.g;
    const T *fn = static_cast<const T *>(a.fn);
    const int body = active ? a.bead_body[k] : 0;
    // kinematics of the step (translation-only or fixed bodies): FP64 storage
    // forms them here in FP64 as the FP64 coupling does; FP32 storage reads
    // them as the body kernel prepared them for this step (k_adj_body_pre)
    Q Rm[9], Vp[3], wl[3];
    double Xp[3] = {0, 0, 0};
    const BodyAdj &BK = a.adj[body];
    if constexpr (sizeof(T) == 8) {
        const Body &B = a.bodies[body];
        for (int q = 0; q < 3; ++q) {
            double vq = B.V[q], xq = B.X[q];
            if (B.fixed == 2) {
                vq += 0.5 * B.F_last[q] / B.mass;
                xq += vq;
            }
            Vp[q] = vq;
            Xp[q] = xq;
        }
        quat_to_R(B.q, Rm);
        const double w0[3] = {B.fixed == 2 ? 0.0 : B.w[0], B.fixed == 2 ? 0.0 : B.w[1], B.fixed == 2 ? 0.0 : B.w[2]};
        for (int q = 0; q < 3; ++q) wl[q] = Rm[3 * q] * w0[0] + Rm[3 * q + 1] * w0[1] + Rm[3 * q + 2] * w0[2];
    } else {
        for (int q = 0; q < 9; ++q) Rm[q] = BK.Rf[q];
        for (int q = 0; q < 3; ++q) {
            Vp[q] = BK.Vf[q];
            wl[q] = BK.wlf[q];
        }
    }
    Q s[3] = {Q(0), Q(0), Q(0)};
    if (active) { s[0] = (Q)a.s[3 * k]; s[1] = (Q)a.s[3 * k + 1]; s[2] = (Q)a.s[3 * k + 2]; }
    Q rel[3], v[3], wxr[3];
    for (int q = 0; q < 3; ++q) rel[q] = Rm[3 * q] * s[0] + Rm[3 * q + 1] * s[1] + Rm[3 * q + 2] * s[2];
    wxr[0] = wl[1] * rel[2] - wl[2] * rel[1];
    wxr[1] = wl[2] * rel[0] - wl[0] * rel[2];
    wxr[2] = wl[0] * rel[1] - wl[1] * rel[0];
    for (int q = 0; q < 3; ++q) v[q] = Vp[q] + wxr[q];

    const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    const int n3[3] = {g.nx, g.ny, g.nz};
    int xyz[3];
    Q tw[3], wt = Q(1);
    for (int q = 0; q < 3; ++q) {
        // the cell and fraction exactly as the forward coupling of this
        // precision forms them (they decide the side of a cell face a bead on
        // it takes, where the trilinear weights have a kink)
        int raw;
        Q fr;
        if constexpr (sizeof(T) == 8) {
            const double tq = (Xp[q] + rel[q]) - 0.5;
            const double fl = floor(tq);
            raw = (int)fl;
            fr = tq - fl;
        } else {
            const Q tq = BK.Xf[q] + rel[q];              // r - 1/2 - floor(X - 1/2)
            const Q fl = floor(tq);
            raw = BK.Xi[q] + (int)fl;
            fr = tq - fl;
        }
        int b0 = raw % n3[q];
        if (b0 < 0) b0 += n3[q];
        xyz[q] = o[q] ? (b0 + 1 == n3[q] ? 0 : b0 + 1) : b0;
        tw[q] = o[q] ? fr : Q(1) - fr;
        wt *= tw[q];
    }
    const long long n = nidx(g, xyz[0], xyz[1], xyz[2]);
    const bool fluid = active && !is_wall(g, xyz[0], xyz[1], xyz[2]);
    Q uc[3] = {Q(0), Q(0), Q(0)}, rho = Q(1);
    if (fluid) {
        R rr, j[3];
        node_rho_j<R>(fn, g, xyz[0], xyz[1], xyz[2], n, a.odd, (R)a.rho0, rr, j);
        rho = (Q)rr;
        const T *Fp = static_cast<const T *>(a.Fprev);
        for (int q = 0; q < 3; ++q) uc[q] = ((Q)j[q] + Q(0.5) * ((Q)a.gforce[q] + (Q)Fp[q * g.N + n])) / rho;
    }
    Q ub[3], lsum[3];
    const T *lFn = static_cast<const T *>(a.lFn);
    Q lFc[3] = {Q(0), Q(0), Q(0)};
    if (fluid)
        for (int q = 0; q < 3; ++q) lFc[q] = (Q)lFn[q * g.N + n];
    for (int q = 0; q < 3; ++q) {
        ub[q] = fluid ? wt * uc[q] : Q(0);
        lsum[q] = fluid ? wt * lFc[q] : Q(0);
    }
    for (int off = 1; off < 8; off <<= 1)
        for (int q = 0; q < 3; ++q) {
            ub[q] += __shfl_xor_sync(0xffffffffu, ub[q], off, 8);
            lsum[q] += __shfl_xor_sync(0xffffffffu, lsum[q], off, 8);
        }
    // F_b = -gamma (v - u_b); lam F_b = lam F_tot - sum_c w_c lam F_node(c)
    const BodyAdj &BA = a.adj[body];
    const Q gam = (Q)a.gamma;
    Q Fb[3], lFb[3], lv[3], lub[3], lg = Q(0);
    for (int q = 0; q < 3; ++q) {
        Fb[q] = -gam * (v[q] - ub[q]);
        lFb[q] = (Q)BA.lFt[q] - lsum[q];
        lv[q] = -gam * lFb[q];
        lub[q] = gam * lFb[q];
        lg += -(v[q] - ub[q]) * lFb[q];
    }
    // this lane's node: interpolation and spread terms
    Q lw = Q(0);
    if (fluid) {
        Q luc[3];
        for (int q = 0; q < 3; ++q) {
            lw += -Fb[q] * lFc[q] + uc[q] * lub[q];
            luc[q] = wt * lub[q];
        }
        const Q ir = Q(1) / rho;
        const Q lrho = -(luc[0] * uc[0] + luc[1] * uc[1] + luc[2] * uc[2]) * ir;
        const Q lj[3] = {luc[0] * ir, luc[1] * ir, luc[2] * ir};
        T *lf = static_cast<T *>(a.lam_f);
        T *lFp = static_cast<T *>(a.lFp);
        // the pre-collision population of the node, in natural layout
#pragma unroll
        for (int i = 0; i < 19; ++i)
            atomicAdd(&lf[i * g.N + n], (T)(lrho + cx(i) * lj[0] + cy(i) * lj[1] + cz(i) * lj[2]));
        for (int q = 0; q < 3; ++q) atomicAdd(&lFp[q * g.N + n], (T)(Q(0.5) * luc[q] * ir));
    }
    // trilinear weight: d w / d r_q = (o_q ? 1 : -1) prod_{q' != q} tw_q'
    Q lr[3];
    lr[0] = lw * (o[0] ? Q(1) : Q(-1)) * tw[1] * tw[2];
    lr[1] = lw * (o[1] ? Q(1) : Q(-1)) * tw[0] * tw[2];
    lr[2] = lw * (o[2] ? Q(1) : Q(-1)) * tw[0] * tw[1];
    if (!fluid) lr[0] = lr[1] = lr[2] = Q(0);
    for (int off = 1; off < 8; off <<= 1)
        for (int q = 0; q < 3; ++q) lr[q] += __shfl_xor_sync(0xffffffffu, lr[q], off, 8);
    if (active && c == 0) {
        atomicAdd(a.lgam, (double)lg);
        double lrel[3];
        lrel[0] = (double)lr[0] + (double)(lv[1] * wl[2] - lv[2] * wl[1]);
        lrel[1] = (double)lr[1] + (double)(lv[2] * wl[0] - lv[0] * wl[2]);
        lrel[2] = (double)lr[2] + (double)(lv[0] * wl[1] - lv[1] * wl[0]);
        for (int q = 0; q < 3; ++q)
            a.dJds[3 * k + q] += (double)Rm[q] * lrel[0] + (double)Rm[3 + q] * lrel[1] + (double)Rm[6 + q] * lrel[2];
        BodyAdj *BAw = a.adj + body;
        for (int q = 0; q < 3; ++q) {
            atomicAdd(&BAw->lXp[q], (double)lr[q]);
            atomicAdd(&BAw->lVp[q], (double)lv[q]);
        }
    }
}

// second half kick reversed (plus the objective's contribution)
__global__ void k_adj_body_pre(const Body *bodies, BodyAdj *adj, int nb, int jb, int axis, double jw) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const Body &B = bodies[b];
    BodyAdj &A = adj[b];
    // kick and drift of the step, then its kinematics in FP32 as the body
    // prologue hands them to the FP32 coupling
    double Rd[9];
    quat_to_R(B.q, Rd);
    const double w0[3] = {B.fixed == 2 ? 0.0 : B.w[0], B.fixed == 2 ? 0.0 : B.w[1], B.fixed == 2 ? 0.0 : B.w[2]};
    for (int q = 0; q < 9; ++q) A.Rf[q] = (float)Rd[q];
    for (int q = 0; q < 3; ++q) {
        double vq = B.V[q], xq = B.X[q];
        if (B.fixed == 2) {
            vq += 0.5 * B.F_last[q] / B.mass;
            xq += vq;
        }
        A.Vf[q] = (float)vq;
        A.wlf[q] = (float)(Rd[3 * q] * w0[0] + Rd[3 * q + 1] * w0[1] + Rd[3 * q + 2] * w0[2]);
        const double h = xq - 0.5, fl = floor(h);
        A.Xi[q] = (int)fl;
        A.Xf[q] = (float)(h - fl);
    }
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

// Several device-to-device copies in one launch (a state save or restore):
// segment k copies bytes (a multiple of 4) from src to dst, in 16-byte words
// when both addresses allow it, else in 4-byte words.
struct CopySeg {
    const void *src;
    void *dst;
    unsigned long long bytes;
};
struct CopyList {
    CopySeg seg[12];
    int n;
};

__global__ void k_copy_segments(const CopyList L) {
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nt = (unsigned long long)gridDim.x * blockDim.x;
    for (int k = 0; k < L.n; ++k) {
        const CopySeg c = L.seg[k];
        unsigned long long n16 = 0;
        if ((((uintptr_t)c.src | (uintptr_t)c.dst) & 15u) == 0) {
            n16 = c.bytes / 16;
            const uint4 *s4 = static_cast<const uint4 *>(c.src);
            uint4 *d4 = static_cast<uint4 *>(c.dst);
            for (unsigned long long i = tid; i < n16; i += nt) d4[i] = s4[i];
        }
        const unsigned long long w0 = 4 * n16, nw = c.bytes / 4;   // 4-byte words left: [w0, nw)
        const uint32_t *s1 = static_cast<const uint32_t *>(c.src);
        uint32_t *d1 = static_cast<uint32_t *>(c.dst);
        for (unsigned long long i = w0 + tid; i < nw; i += nt) d1[i] = s1[i];
    }
}

}  // namespace
}  // namespace lbk

using lbk::BodyAdj;

namespace {

// A whole lattice state between steps: populations, both spread-force
// buffers with their tile flags and lists, the bodies and the step count
// (host and device copies, so a restore needs no host synchronisation).
struct Snapshot {
    void *f = nullptr;
    void *F[2] = {nullptr, nullptr};
    int *tiles[2] = {nullptr, nullptr};
    int *tlist[2] = {nullptr, nullptr};   // list entries, then the count
    Body *bodies = nullptr;
    unsigned long long *dstep = nullptr;
    long long step = 0;
};

// What the reverse pass of one step reads, taped by the two-level schedule.
// Entry 0 receives the segment's snapshot populations; every step reads its
// entry and writes the next one's populations itself. The first step's
// previous spread force is the snapshot's, every later one's the Fnew of the
// entry before.
struct Tape {
    void *f = nullptr;        // populations before the step
    void *Fnew = nullptr;     // spread force the step writes
    Body *bodies = nullptr;   // bodies before the step
};

}  // namespace

struct AdjWork {
    long long N = 0;
    bool fp32 = false;
    int nb = 0, nbeads = 0, list_cap = 0;
    std::vector<Snapshot> snaps;
    std::vector<Tape> tape;
    void *lam[2] = {nullptr, nullptr}, *lFp[2] = {nullptr, nullptr}, *lFn = nullptr;
    BodyAdj *adj = nullptr;
    double *dJds = nullptr, *lgam = nullptr, *vhist = nullptr;
    int vcap = 0;
    Body *turn_bodies = nullptr;
    std::vector<void *> pool;
    size_t bytes = 0;
};

namespace lbk {
void adj_free(lb_ctx *h) {
    if (!h || !h->adjw) return;
    for (void *p : h->adjw->pool) cudaFree(p);
    delete h->adjw;
    h->adjw = nullptr;
}
}  // namespace lbk

namespace {

struct Sizes {
    size_t fbytes, Fbytes, tbytes, lbytes, bbytes;
};

Sizes sizes_of(const lb_ctx *h) {
    const size_t es = h->fp32 ? 4 : 8;
    const size_t N = (size_t)h->g.N;
    return Sizes{es * 19 * N, es * 3 * N, sizeof(int) * (size_t)h->ntx * h->nty * h->ntz,
                 sizeof(int) * (size_t)h->list_cap, sizeof(Body) * h->hb.size()};
}

size_t snapshot_bytes(const Sizes &z) {
    return z.fbytes + 2 * (z.Fbytes + z.tbytes + z.lbytes + sizeof(int)) + z.bbytes + sizeof(unsigned long long);
}

size_t tape_bytes(const Sizes &z) { return z.fbytes + z.Fbytes + z.bbytes; }

template <typename P>
cudaError_t walloc(AdjWork &w, P **p, size_t bytes) {
    bytes = bytes < 16 ? 16 : bytes;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) {
        w.pool.push_back((void *)*p);
        w.bytes += bytes;
    }
    return e;
}

// The handle's workspace with at least nsnap snapshots, ntape tapes and a
// velocity history of nsteps; a previous call's is reused when it is large
// enough for this handle. *alloc_ms: host time spent allocating (0 if reused).
lb_status ensure_work(lb_ctx *h, int nsnap, int ntape, int nsteps, double *alloc_ms) {
    *alloc_ms = 0.0;
    AdjWork *w = h->adjw;
    const int nb = (int)h->hb.size(), nbeads = (int)h->hbody_of.size();
    if (w && w->N == h->g.N && w->fp32 == h->fp32 && w->nb == nb && w->nbeads == nbeads &&
        w->list_cap == h->list_cap && (int)w->snaps.size() >= nsnap && (int)w->tape.size() >= ntape &&
        w->vcap >= nsteps)
        return LB_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const int keep_snaps = w ? std::max(nsnap, (int)w->snaps.size()) : nsnap;
    const int keep_tapes = w ? std::max(ntape, (int)w->tape.size()) : ntape;
    const bool same = w && w->N == h->g.N && w->fp32 == h->fp32 && w->nb == nb && w->nbeads == nbeads &&
                      w->list_cap == h->list_cap;
    lbk::adj_free(h);
    const Sizes z = sizes_of(h);
    const int ns = same ? keep_snaps : nsnap, nt = same ? keep_tapes : ntape;
    size_t need = (size_t)ns * snapshot_bytes(z) + (size_t)nt * tape_bytes(z) + 2 * z.fbytes + 3 * z.Fbytes;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && need + (64u << 20) > free_b)
        return lbk::ctx_fail(h, LB_ERR_OOM, "adjoint: the workspace (" + std::to_string(need >> 20) +
                                                " MiB) does not fit in free device memory");
    w = new AdjWork();
    h->adjw = w;
    w->N = h->g.N;
    w->fp32 = h->fp32;
    w->nb = nb;
    w->nbeads = nbeads;
    w->list_cap = h->list_cap;
    w->snaps.resize(ns);
    w->tape.resize(nt);
    cudaError_t e = cudaSuccess;
    for (auto &S : w->snaps) {
        if (e == cudaSuccess) e = walloc(*w, &S.f, z.fbytes);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = walloc(*w, &S.F[k], z.Fbytes);
            if (e == cudaSuccess) e = walloc(*w, &S.tiles[k], z.tbytes);
            if (e == cudaSuccess) e = walloc(*w, &S.tlist[k], z.lbytes + sizeof(int));
        }
        if (e == cudaSuccess) e = walloc(*w, &S.bodies, z.bbytes);
        if (e == cudaSuccess) e = walloc(*w, &S.dstep, sizeof(unsigned long long));
    }
    for (size_t k = 0; k < w->tape.size(); ++k) {
        Tape &T = w->tape[k];
        if (e == cudaSuccess) {
            // out-of-place steps write the slots of fluid nodes only: the
            // wall-node slots (never read) start as zeros, not garbage
            e = walloc(*w, &T.f, z.fbytes);
            if (e == cudaSuccess) e = cudaMemsetAsync(T.f, 0, z.fbytes, h->stream);
        }
        if (e == cudaSuccess) e = walloc(*w, &T.Fnew, z.Fbytes);
        if (e == cudaSuccess) e = walloc(*w, &T.bodies, z.bbytes);
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = walloc(*w, &w->lam[k], z.fbytes);
        if (e == cudaSuccess) e = walloc(*w, &w->lFp[k], z.Fbytes);
    }
    if (e == cudaSuccess) e = walloc(*w, &w->lFn, z.Fbytes);
    if (e == cudaSuccess) e = walloc(*w, &w->adj, sizeof(BodyAdj) * (nb > 0 ? nb : 1));
    if (e == cudaSuccess) e = walloc(*w, &w->dJds, sizeof(double) * 3 * (nbeads > 0 ? nbeads : 1));
    if (e == cudaSuccess) e = walloc(*w, &w->lgam, sizeof(double));
    w->vcap = std::max(nsteps, 1);
    if (e == cudaSuccess) e = walloc(*w, &w->vhist, sizeof(double) * w->vcap);
    if (e == cudaSuccess) e = walloc(*w, &w->turn_bodies, z.bbytes);
    if (e != cudaSuccess) {
        lbk::adj_free(h);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return lbk::ctx_fail(h, LB_ERR_OOM, "adjoint: device memory");
        }
        return lbk::ctx_fail(h, LB_ERR_CUDA, std::string("adjoint workspace: ") + cudaGetErrorString(e));
    }
    *alloc_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return LB_OK;
}

// One adjoint run: the schedules share the state moves, the reverse step
// and the objective's velocity history.
struct Run {
    lb_ctx *h;
    AdjWork *w;
    Sizes z;
    cudaStream_t s;
    int nsteps, window, body, axis;
    long long n0;               // step count of the start state
    lbk::AdjArgs aa{};
    int cur = 0;                // lam[cur] holds the adjoint of the state after the step reversed next
    dim3 grid, block;
    // timing
    bool timed = false;
    std::vector<cudaEvent_t> ev;    // pairs around each reversed step's kernels
    size_t ev_used = 0;
    long long recompute_steps = 0, reversed = 0;
    bool first_sweep = true;
    long long forward_steps = 0;
    cudaEvent_t ev_start = nullptr, ev_first = nullptr, ev_end = nullptr;

    lb_status fail_cuda(cudaError_t e, const char *what) {
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return lbk::ctx_fail(h, LB_ERR_OOM, "adjoint: device memory");
        }
        return lbk::ctx_fail(h, LB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }

    // Where the current state's populations are: the handle's array (null),
    // or a snapshot's or tape entry's, which the next step or turn reads in
    // place (an out-of-place step leaves its result in the handle's array).
    const void *cf = nullptr;
    const void *pops() const { return cf ? cf : h->f; }

    // The state's parts as copy segments between a snapshot and the handle
    // (to_snapshot: handle -> snapshot); the populations when with_f.
    lbk::CopyList parts(const Snapshot &S, bool to_snapshot, bool with_f, const void *f_src) {
        lbk::CopyList L{};
        auto add = [&](void *snap, const void *hnd, size_t bytes) {
            lbk::CopySeg &c = L.seg[L.n++];
            c.src = to_snapshot ? hnd : snap;
            c.dst = to_snapshot ? snap : const_cast<void *>(hnd);
            c.bytes = bytes;
        };
        if (with_f) {
            if (to_snapshot) add(S.f, f_src, z.fbytes);
            else add(S.f, h->f, z.fbytes);
        }
        for (int k = 0; k < 2; ++k) {
            add(S.F[k], h->Fbuf[k], z.Fbytes);
            add(S.tiles[k], h->tiles[k], z.tbytes);
            add(S.tlist[k], h->tlist[k], z.lbytes);
            add((char *)S.tlist[k] + z.lbytes, h->tcount[k], sizeof(int));
        }
        add(S.bodies, h->db, z.bbytes);
        add(S.dstep, h->step_dev, sizeof(unsigned long long));
        return L;
    }
    cudaError_t copy(const lbk::CopyList &L) {
        unsigned long long words = 0;
        for (int k = 0; k < L.n; ++k) words += (L.seg[k].bytes + 15) / 16;
        const unsigned long long want = (words + 255) / 256;
        const unsigned grid = (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>(want, 4096));
        lbk::k_copy_segments<<<grid, 256, 0, s>>>(L);
        return cudaGetLastError();
    }

    // One launch for the whole state (the populations only if they are not
    // already the snapshot's).
    cudaError_t save(Snapshot &S) {
        S.step = h->step;
        return copy(parts(S, true, pops() != S.f, pops()));
    }
    // Everything but the populations, which stay in the snapshot for the next
    // step or turn to read; whole: the populations too (the handle is left
    // holding the state).
    cudaError_t restore(const Snapshot &S, bool whole = false) {
        cf = whole ? nullptr : S.f;
        h->step = S.step;
        return copy(parts(S, false, whole, nullptr));
    }

    // Steps the handle from relative step a to b (its state is a), recording
    // the pulled body's velocity after each step of the objective's window.
    lb_status advance(int a, int b) {
        if (b <= a) return LB_OK;
        if (!first_sweep) recompute_steps += b - a;
        else forward_steps += b - a;
        const int wstart = nsteps - window;
        auto record = [&](int n) -> lb_status {
            lbk::k_record_v<<<1, 1, 0, s>>>(h->db, body, axis, w->vhist, n);
            cudaError_t e = cudaGetLastError();
            return e == cudaSuccess ? LB_OK : fail_cuda(e, "record launch");
        };
        lb_status st;
        int n0s = a;
        if (cf) {                       // the first step reads the snapshot's populations
            if ((st = lbk::ctx_step_oop(h, cf, h->f)) != LB_OK) return st;
            cf = nullptr;
            if (a >= wstart && (st = record(a)) != LB_OK) return st;
            ++n0s;
        }
        const int n1 = std::max(n0s, std::min(b, wstart));
        if (n1 > n0s && (st = lb_step(h, n1 - n0s)) != LB_OK) return st;
        for (int n = n1; n < b; ++n) {
            if ((st = lb_step(h, 1)) != LB_OK) return st;
            if ((st = record(n)) != LB_OK) return st;
        }
        return LB_OK;
    }

    cudaError_t zero(void *p, long long n) {
        if (h->fp32) lbk::k_zero<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((float *)p, n);
        else lbk::k_zero<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double *)p, n);
        return cudaGetLastError();
    }

    void mark_first() {
        if (first_sweep && timed) cudaEventRecord(ev_first, s);
        first_sweep = false;
    }

    // The reverse pass of relative step n from what it reads: the populations
    // before it (AA layout of its parity), the spread force it reads and the
    // one it writes, and the bodies before it.
    lb_status reverse_step(int n, const void *fn, const void *Fprev, const void *Fnew, const Body *bodies) {
        const int nb = (int)h->hb.size(), nbeads = (int)h->hbody_of.size();
        if (timed) {
            if (ev_used + 2 > ev.size()) {
                cudaEvent_t e0, e1;
                if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
                    return fail_cuda(cudaGetLastError(), "event create");
                ev.push_back(e0);
                ev.push_back(e1);
            }
            cudaEventRecord(ev[ev_used], s);
        }
        const double jw = n >= nsteps - window ? 1.0 / window : 0.0;
        lbk::k_adj_body_pre<<<(nb + 63) / 64, 64, 0, s>>>(bodies, w->adj, nb, jw != 0.0 ? body : -1, axis, jw);
        aa.fn = fn;
        aa.odd = ((n0 + n) & 1) != 0;
        aa.Fprev = Fprev;
        aa.Fnew = Fnew;
        aa.lam_in = w->lam[cur];
        aa.lam_out = w->lam[cur ^ 1];
        aa.lFp_in = w->lFp[cur];
        aa.lFn = w->lFn;
        aa.lFp_out = w->lFp[cur ^ 1];
        if (h->fp32) lbk::k_adj_collide<float><<<grid, block, 0, s>>>(aa);
        else lbk::k_adj_collide<double><<<grid, block, 0, s>>>(aa);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(e, "adjoint collide launch");
        lbk::AdjCouple ac{};
        ac.g = h->g;
        ac.fn = fn;
        ac.odd = aa.odd;
        ac.rho0 = h->p.rho0;
        ac.gamma = h->p.gamma_bead;
        ac.gforce = h->gforce;
        ac.Fprev = Fprev;
        ac.lFn = w->lFn;
        ac.lam_f = w->lam[cur ^ 1];
        ac.lFp = w->lFp[cur ^ 1];
        ac.s = h->ds;
        ac.bead_body = h->dbody_of;
        ac.bodies = bodies;
        ac.adj = w->adj;
        ac.dJds = w->dJds;
        ac.lgam = w->lgam;
        ac.nbeads = nbeads;
        const unsigned cg = (unsigned)((8LL * nbeads + 127) / 128);
        if (h->fp32) lbk::k_adj_couple<float><<<cg, 128, 0, s>>>(ac);
        else lbk::k_adj_couple<double><<<cg, 128, 0, s>>>(ac);
        lbk::k_adj_body_post<<<(nb + 63) / 64, 64, 0, s>>>(bodies, w->adj, nb);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail_cuda(e, "adjoint coupling launch");
        if (timed) {
            cudaEventRecord(ev[ev_used + 1], s);
            ev_used += 2;
        }
        cur ^= 1;
        ++reversed;
        return LB_OK;
    }

    // The turn at relative step n (the handle holds the state before it):
    // re-run its prologue and coupling, then reverse it in place.
    lb_status turn(int n) {
        mark_first();
        cudaError_t e = cudaMemcpyAsync(w->turn_bodies, h->db, z.bbytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail_cuda(e, "turn copy");
        lb_status st = lbk::ctx_turn(h, pops());
        if (st != LB_OK) return st;
        const int curb = (int)((n0 + n) & 1), prev = curb ^ 1;
        return reverse_step(n, pops(), h->Fbuf[prev], h->Fbuf[curb], w->turn_bodies);
    }
};

// Two-level schedule: snapshots every K steps in the forward sweep, each
// segment re-run with every step taped, then walked backwards.
lb_status run_two_level(Run &R, int c) {
    AdjWork *w = R.w;
    lb_ctx *h = R.h;
    const int T = R.nsteps;
    const int K = (T + c - 1) / c, nseg = (T + K - 1) / K;
    for (int sg = 0; sg < nseg; ++sg) {
        cudaError_t e = R.save(w->snaps[sg]);
        if (e != cudaSuccess) return R.fail_cuda(e, "snapshot");
        const int a0 = sg * K, a1 = std::min(T, a0 + K);
        lb_status st = R.advance(a0, a1);
        if (st != LB_OK) return st;
    }
    cudaError_t e = R.save(w->snaps[nseg]);
    if (e != cudaSuccess) return R.fail_cuda(e, "snapshot");
    R.mark_first();
    // The re-run of steps [a0, a1) from the state in tape entry 0: each step
    // reads the populations where the one before left them and stores its own
    // into the next entry (the last into the handle's array), so the tape is
    // written by the steps themselves.
    auto rerun = [&](int a0, int a1) -> lb_status {
        for (int n = a0; n < a1; ++n) {
            Tape &Tp = w->tape[n - a0];
            const int curb = (int)((R.n0 + n) & 1);
            cudaError_t ce = cudaMemcpyAsync(Tp.bodies, h->db, R.z.bbytes, cudaMemcpyDeviceToDevice, R.s);
            if (ce != cudaSuccess) return R.fail_cuda(ce, "tape");
            void *dst = n + 1 < a1 ? w->tape[n + 1 - a0].f : h->f;
            lb_status st = lbk::ctx_step_oop(h, Tp.f, dst);
            if (st != LB_OK) return st;
            ce = cudaMemcpyAsync(Tp.Fnew, h->Fbuf[curb], R.z.Fbytes, cudaMemcpyDeviceToDevice, R.s);
            if (ce != cudaSuccess) return R.fail_cuda(ce, "tape");
        }
        return LB_OK;
    };
    // A full segment re-runs the same steps on the same buffers whatever its
    // snapshot (entry 0 receives the snapshot's populations), so its launches
    // are captured once per starting parity as a CUDA graph and replayed:
    // host launch cost would otherwise exceed the segment's device time.
    cudaGraphExec_t gx[2] = {nullptr, nullptr};
    bool graphs = K > 1 && !h->timing;      // per-kernel timing events stay eager
    auto drop = [&]() {
        for (auto &g : gx)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    };
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const Snapshot &Sg = w->snaps[sg];
        if ((e = R.restore(Sg)) != cudaSuccess) return drop(), R.fail_cuda(e, "restore");
        if ((e = cudaMemcpyAsync(w->tape[0].f, Sg.f, R.z.fbytes, cudaMemcpyDeviceToDevice, R.s)) != cudaSuccess)
            return drop(), R.fail_cuda(e, "tape");
        const int a0 = sg * K, a1 = std::min(T, a0 + K);
        R.recompute_steps += a1 - a0;
        lb_status st = LB_OK;
        const int p = (int)((R.n0 + a0) & 1);
        if (graphs && a1 - a0 == K && !gx[p]) {
            // capture (nothing runs; the host step mirror is put back after)
            const long long step0 = h->step;
            cudaGraph_t gr = nullptr;
            e = cudaStreamBeginCapture(R.s, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                st = rerun(a0, a1);
                e = cudaStreamEndCapture(R.s, &gr);
                if (st == LB_OK && e == cudaSuccess) e = cudaGraphInstantiate(&gx[p], gr, 0);
                if (gr) cudaGraphDestroy(gr);
            }
            h->step = step0;
            if (st != LB_OK) return drop(), st;
            if (e != cudaSuccess) {           // not capturable here: step eagerly from now on
                cudaGetLastError();
                gx[p] = nullptr;
                graphs = false;
            }
        }
        if (graphs && a1 - a0 == K && gx[p]) {
            if ((e = cudaGraphLaunch(gx[p], R.s)) != cudaSuccess) return drop(), R.fail_cuda(e, "re-run graph");
            h->step += K;
        } else if ((st = rerun(a0, a1)) != LB_OK) {
            return drop(), st;
        }
        R.cf = nullptr;
        const int prev0 = p ^ 1;
        for (int n = a1 - 1; n >= a0; --n) {
            const Tape &Tp = w->tape[n - a0];
            const void *Fprev = n == a0 ? Sg.F[prev0] : w->tape[n - 1 - a0].Fnew;
            st = R.reverse_step(n, Tp.f, Fprev, Tp.Fnew, Tp.bodies);
            if (st != LB_OK) return drop(), st;
        }
    }
    drop();
    // leave the handle where the forward sweep ended
    if ((e = R.restore(w->snaps[nseg], true)) != cudaSuccess) return R.fail_cuda(e, "restore");
    return LB_OK;
}

// Binomial (revolve) schedule. Slot `fin` receives the final state; the
// other slots hold checkpoints. `have` is the relative step the handle
// holds as a whole state (-1 after a turn).
struct Binomial {
    Run &R;
    int fin;
    std::vector<int> free_slots;
    int have = 0;
    bool final_saved = false;

    static double choose(int n, int k) {
        double r = 1.0;
        for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
        return r;
    }

    lb_status to_state(int a, int slot_a) {
        if (have == a) return LB_OK;
        cudaError_t e = R.restore(R.w->snaps[slot_a]);
        if (e != cudaSuccess) return R.fail_cuda(e, "restore");
        have = a;
        return LB_OK;
    }

    // the turn at step a (state a in slot_a): before the first turn, the last
    // step is run whole once so that the final state can be kept
    lb_status turn_at(int a, int slot_a) {
        lb_status st = to_state(a, slot_a);
        if (st != LB_OK) return st;
        if (!final_saved) {
            if ((st = R.advance(a, a + 1)) != LB_OK) return st;
            cudaError_t e = R.save(R.w->snaps[fin]);
            if (e != cudaSuccess) return R.fail_cuda(e, "snapshot");
            final_saved = true;
            R.mark_first();
            have = a + 1;
            if ((st = to_state(a, slot_a)) != LB_OK) return st;
        }
        st = R.turn(a);
        have = -1;
        return st;
    }

    // reverse steps [a, b) given state a in slot_a and the free slots
    lb_status reverse(int a, int b, int slot_a) {
        const int l = b - a;
        if (l == 1) return turn_at(a, slot_a);
        const int S = (int)free_slots.size() + 1;   // states available, slot_a included
        lb_status st;
        if (S == 1) {
            for (int n = b - 1; n >= a; --n) {
                if ((st = to_state(a, slot_a)) != LB_OK) return st;
                if ((st = R.advance(a, n)) != LB_OK) return st;
                have = n;
                if (n == a) { if ((st = turn_at(a, slot_a)) != LB_OK) return st; continue; }
                // state n is held but has no slot: the final state needs it whole first
                if (!final_saved) {
                    if ((st = R.advance(n, n + 1)) != LB_OK) return st;
                    cudaError_t e = R.save(R.w->snaps[fin]);
                    if (e != cudaSuccess) return R.fail_cuda(e, "snapshot");
                    final_saved = true;
                    R.mark_first();
                    have = -1;
                    if ((st = to_state(a, slot_a)) != LB_OK) return st;
                    if ((st = R.advance(a, n)) != LB_OK) return st;
                    have = n;
                }
                if ((st = R.turn(n)) != LB_OK) return st;
                have = -1;
            }
            return LB_OK;
        }
        int r = 0;
        while (choose(S + r, S) < (double)l) ++r;
        int m1 = (int)std::min((double)(l - 1), choose(S + r - 1, S));
        if (m1 < 1) m1 = 1;
        const int m = a + m1;
        if ((st = to_state(a, slot_a)) != LB_OK) return st;
        if ((st = R.advance(a, m)) != LB_OK) return st;
        have = m;
        const int slot_m = free_slots.back();
        free_slots.pop_back();
        cudaError_t e = R.save(R.w->snaps[slot_m]);
        if (e != cudaSuccess) return R.fail_cuda(e, "snapshot");
        if ((st = reverse(m, b, slot_m)) != LB_OK) return st;
        free_slots.push_back(slot_m);
        return reverse(a, m, slot_a);
    }
};

lb_status run_binomial(Run &R, int S) {
    // slots 0..S-1 checkpoints (slot 0: the start state), slot S the final state
    Binomial B{R, S, {}, 0, false};
    for (int k = S - 1; k >= 1; --k) B.free_slots.push_back(k);
    cudaError_t e = R.save(R.w->snaps[0]);
    if (e != cudaSuccess) return R.fail_cuda(e, "snapshot");
    lb_status st = B.reverse(0, R.nsteps, 0);
    if (st != LB_OK) return st;
    if ((e = R.restore(R.w->snaps[S], true)) != cudaSuccess) return R.fail_cuda(e, "restore");
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_adjoint_drag_ex(lb_handle h, int nsteps, int window, int body, int axis,
                                        const lb_adjoint_opts *opts, double *J, double *dJ_dgamma,
                                        double *dJ_dbeads, lb_adjoint_stats *stats) {
    if (!h) return LB_ERR_ARG;
    if (nsteps < 1 || window < 1 || window > nsteps || axis < 0 || axis > 2 || !J || !dJ_dgamma)
        return lbk::ctx_fail(h, LB_ERR_ARG, "need nsteps >= window >= 1, axis 0-2, J and dJ_dgamma");
    const int schedule = opts ? opts->schedule : LB_ADJ_TWO_LEVEL;
    const int snapshots = opts ? opts->snapshots : 0;
    if ((schedule != LB_ADJ_TWO_LEVEL && schedule != LB_ADJ_BINOMIAL) || snapshots < 0)
        return lbk::ctx_fail(h, LB_ERR_ARG, "unknown adjoint schedule or snapshots < 0");
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

    int nsnap, ntape, c = 0, S = 0;
    if (schedule == LB_ADJ_TWO_LEVEL) {
        c = snapshots > 0 ? snapshots : (int)std::ceil(std::sqrt((double)nsteps));
        if (c > nsteps) c = nsteps;
        const int K = (nsteps + c - 1) / c;
        nsnap = (nsteps + K - 1) / K + 1;
        ntape = K;
    } else {
        S = snapshots > 0 ? snapshots : 16;
        if (S > nsteps) S = nsteps;
        nsnap = S + 1;
        ntape = 0;
    }
    double alloc_ms = 0.0;
    if ((st = ensure_work(h, nsnap, ntape, nsteps, &alloc_ms)) != LB_OK) return st;
    AdjWork *w = h->adjw;

    Run R{};
    R.h = h;
    R.w = w;
    R.z = sizes_of(h);
    R.s = h->stream;
    R.nsteps = nsteps;
    R.window = window;
    R.body = body;
    R.axis = axis;
    R.n0 = h->step;
    R.timed = stats != nullptr;
    R.block = h->block;
    R.grid = dim3((h->g.nx + h->block.x - 1) / h->block.x, (h->g.ny + h->block.y - 1) / h->block.y, h->g.nz);
    R.aa.g = h->g;
    R.aa.gforce = h->gforce;
    R.aa.gforce_f = h->gforce_f;
    {
        static const int modes[6] = {4, 5, 6, 7, 8, 9};
        auto rate = [&](int k) {
            if (h->p.collision == 0) return 1.0 - 1.0 / h->p.tau;   // BGK = MRT with equal rates
            return k == 4 ? h->p.gamma_bulk : (k <= 9 ? h->p.gamma_shear : (k <= 15 ? h->p.gamma_odd : h->p.gamma_even));
        };
        R.aa.pd.rho0 = h->p.rho0;
        for (int q = 0; q < 6; ++q) {
            R.aa.pd.A[q] = 1.0 - rate(modes[q]);
            R.aa.pd.H[q] = 0.5 * (1.0 + rate(modes[q]));
        }
        for (int k = 4; k <= 18; ++k) R.aa.pd.G[k - 4] = rate(k);
        R.aa.pf.rho0 = (float)R.aa.pd.rho0;
        for (int q = 0; q < 6; ++q) { R.aa.pf.A[q] = (float)R.aa.pd.A[q]; R.aa.pf.H[q] = (float)R.aa.pd.H[q]; }
        for (int q = 0; q < 15; ++q) R.aa.pf.G[q] = (float)R.aa.pd.G[q];
    }
    auto destroy_events = [&]() {
        for (cudaEvent_t e : R.ev) cudaEventDestroy(e);
        if (R.ev_start) cudaEventDestroy(R.ev_start);
        if (R.ev_first) cudaEventDestroy(R.ev_first);
        if (R.ev_end) cudaEventDestroy(R.ev_end);
    };
    cudaError_t e = cudaSuccess;
    if (R.timed) {
        R.ev.reserve(2 * (size_t)nsteps);
        e = cudaEventCreate(&R.ev_start);
        if (e == cudaSuccess) e = cudaEventCreate(&R.ev_first);
        if (e == cudaSuccess) e = cudaEventCreate(&R.ev_end);
        if (e == cudaSuccess) e = cudaEventRecord(R.ev_start, R.s);
        if (e != cudaSuccess) {
            destroy_events();
            return R.fail_cuda(e, "events");
        }
    }
    const long long N = h->g.N;
    e = R.zero(w->lam[0], 19 * N);
    if (e == cudaSuccess) e = R.zero(w->lFp[0], 3 * N);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->adj, 0, sizeof(BodyAdj) * nb, R.s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->dJds, 0, sizeof(double) * 3 * nbeads, R.s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->lgam, 0, sizeof(double), R.s);
    if (e != cudaSuccess) {
        destroy_events();
        return R.fail_cuda(e, "adjoint init");
    }
    st = schedule == LB_ADJ_TWO_LEVEL ? run_two_level(R, c) : run_binomial(R, S);
    if (st != LB_OK) {
        destroy_events();
        return st;
    }
    std::vector<double> vh(nsteps);
    e = cudaMemcpyAsync(vh.data(), w->vhist, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, R.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dJ_dgamma, w->lgam, sizeof(double), cudaMemcpyDeviceToHost, R.s);
    if (e == cudaSuccess && dJ_dbeads)
        e = cudaMemcpyAsync(dJ_dbeads, w->dJds, sizeof(double) * 3 * nbeads, cudaMemcpyDeviceToHost, R.s);
    if (e == cudaSuccess && R.timed) e = cudaEventRecord(R.ev_end, R.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(R.s);
    if (e != cudaSuccess) {
        destroy_events();
        return R.fail_cuda(e, "adjoint read-back");
    }
    double Jv = 0.0;
    for (int n = nsteps - window; n < nsteps; ++n) Jv += vh[n];
    *J = Jv / window;
    if (stats) {
        float total = 0.f, first = 0.f, rev = 0.f;
        cudaEventElapsedTime(&total, R.ev_start, R.ev_end);
        cudaEventElapsedTime(&first, R.ev_start, R.ev_first);
        for (size_t k = 0; k + 1 < R.ev_used; k += 2) {
            float t = 0.f;
            cudaEventElapsedTime(&t, R.ev[k], R.ev[k + 1]);
            rev += t;
        }
        stats->alloc_ms = alloc_ms;
        stats->forward_ms = first;
        stats->reverse_ms = rev;
        stats->recompute_ms = (double)total - first - rev;
        stats->forward_steps = R.forward_steps;
        stats->recompute_steps = R.recompute_steps;
        stats->reversed_steps = R.reversed;
        stats->workspace_bytes = (double)w->bytes;
    }
    destroy_events();
    return LB_OK;
}

extern "C" lb_status lb_adjoint_drag(lb_handle h, int nsteps, int window, int body, int axis, int checkpoints,
                                     double *J, double *dJ_dgamma, double *dJ_dbeads) {
    lb_adjoint_opts o{LB_ADJ_TWO_LEVEL, checkpoints < 0 ? 0 : checkpoints};
    if (h && checkpoints < 0) return lbk::ctx_fail(h, LB_ERR_ARG, "checkpoints must be >= 0");
    return lb_adjoint_drag_ex(h, nsteps, window, body, axis, &o, J, dJ_dgamma, dJ_dbeads, nullptr);
}
