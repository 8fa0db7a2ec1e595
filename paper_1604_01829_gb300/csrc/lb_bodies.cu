// Raspberry kernels (Ustach & Faller, arXiv:1604.01829):
//  - rigid-body integration of the centre of mass by velocity Verlet and of
//    the orientation by a quaternion (Sec. 2.3), one thread per body in FP64;
//  - virtual sites r_b = X + R(q) s_b, v_b = V + omega x (r_b - X) (Sec. 1.2);
//  - friction coupling F_b = -gamma (v_b - u(r_b)) + f_s, Eq.
//    (latticeboltzmannfriction) in Sec. 1.1, with u trilinearly interpolated
//    from the 8 surrounding nodes and -F_b spread back onto the same nodes
//    with the same weights, so the exchange conserves momentum; bead forces
//    and torques summed onto the body (Sec. 2.3).
#include "lb_internal.h"

namespace lbk {

namespace {

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// lab = R body, Hamilton convention, q = (w, x, y, z)
__device__ __forceinline__ void quat_to_R(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - z * w); R[2] = 2.0 * (x * z + y * w);
    R[3] = 2.0 * (x * y + z * w); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - x * w);
    R[6] = 2.0 * (x * z - y * w); R[7] = 2.0 * (y * z + x * w); R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Euler's equations I dw/dt = T - w x (I w) over half a step, explicit in w
__device__ __forceinline__ void euler_half_explicit(double w[3], const double I[3], const double T[3]) {
    const double Iw[3] = {I[0] * w[0], I[1] * w[1], I[2] * w[2]};
    double c[3];
    cross3(w, Iw, c);
    for (int a = 0; a < 3; ++a) w[a] += 0.5 * (T[a] - c[a]) / I[a];
}

// ... and implicit in w (fixed point), so that the two half kicks around a
// step boundary form the trapezoidal rule: a second-order, time-symmetric
// rotation update like the velocity-Verlet rotation schemes of Sec. 2.3.
__device__ __forceinline__ void euler_half_implicit(double w[3], const double I[3], const double T[3]) {
    const double w0[3] = {w[0], w[1], w[2]};
    for (int it = 0; it < 6; ++it) {
        const double Iw[3] = {I[0] * w[0], I[1] * w[1], I[2] * w[2]};
        double c[3];
        cross3(w, Iw, c);
        for (int a = 0; a < 3; ++a) w[a] = w0[a] + 0.5 * (T[a] - c[a]) / I[a];
    }
}

// Totals of a finished step, then its second half kick: V += F/(2M),
// implicit Euler half kick of the body-frame omega.
__device__ void kick2(Body &B) {
    double Tb[3];
    for (int a = 0; a < 3; ++a) {
        B.F_tot[a] = B.acc[a] + B.F_ext[a];
        B.T_tot[a] = B.acc[3 + a] + B.T_ext[a];
    }
    for (int a = 0; a < 3; ++a) Tb[a] = B.R[a] * B.T_tot[0] + B.R[3 + a] * B.T_tot[1] + B.R[6 + a] * B.T_tot[2];
    for (int a = 0; a < 3; ++a) {
        B.F_last[a] = B.F_tot[a];
        B.T_last[a] = Tb[a];
    }
    if (B.fixed) return;
    for (int a = 0; a < 3; ++a) B.V[a] += 0.5 * B.F_tot[a] / B.mass;
    euler_half_implicit(B.w, B.I, Tb);
}

// First half kick with last step's force and torque, then drift: X += V,
// q <- q (x) exp(omega/2) with the half-step body-frame omega.
__device__ void kick_drift(Body &B) {
    if (!B.fixed) {
        for (int a = 0; a < 3; ++a) {
            B.V[a] += 0.5 * B.F_last[a] / B.mass;
            B.X[a] += B.V[a];
        }
        euler_half_explicit(B.w, B.I, B.T_last);
        const double wn = sqrt(B.w[0] * B.w[0] + B.w[1] * B.w[1] + B.w[2] * B.w[2]);
        double *q = B.q;
        if (wn > 0.0) {
            double sh, ch;
            sincos(0.5 * wn, &sh, &ch);
            const double d[4] = {ch, sh * B.w[0] / wn, sh * B.w[1] / wn, sh * B.w[2] / wn};
            const double r[4] = {q[0] * d[0] - q[1] * d[1] - q[2] * d[2] - q[3] * d[3],
                                 q[0] * d[1] + q[1] * d[0] + q[2] * d[3] - q[3] * d[2],
                                 q[0] * d[2] - q[1] * d[3] + q[2] * d[0] + q[3] * d[1],
                                 q[0] * d[3] + q[1] * d[2] - q[2] * d[1] + q[3] * d[0]};
            for (int a = 0; a < 4; ++a) q[a] = r[a];
        }
        const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int a = 0; a < 4; ++a) q[a] /= qn;
    }
    quat_to_R(B.q, B.R);
    for (int a = 0; a < 3; ++a) B.wl[a] = B.R[3 * a] * B.w[0] + B.R[3 * a + 1] * B.w[1] + B.R[3 * a + 2] * B.w[2];
    for (int a = 0; a < 6; ++a) B.acc[a] = 0.0;
}

// Step prologue in one launch: threads [0, nb) finish the previous step's
// bodies (second half kick) if asked and start this step's (half kick,
// drift, rotation); every thread also clears one flagged 4x4x4 tile of this
// step's spread-force buffer.
__global__ void k_step_pre(Body *bodies, int nb, int finish_prev, double *F, unsigned char *tiles, Geom g,
                           int ntx, int nty, int ntz) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < nb) {
        Body &B = bodies[t];
        if (finish_prev) kick2(B);
        kick_drift(B);
    }
    const long long nt = (long long)ntx * nty * ntz;
    if (t >= nt || !tiles[t]) return;
    const int tx = (int)(t % ntx), ty = (int)((t / ntx) % nty), tz = (int)(t / ((long long)ntx * nty));
    for (int dz = 0; dz < 4; ++dz) {
        const int z = 4 * tz + dz;
        if (z >= g.nz) break;
        for (int dy = 0; dy < 4; ++dy) {
            const int y = 4 * ty + dy;
            if (y >= g.ny) break;
            for (int dx = 0; dx < 4; ++dx) {
                const int x = 4 * tx + dx;
                if (x >= g.nx) break;
                const long long n = nidx(g, x, y, z);
                F[n] = 0.0;
                F[g.N + n] = 0.0;
                F[2 * g.N + n] = 0.0;
            }
        }
    }
    tiles[t] = 0;
}

// Pre-collision density and momentum of one node in the compute precision R.
template <typename R, typename T>
__device__ __forceinline__ void node_rho_j(const T *A, const Geom &g, int x, int y, int z, long long n,
                                           bool odd, R rho0, R &rho, R j[3]) {
    R s = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const R v = (R)load_pre(A, g, x, y, z, n, i, odd);
        s += v;
        if (cx(i)) jx += cx(i) * v;
        if (cy(i)) jy += cy(i) * v;
        if (cz(i)) jz += cz(i) * v;
    }
    rho = sizeof(T) == 4 ? rho0 + s : s;
    j[0] = jx; j[1] = jy; j[2] = jz;
}

// Eight lanes per bead, one per surrounding node: lane 0 of the group forms
// the virtual site, every lane interpolates its node's velocity and spreads
// its share of -F_b, the group reduces by shuffles. Node arithmetic runs in
// the storage precision (FP32 deviations or FP64), bead and body sums in FP64.
template <typename T>
__global__ void __launch_bounds__(128) k_couple(const CoupleArgs a) {
    using R = T;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t >> 3;
    const int c = t & 7;
    const int lane = threadIdx.x & 31;
    const bool active = k < a.nbeads;
    const Geom &g = a.g;
    const T *A = static_cast<const T *>(a.f);
    const int body = active ? a.bead_body[k] : -1;

    double rel[3] = {0, 0, 0}, r[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    if (active && c == 0) {
        const Body &B = a.bodies[body];
        const double s[3] = {a.s[3 * k], a.s[3 * k + 1], a.s[3 * k + 2]};
        double wxr[3];
        for (int q = 0; q < 3; ++q) rel[q] = B.R[3 * q] * s[0] + B.R[3 * q + 1] * s[1] + B.R[3 * q + 2] * s[2];
        for (int q = 0; q < 3; ++q) r[q] = B.X[q] + rel[q];
        cross3(B.wl, rel, wxr);
        for (int q = 0; q < 3; ++q) v[q] = B.V[q] + wxr[q];
    }
    for (int q = 0; q < 3; ++q) r[q] = __shfl_sync(0xffffffffu, r[q], 0, 8);

    // this lane's node among the 8 around r (centres at integer + 1/2), periodic
    const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    const int n3[3] = {g.nx, g.ny, g.nz};
    int xyz[3];
    double wt = 1.0;
    for (int q = 0; q < 3; ++q) {
        const double tq = r[q] - 0.5;
        const double fl = floor(tq);
        const double fr = tq - fl;
        int b0 = (int)fl % n3[q];
        if (b0 < 0) b0 += n3[q];
        xyz[q] = o[q] ? (b0 + 1 == n3[q] ? 0 : b0 + 1) : b0;
        wt *= o[q] ? fr : 1.0 - fr;
    }
    const long long n = nidx(g, xyz[0], xyz[1], xyz[2]);
    const bool fluid = active && !is_wall(g, xyz[0], xyz[1], xyz[2]);
    double ub[3] = {0.0, 0.0, 0.0};
    if (fluid) {                         // wall nodes carry u = 0
        R rho, j[3];
        node_rho_j<R>(A, g, xyz[0], xyz[1], xyz[2], n, a.odd, (R)a.rho0, rho, j);
        const R ir = R(1) / rho;
        const R ux = (j[0] + R(0.5) * (R)(a.gforce[0] + a.Fprev[n])) * ir;
        const R uy = (j[1] + R(0.5) * (R)(a.gforce[1] + a.Fprev[g.N + n])) * ir;
        const R uz = (j[2] + R(0.5) * (R)(a.gforce[2] + a.Fprev[2 * g.N + n])) * ir;
        ub[0] = wt * (double)ux;
        ub[1] = wt * (double)uy;
        ub[2] = wt * (double)uz;
    }
    for (int off = 1; off < 8; off <<= 1)
        for (int q = 0; q < 3; ++q) ub[q] += __shfl_xor_sync(0xffffffffu, ub[q], off, 8);

    // Eq. (latticeboltzmannfriction): F_b = -gamma (v - u(r)) + f_s
    double Fb[3] = {0.0, 0.0, 0.0};
    if (active && c == 0) {
        double fs[3] = {0.0, 0.0, 0.0};
        if (a.noise_amp > 0.0) {
            const uint32_t step = (uint32_t)(*a.step_base) + a.step_off;
            const uint4 rr = philox4x32_10(make_uint4((uint32_t)k, step, a.instance, 4u), make_uint2(a.key0, a.key1));
            fs[0] = a.noise_amp * unit_uniform_d(rr.x);
            fs[1] = a.noise_amp * unit_uniform_d(rr.y);
            fs[2] = a.noise_amp * unit_uniform_d(rr.z);
        }
        for (int q = 0; q < 3; ++q) Fb[q] = -a.gamma * (v[q] - ub[q]) + fs[q];
        for (int q = 0; q < 3; ++q) a.F_bead[3 * k + q] = Fb[q];
    }
    for (int q = 0; q < 3; ++q) Fb[q] = __shfl_sync(0xffffffffu, Fb[q], 0, 8);

    // spread -w F_b onto this lane's node; a wall node takes nothing
    if (fluid) {
        atomicAdd(&a.Fcur[n], -wt * Fb[0]);
        atomicAdd(&a.Fcur[g.N + n], -wt * Fb[1]);
        atomicAdd(&a.Fcur[2 * g.N + n], -wt * Fb[2]);
        a.tiles_cur[tile_of(xyz[0], xyz[1], xyz[2], a.ntx, a.nty)] = 1;
    }

    // force and torque on the body: sum the (up to 4) beads of this warp
    // that belong to the warp's first body, atomics for the others
    double FT[6] = {0, 0, 0, 0, 0, 0};
    if (active && c == 0) {
        double tq[3];
        cross3(rel, Fb, tq);
        for (int q = 0; q < 3; ++q) { FT[q] = Fb[q]; FT[3 + q] = tq[q]; }
    }
    const int b_first = __shfl_sync(0xffffffffu, body, 0);
    const bool lead = active && c == 0;
    const bool same = lead && body == b_first;
    double red[6];
    for (int q = 0; q < 6; ++q) red[q] = same ? FT[q] : 0.0;
    for (int q = 0; q < 6; ++q) {
        red[q] += __shfl_xor_sync(0xffffffffu, red[q], 8);
        red[q] += __shfl_xor_sync(0xffffffffu, red[q], 16);
    }
    if (lane == 0 && b_first >= 0)
        for (int q = 0; q < 6; ++q) atomicAdd(&a.bodies[b_first].acc[q], red[q]);
    if (lead && !same)
        for (int q = 0; q < 6; ++q) atomicAdd(&a.bodies[body].acc[q], FT[q]);
}

__global__ void k_kick2(Body *bodies, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) kick2(bodies[b]);
}

}  // namespace

cudaError_t launch_step_pre(Body *b, int nbodies, bool finish_prev, double *F, unsigned char *tiles,
                            const Geom &g, int ntx, int nty, int ntz, cudaStream_t s) {
    const long long nt = (long long)ntx * nty * ntz;
    const long long n = nt > nbodies ? nt : nbodies;
    k_step_pre<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b, nbodies, finish_prev ? 1 : 0, F, tiles, g, ntx,
                                                           nty, ntz);
    return cudaGetLastError();
}

cudaError_t launch_couple(const CoupleArgs &a, cudaStream_t s) {
    if (a.nbeads <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((8LL * a.nbeads + 127) / 128);
    if (a.fp32) k_couple<float><<<grid, 128, 0, s>>>(a);
    else k_couple<double><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_kick2(Body *b, int nbodies, cudaStream_t s) {
    if (nbodies <= 0) return cudaSuccess;
    k_kick2<<<(nbodies + 63) / 64, 64, 0, s>>>(b, nbodies);
    return cudaGetLastError();
}

}  // namespace lbk
