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

// First half kick with last step's force and torque, then drift: X += V,
// q <- q (x) exp(omega/2) with the half-step body-frame omega.
__global__ void k_kick_drift(Body *bodies, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    Body &B = bodies[b];
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

// Zero the spread-force entries of every flagged 4x4x4 tile and clear the flag.
__global__ void k_clear_tiles(double *F, unsigned char *tiles, Geom g, int ntx, int nty, int ntz) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
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

template <typename T>
__device__ __forceinline__ void node_rho_j(const T *A, const Geom &g, int x, int y, int z, long long n,
                                           bool odd, double rho0, double &rho, double j[3]) {
    double s = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const double v = (double)load_pre(A, g, x, y, z, n, i, odd);
        s += v;
        if (cx(i)) jx += cx(i) * v;
        if (cy(i)) jy += cy(i) * v;
        if (cz(i)) jz += cz(i) * v;
    }
    rho = sizeof(T) == 4 ? rho0 + s : s;
    j[0] = jx; j[1] = jy; j[2] = jz;
}

// One thread per bead.
template <typename T>
__global__ void __launch_bounds__(128) k_couple(const CoupleArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nbeads) return;
    const Geom &g = a.g;
    const T *A = static_cast<const T *>(a.f);
    Body &B = a.bodies[a.bead_body[k]];
    const double s[3] = {a.s[3 * k], a.s[3 * k + 1], a.s[3 * k + 2]};
    double rel[3], r[3], v[3], wxr[3];
    for (int c = 0; c < 3; ++c) rel[c] = B.R[3 * c] * s[0] + B.R[3 * c + 1] * s[1] + B.R[3 * c + 2] * s[2];
    for (int c = 0; c < 3; ++c) r[c] = B.X[c] + rel[c];
    cross3(B.wl, rel, wxr);
    for (int c = 0; c < 3; ++c) v[c] = B.V[c] + wxr[c];

    // 8 surrounding nodes (centres at integer + 1/2), periodic
    int base[3];
    double fr[3];
    for (int c = 0; c < 3; ++c) {
        const double t = r[c] - 0.5;
        const double fl = floor(t);
        base[c] = (int)fl;
        fr[c] = t - fl;
    }
    const int n3[3] = {g.nx, g.ny, g.nz};
    int cc[3][2];
    for (int c = 0; c < 3; ++c) {
        int b0 = base[c] % n3[c];
        if (b0 < 0) b0 += n3[c];
        cc[c][0] = b0;
        cc[c][1] = b0 + 1 == n3[c] ? 0 : b0 + 1;
    }
    const double gx = a.gforce[0], gy = a.gforce[1], gz = a.gforce[2];
    double ub[3] = {0.0, 0.0, 0.0};
    double wgt[8];
    long long nn[8];
    bool fl8[8];
#pragma unroll
    for (int ci = 0; ci < 8; ++ci) {
        const int ox = ci & 1, oy = (ci >> 1) & 1, oz = (ci >> 2) & 1;
        const double wt = (ox ? fr[0] : 1.0 - fr[0]) * (oy ? fr[1] : 1.0 - fr[1]) * (oz ? fr[2] : 1.0 - fr[2]);
        const int x = cc[0][ox], y = cc[1][oy], z = cc[2][oz];
        const long long n = nidx(g, x, y, z);
        wgt[ci] = wt;
        nn[ci] = n;
        fl8[ci] = !is_wall(g, x, y, z);
        if (!fl8[ci]) continue;             // wall nodes carry u = 0
        double rho, j[3];
        node_rho_j(A, g, x, y, z, n, a.odd, a.rho0, rho, j);
        ub[0] += wt * (j[0] + 0.5 * (gx + a.Fprev[n])) / rho;
        ub[1] += wt * (j[1] + 0.5 * (gy + a.Fprev[g.N + n])) / rho;
        ub[2] += wt * (j[2] + 0.5 * (gz + a.Fprev[2 * g.N + n])) / rho;
    }
    double fs[3] = {0.0, 0.0, 0.0};
    if (a.noise_amp > 0.0) {
        const uint32_t step = (uint32_t)(*a.step_base) + a.step_off;
        const uint4 rr = philox4x32_10(make_uint4((uint32_t)k, step, a.instance, 4u), make_uint2(a.key0, a.key1));
        fs[0] = a.noise_amp * unit_uniform_d(rr.x);
        fs[1] = a.noise_amp * unit_uniform_d(rr.y);
        fs[2] = a.noise_amp * unit_uniform_d(rr.z);
    }
    double Fb[3];
    for (int c = 0; c < 3; ++c) Fb[c] = -a.gamma * (v[c] - ub[c]) + fs[c];
    // spread -F_b with the interpolation weights; wall corners take nothing
#pragma unroll
    for (int ci = 0; ci < 8; ++ci) {
        if (!fl8[ci]) continue;
        const long long n = nn[ci];
        atomicAdd(&a.Fcur[n], -wgt[ci] * Fb[0]);
        atomicAdd(&a.Fcur[g.N + n], -wgt[ci] * Fb[1]);
        atomicAdd(&a.Fcur[2 * g.N + n], -wgt[ci] * Fb[2]);
        int x, y, z;
        x = (int)(n % g.nx);
        y = (int)((n / g.nx) % g.ny);
        z = (int)(n / ((long long)g.nx * g.ny));
        a.tiles_cur[tile_of(x, y, z, a.ntx, a.nty)] = 1;
    }
    for (int c = 0; c < 3; ++c) a.F_bead[3 * k + c] = Fb[c];
    double tq[3];
    cross3(rel, Fb, tq);
    for (int c = 0; c < 3; ++c) {
        atomicAdd(&B.acc[c], Fb[c]);
        atomicAdd(&B.acc[3 + c], tq[c]);
    }
}

// Totals, then the second half kick: V += F/(2M), implicit Euler half kick of w.
__global__ void k_kick2(Body *bodies, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    Body &B = bodies[b];
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

}  // namespace

cudaError_t launch_kick_drift(Body *b, int nbodies, cudaStream_t s) {
    if (nbodies <= 0) return cudaSuccess;
    k_kick_drift<<<(nbodies + 63) / 64, 64, 0, s>>>(b, nbodies);
    return cudaGetLastError();
}

cudaError_t launch_clear_tiles(double *F, unsigned char *tiles, const Geom &g, int ntx, int nty, int ntz,
                               cudaStream_t s) {
    const long long nt = (long long)ntx * nty * ntz;
    k_clear_tiles<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(F, tiles, g, ntx, nty, ntz);
    return cudaGetLastError();
}

cudaError_t launch_couple(const CoupleArgs &a, cudaStream_t s) {
    if (a.nbeads <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.nbeads + 127) / 128);
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
