// Rigid raspberry bodies (Ustach & Faller, arXiv:1604.01829, Sec. 1.2 and
// Sec. 2.3): quaternion rotation, velocity-Verlet half kicks and drift. One
// thread per body, FP64; shared by the single-lattice and batched paths.
#pragma once

#include "lb_internal.h"

namespace lbk {

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

// Euler's equations I dw/dt = T - w x (I w) over half a step of length dt,
// explicit in w
__device__ __forceinline__ void euler_half_explicit(double w[3], const double I[3], const double invI[3],
                                                    const double T[3], double dt) {
    const double Iw[3] = {I[0] * w[0], I[1] * w[1], I[2] * w[2]};
    double c[3];
    cross3(w, Iw, c);
    for (int a = 0; a < 3; ++a) w[a] += 0.5 * dt * (T[a] - c[a]) * invI[a];
}

// ... and implicit in w (fixed point), so that the two half kicks around a
// step boundary form the trapezoidal rule: a second-order, time-symmetric
// rotation update like the velocity-Verlet rotation schemes of Sec. 2.3.
__device__ __forceinline__ void euler_half_implicit(double w[3], const double I[3], const double invI[3],
                                                    const double T[3], double dt) {
    const double w0[3] = {w[0], w[1], w[2]};
    for (int it = 0; it < 6; ++it) {
        const double Iw[3] = {I[0] * w[0], I[1] * w[1], I[2] * w[2]};
        double c[3];
        cross3(w, Iw, c);
        for (int a = 0; a < 3; ++a) w[a] = w0[a] + 0.5 * dt * (T[a] - c[a]) * invI[a];
    }
}

// Totals of a finished (sub)step, then its second half kick over dt:
// V += dt F/(2M), implicit Euler half kick of the body-frame omega. dt = 1
// without MD substeps (dt = 1/n with n substeps per LB step).
__device__ __forceinline__ void kick2(Body &B, double dt = 1.0) {
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
    if (B.fixed == 1) return;
    for (int a = 0; a < 3; ++a) B.V[a] += 0.5 * dt * B.F_tot[a] * B.inv_mass;
    if (B.fixed == 2) return;          // orientation held
    euler_half_implicit(B.w, B.I, B.inv_I, Tb, dt);
}

// First half kick over dt with the last (sub)step's force and torque, then
// drift: X += dt V, q <- q (x) exp(omega dt / 2) with the half-step
// body-frame omega.
__device__ __forceinline__ void kick_drift(Body &B, double dt = 1.0) {
    if (B.fixed == 2) {                // translation only, orientation held
        for (int a = 0; a < 3; ++a) {
            B.V[a] += 0.5 * dt * B.F_last[a] * B.inv_mass;
            B.X[a] += dt * B.V[a];
            B.w[a] = 0.0;
        }
    } else if (!B.fixed) {
        for (int a = 0; a < 3; ++a) {
            B.V[a] += 0.5 * dt * B.F_last[a] * B.inv_mass;
            B.X[a] += dt * B.V[a];
        }
        euler_half_explicit(B.w, B.I, B.inv_I, B.T_last, dt);
        const double wn = sqrt(B.w[0] * B.w[0] + B.w[1] * B.w[1] + B.w[2] * B.w[2]);
        double *q = B.q;
        if (wn > 0.0) {
            double sh, ch;
            sincos(0.5 * wn * dt, &sh, &ch);
            const double sw = sh / wn;
            const double d[4] = {ch, sw * B.w[0], sw * B.w[1], sw * B.w[2]};
            const double r[4] = {q[0] * d[0] - q[1] * d[1] - q[2] * d[2] - q[3] * d[3],
                                 q[0] * d[1] + q[1] * d[0] + q[2] * d[3] - q[3] * d[2],
                                 q[0] * d[2] - q[1] * d[3] + q[2] * d[0] + q[3] * d[1],
                                 q[0] * d[3] + q[1] * d[2] - q[2] * d[1] + q[3] * d[0]};
            for (int a = 0; a < 4; ++a) q[a] = r[a];
        }
        const double iqn = rsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int a = 0; a < 4; ++a) q[a] *= iqn;
    }
    quat_to_R(B.q, B.R);
    for (int a = 0; a < 3; ++a) B.wl[a] = B.R[3 * a] * B.w[0] + B.R[3 * a + 1] * B.w[1] + B.R[3 * a + 2] * B.w[2];
    for (int a = 0; a < 6; ++a) B.acc[a] = 0.0;
    for (int a = 0; a < 9; ++a) B.Rf[a] = (float)B.R[a];
    for (int a = 0; a < 3; ++a) {
        B.Vf[a] = (float)B.V[a];
        B.wlf[a] = (float)B.wl[a];
        const double h = B.X[a] - 0.5, fl = floor(h);
        B.Xi[a] = (int)fl;
        B.Xf[a] = (float)(h - fl);
    }
}

// Trajectory record of body b after the drift of step *step_base + step_off.
__device__ __forceinline__ void record_body(const Recorder &r, const Body &B, int b, int nb) {
    if (!r.ring) return;
    const unsigned long long t1 = *r.step_base + r.step_off + 1ull;
    if (t1 % (unsigned long long)r.every) return;
    const unsigned long long slot = (t1 / (unsigned long long)r.every - 1ull) % (unsigned long long)r.cap;
    double *o = r.ring + (slot * (unsigned long long)nb + (unsigned long long)b) * 7ull;
    o[0] = B.X[0];
    o[1] = B.X[1];
    o[2] = B.X[2];
    o[3] = B.q[0];
    o[4] = B.q[1];
    o[5] = B.q[2];
    o[6] = B.q[3];
}

}  // namespace lbk
