// Friction coupling of one raspberry bead to the fluid (Ustach & Faller,
// arXiv:1604.01829, Sec. 1.1, Eq. (latticeboltzmannfriction)), shared by
// the single-lattice and batched coupling kernels.
#pragma once

#include "lb_rigid.cuh"

namespace lbk {

// Pre-collision density and momentum of one node in the compute precision R.
// A periodic box without walls (the common case) takes the neighbours from
// per-axis wrapped offsets, so the 19 loads issue back to back; boxes with
// walls go through load_pre (wall and moving-wall tests per link).
template <typename R, typename T>
__device__ __forceinline__ void node_rho_j(const T *A, const Geom &g, int x, int y, int z, long long n,
                                           bool odd, R rho0, R &rho, R j[3], int *err = nullptr) {
    R v[19];
    if (g.cmap) {                        // compact pore layout (batched pore instances)
#pragma unroll
        for (int i = 0; i < 19; ++i) v[i] = (R)compact_load_pre(A, g, x, y, z, i, odd);
    } else if (g.pore_axis < 0 && !g.chan) {
        const int nx = g.nx, nxy = g.nx * g.ny;
        const int xo[3] = {(x == 0 ? nx : x) - 1, x, x + 1 == nx ? 0 : x + 1};
        const int yo[3] = {((y == 0 ? g.ny : y) - 1) * nx, y * nx, (y + 1 == g.ny ? 0 : y + 1) * nx};
        const int zo[3] = {((z == 0 ? g.nz : z) - 1) * nxy, z * nxy, (z + 1 == g.nz ? 0 : z + 1) * nxy};
        if (!odd) {
#pragma unroll
            for (int i = 0; i < 19; ++i) v[i] = (R)A[(long long)i * g.N + chk(n, g.N, err)];
        } else {
            v[0] = (R)A[chk(n, g.N, err)];
#pragma unroll
            for (int i = 1; i < 19; ++i)
                v[i] = (R)A[(long long)opp(i) * g.N + chk((unsigned)(xo[1 - cx(i)] + yo[1 - cy(i)] + zo[1 - cz(i)]), g.N, err)];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 19; ++i) v[i] = (R)load_pre(A, g, x, y, z, n, i, odd);
    }
    R s = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        s += v[i];
        if (cx(i)) jx += cx(i) * v[i];
        if (cy(i)) jy += cy(i) * v[i];
        if (cz(i)) jz += cz(i) * v[i];
    }
    rho = sizeof(T) == 4 ? rho0 + s : s;
    j[0] = jx; j[1] = jy; j[2] = jz;
}

// WCA force of the pore-wall beads on a colloid bead at r (lab frame), from
// the wall beads in a window around the nearest one (the window covers every
// wall bead within the cutoff), minimum image along the periodic axis.
// Components are selected, not indexed, so nothing goes to local memory.
__device__ __forceinline__ void wall_bead_force(const WallBeads &w, const double r[3], double F[3]) {
    F[0] = F[1] = F[2] = 0.0;
    const int ax = w.axis;
    const double ru = ax == 0 ? r[1] : r[0], rv = ax == 2 ? r[1] : r[2], rz = ax == 0 ? r[0] : (ax == 1 ? r[1] : r[2]);
    const double du = ru - w.cu, dv = rv - w.cv;
    const double rho2 = du * du + dv * dv;
    const double reach = w.Rc - sqrt(w.rcut2);
    if (reach > 0.0 && rho2 < reach * reach) return;          // no wall bead within the cutoff
    const double twopi = 6.283185307179586;
    const double phi = atan2(dv, du);
    const int j0 = (int)lrint(phi * w.ntheta / twopi);
    const int k0 = (int)lrint(rz * w.nrow / w.L - 0.5);
    const bool all_j = 2 * w.wt + 1 >= w.ntheta, all_k = 2 * w.wz + 1 >= w.nrow;
    const int jlo = all_j ? 0 : j0 - w.wt, jhi = all_j ? w.ntheta - 1 : j0 + w.wt;
    const int klo = all_k ? 0 : k0 - w.wz, khi = all_k ? w.nrow - 1 : k0 + w.wz;
    for (int kk = klo; kk <= khi; ++kk) {
        int k = kk % w.nrow;
        if (k < 0) k += w.nrow;
        for (int jj = jlo; jj <= jhi; ++jj) {
            int j = jj % w.ntheta;
            if (j < 0) j += w.ntheta;
            double sn, cs;
            sincos(twopi * j / w.ntheta, &sn, &cs);
            const double eu = du - w.Rc * cs, ev = dv - w.Rc * sn;
            double ez = rz - (k + 0.5) * w.L / w.nrow;
            ez -= w.L * floor(ez / w.L + 0.5);
            const double d2 = eu * eu + ev * ev + ez * ez;
            if (d2 >= w.rcut2) continue;
            const double sr2 = w.sigma2 / d2, sr6 = sr2 * sr2 * sr2;
            const double fm = 24.0 * w.eps * (2.0 * sr6 * sr6 - sr6) / d2;
            // back to x, y, z: (u, v, axis) = (y, z, x), (x, z, y) or (x, y, z)
            if (ax == 0) { F[1] += fm * eu; F[2] += fm * ev; F[0] += fm * ez; }
            else if (ax == 1) { F[0] += fm * eu; F[2] += fm * ev; F[1] += fm * ez; }
            else { F[0] += fm * eu; F[1] += fm * ev; F[2] += fm * ez; }
        }
    }
}

// Force and torque of the pore-wall beads on every bead of a body (one
// thread per bead, FP64): added to the body's accumulators, not the fluid.
__device__ __forceinline__ void wall_bead_body(const WallBeads &w, Body *bodies, const double *s,
                                               const int *bead_body, int k) {
    Body &B = bodies[bead_body[k]];
    const double s0 = s[3 * k], s1 = s[3 * k + 1], s2 = s[3 * k + 2];
    double rel[3], r[3], F[3], tq[3];
    for (int q = 0; q < 3; ++q) {
        rel[q] = B.R[3 * q] * s0 + B.R[3 * q + 1] * s1 + B.R[3 * q + 2] * s2;
        r[q] = B.X[q] + rel[q];
    }
    wall_bead_force(w, r, F);
    if (F[0] == 0.0 && F[1] == 0.0 && F[2] == 0.0) return;
    cross3(rel, F, tq);
    for (int q = 0; q < 3; ++q) {
        atomicAdd(&B.acc[q], F[q]);
        atomicAdd(&B.acc[3 + q], tq[q]);
    }
}

// Flags `tile` in the tile flags of this step's force buffer when this lane
// spread a force onto one of its nodes (fluid) and, the first time a tile is
// flagged, appends it to the list of flagged tiles (cleared two steps later);
// the appends of a warp take one atomic on the list's counter. Every lane of
// the warp calls it (ballot).
__device__ __forceinline__ void flag_tile(const CoupleArgs &a, bool fluid, int tile, int lane) {
    const bool first = fluid && a.tiles_cur[tile] == 0 && atomicExch(&a.tiles_cur[tile], 1) == 0;
    const unsigned m = __ballot_sync(0xffffffffu, first);
    if (m == 0u) return;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(a.tcount, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (first) a.tlist[chk(base + __popc(m & ((1u << lane) - 1u)), a.list_cap, a.err)] = a.tile_base + tile;
}

// FP32 storage: the same coupling with every per-bead quantity in FP32
// (GB300's FP64 pipe is narrow and one bead's FP64 work, done by one lane,
// would bound the kernel). The virtual site is formed relative to the body:
// floor and fraction of X - 1/2 come from the body (FP64, once per step),
// the offset R s in FP32 (|s| of a few units: 1e-6 absolute), so positions
// keep their resolution for any box size. Body sums are accumulated in FP64.
__device__ __forceinline__ void couple_bead_f32(const CoupleArgs &a, int k, int k_rng, int c, int lane,
                                                bool active) {
    const Geom &g = a.g;
    const float *A = static_cast<const float *>(a.f);
    const int body = active ? chk(a.bead_body[chk(k, a.nbeads, a.err)], a.nbodies, a.err) : -1;
    const Body *Bp = active ? &a.bodies[body] : nullptr;

    float rel[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
    if (active && c == 0) {
        const float s0 = a.sf[3 * k], s1 = a.sf[3 * k + 1], s2 = a.sf[3 * k + 2];
        for (int q = 0; q < 3; ++q) rel[q] = Bp->Rf[3 * q] * s0 + Bp->Rf[3 * q + 1] * s1 + Bp->Rf[3 * q + 2] * s2;
        const float *w = Bp->wlf;
        v[0] = Bp->Vf[0] + (w[1] * rel[2] - w[2] * rel[1]);
        v[1] = Bp->Vf[1] + (w[2] * rel[0] - w[0] * rel[2]);
        v[2] = Bp->Vf[2] + (w[0] * rel[1] - w[1] * rel[0]);
    }
    for (int q = 0; q < 3; ++q) rel[q] = __shfl_sync(0xffffffffu, rel[q], 0, 8);

    const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    const int n3[3] = {g.nx, g.ny, g.nz};
    int xyz[3] = {0, 0, 0};
    int ywall = -1;                      // channel: this corner lies beyond the lower (0) or upper (1) wall
    float wt = 1.f;
    if (active) {
        for (int q = 0; q < 3; ++q) {
            const float tq = Bp->Xf[q] + rel[q];          // r - 1/2 - floor(X - 1/2)
            const float fl = floorf(tq);
            const float fr = tq - fl;
            const int raw = Bp->Xi[q] + (int)fl;
            if (q == 1 && g.chan) {
                const int yr = raw + o[1];
                ywall = yr < 0 ? 0 : (yr >= g.ny ? 1 : -1);
            }
            int b0 = raw % n3[q];
            if (b0 < 0) b0 += n3[q];
            xyz[q] = o[q] ? (b0 + 1 == n3[q] ? 0 : b0 + 1) : b0;
            wt *= o[q] ? fr : 1.f - fr;
        }
    }
    const long long n = chk(nidx(g, xyz[0], xyz[1], xyz[2]), g.N, a.err);
    const bool fluid = active && ywall < 0 && !is_wall(g, xyz[0], xyz[1], xyz[2]);
    float ub[3] = {0.f, 0.f, 0.f};
    if (active && ywall >= 0)            // a node beyond a moving wall carries the wall's velocity
        for (int q = 0; q < 3; ++q) ub[q] = wt * (float)g.wchan[38 + 3 * ywall + q];
    if (fluid) {                         // wall nodes carry u = 0
        float rho, j[3];
        node_rho_j<float>(A, g, xyz[0], xyz[1], xyz[2], chk(n, g.N, a.err), a.odd, a.rho0_f, rho, j, a.err);
        const float ir = 1.f / rho;
        const float *Fp = static_cast<const float *>(a.Fprev);
        ub[0] = wt * ((j[0] + 0.5f * (a.gforce_f[0] + Fp[n])) * ir);
        ub[1] = wt * ((j[1] + 0.5f * (a.gforce_f[1] + Fp[g.N + n])) * ir);
        ub[2] = wt * ((j[2] + 0.5f * (a.gforce_f[2] + Fp[2 * g.N + n])) * ir);
    }
    for (int off = 1; off < 8; off <<= 1)
        for (int q = 0; q < 3; ++q) ub[q] += __shfl_xor_sync(0xffffffffu, ub[q], off, 8);

    // Eq. (latticeboltzmannfriction): F_b = -gamma (v - u(r)) + f_s
    float Fb[3] = {0.f, 0.f, 0.f};
    if (active && c == 0) {
        float fs[3] = {0.f, 0.f, 0.f};
        if (a.noise_amp_f > 0.f) {
            const uint32_t step = (uint32_t)(*a.step_base) + a.step_off;
            const uint4 rr = philox4x32_10(make_uint4((uint32_t)k_rng, step, a.instance, a.call), make_uint2(a.key0, a.key1));
            fs[0] = a.noise_amp_f * unit_uniform_f(rr.x);
            fs[1] = a.noise_amp_f * unit_uniform_f(rr.y);
            fs[2] = a.noise_amp_f * unit_uniform_f(rr.z);
        }
        for (int q = 0; q < 3; ++q) Fb[q] = -a.gamma_f * (v[q] - ub[q]) + fs[q];
        for (int q = 0; q < 3; ++q) a.F_bead[3 * k + q] = (double)Fb[q];
    }
    for (int q = 0; q < 3; ++q) Fb[q] = __shfl_sync(0xffffffffu, Fb[q], 0, 8);

    int tile = 0;
    if (fluid) {
        float *Fc = static_cast<float *>(a.Fcur);
        const float wdt = wt * a.dt_f;
        atomicAdd(&Fc[n], -wdt * Fb[0]);
        atomicAdd(&Fc[g.N + n], -wdt * Fb[1]);
        atomicAdd(&Fc[2 * g.N + n], -wdt * Fb[2]);
        tile = chk((int)tile_of(xyz[0], xyz[1], xyz[2], a.ntx, a.nty), a.ntiles, a.err);
    }
    flag_tile(a, fluid, tile, lane);

    // force and torque: FP32 sums over the (up to 4) beads of the warp's first
    // body, FP64 accumulation on the body
    float FT[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (active && c == 0) {
        FT[0] = Fb[0]; FT[1] = Fb[1]; FT[2] = Fb[2];
        FT[3] = rel[1] * Fb[2] - rel[2] * Fb[1];
        FT[4] = rel[2] * Fb[0] - rel[0] * Fb[2];
        FT[5] = rel[0] * Fb[1] - rel[1] * Fb[0];
    }
    const int b_first = __shfl_sync(0xffffffffu, body, 0);
    const bool lead = active && c == 0;
    const bool same = lead && body == b_first;
    float red[6];
    for (int q = 0; q < 6; ++q) red[q] = same ? FT[q] : 0.f;
    for (int q = 0; q < 6; ++q) {
        red[q] += __shfl_xor_sync(0xffffffffu, red[q], 8);
        red[q] += __shfl_xor_sync(0xffffffffu, red[q], 16);
    }
    if (lane == 0 && b_first >= 0)
        for (int q = 0; q < 6; ++q) atomicAdd(&a.bodies[b_first].acc[q], (double)red[q]);
    if (lead && !same)
        for (int q = 0; q < 6; ++q) atomicAdd(&a.bodies[body].acc[q], (double)FT[q]);
}

// Eight lanes per bead, one per surrounding node: lane 0 of the group forms
// the virtual site, every lane interpolates its node's velocity and spreads
// its share of -F_b, the group reduces by shuffles. FP64 storage: node, bead
// and body arithmetic in FP64; FP32 storage: couple_bead_f32.
// k: bead index into a.s / a.bead_body / a.F_bead; k_rng: the bead's index
// within its own lattice (Philox counter word); c: this lane's corner 0-7.
// All 32 lanes of the warp must call it (shuffles), active or not.
template <typename T>
__device__ __forceinline__ void couple_bead(const CoupleArgs &a, int k, int k_rng, int c, int lane, bool active) {
    if constexpr (sizeof(T) == 4) {
        couple_bead_f32(a, k, k_rng, c, lane, active);
        return;
    }
    using R = T;
    const Geom &g = a.g;
    const T *A = static_cast<const T *>(a.f);
    const int body = active ? chk(a.bead_body[chk(k, a.nbeads, a.err)], a.nbodies, a.err) : -1;

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
    // positions in FP64; the weight and the node sums in the storage precision
    R wt = R(1);
    int ywall = -1;                      // channel: this corner lies beyond the lower (0) or upper (1) wall
    for (int q = 0; q < 3; ++q) {
        const double tq = r[q] - 0.5;
        const double fl = floor(tq);
        const R fr = (R)(tq - fl);
        if (q == 1 && g.chan) {
            const int yr = (int)fl + o[1];
            ywall = yr < 0 ? 0 : (yr >= g.ny ? 1 : -1);
        }
        int b0 = (int)fl % n3[q];
        if (b0 < 0) b0 += n3[q];
        xyz[q] = o[q] ? (b0 + 1 == n3[q] ? 0 : b0 + 1) : b0;
        wt *= o[q] ? fr : R(1) - fr;
    }
    const long long n = chk(nidx(g, xyz[0], xyz[1], xyz[2]), g.N, a.err);
    const bool fluid = active && ywall < 0 && !is_wall(g, xyz[0], xyz[1], xyz[2]);
    R ub[3] = {R(0), R(0), R(0)};
    if (active && ywall >= 0)            // a node beyond a moving wall carries the wall's velocity
        for (int q = 0; q < 3; ++q) ub[q] = wt * (R)g.wchan[38 + 3 * ywall + q];
    if (fluid) {                         // wall nodes carry u = 0
        R rho, j[3];
        node_rho_j<R>(A, g, xyz[0], xyz[1], xyz[2], chk(n, g.N, a.err), a.odd, (R)a.rho0, rho, j, a.err);
        const R ir = R(1) / rho;
        const T *Fp = static_cast<const T *>(a.Fprev);
        R gx, gy, gz;
        if constexpr (sizeof(R) == 4) { gx = a.gforce_f[0]; gy = a.gforce_f[1]; gz = a.gforce_f[2]; }
        else { gx = a.gforce[0]; gy = a.gforce[1]; gz = a.gforce[2]; }
        const R ux = (j[0] + R(0.5) * (gx + Fp[n])) * ir;
        const R uy = (j[1] + R(0.5) * (gy + Fp[g.N + n])) * ir;
        const R uz = (j[2] + R(0.5) * (gz + Fp[2 * g.N + n])) * ir;
        ub[0] = wt * ux;
        ub[1] = wt * uy;
        ub[2] = wt * uz;
    }
    for (int off = 1; off < 8; off <<= 1)
        for (int q = 0; q < 3; ++q) ub[q] += __shfl_xor_sync(0xffffffffu, ub[q], off, 8);

    // Eq. (latticeboltzmannfriction): F_b = -gamma (v - u(r)) + f_s
    double Fb[3] = {0.0, 0.0, 0.0};
    if (active && c == 0) {
        double fs[3] = {0.0, 0.0, 0.0};
        if (a.noise_amp > 0.0) {
            const uint32_t step = (uint32_t)(*a.step_base) + a.step_off;
            const uint4 rr = philox4x32_10(make_uint4((uint32_t)k_rng, step, a.instance, a.call), make_uint2(a.key0, a.key1));
            fs[0] = a.noise_amp * unit_uniform_d(rr.x);
            fs[1] = a.noise_amp * unit_uniform_d(rr.y);
            fs[2] = a.noise_amp * unit_uniform_d(rr.z);
        }
        for (int q = 0; q < 3; ++q) Fb[q] = -a.gamma * (v[q] - (double)ub[q]) + fs[q];
        for (int q = 0; q < 3; ++q) a.F_bead[3 * k + q] = Fb[q];
    }
    for (int q = 0; q < 3; ++q) Fb[q] = __shfl_sync(0xffffffffu, Fb[q], 0, 8);

    // spread -w F_b onto this lane's node; a wall node takes nothing
    int tile = 0;
    if (fluid) {
        T *Fc = static_cast<T *>(a.Fcur);
        atomicAdd(&Fc[n], -wt * (T)(a.dt * Fb[0]));
        atomicAdd(&Fc[g.N + n], -wt * (T)(a.dt * Fb[1]));
        atomicAdd(&Fc[2 * g.N + n], -wt * (T)(a.dt * Fb[2]));
        tile = chk((int)tile_of(xyz[0], xyz[1], xyz[2], a.ntx, a.nty), a.ntiles, a.err);
    }
    flag_tile(a, fluid, tile, lane);

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


}  // namespace lbk
