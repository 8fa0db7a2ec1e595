// Raspberry kernels (Ustach & Faller, arXiv:1604.01829):
//  - rigid-body integration of the centre of mass by velocity Verlet and of
//    the orientation by a quaternion (Sec. 2.3), one thread per body in FP64;
//  - virtual sites r_b = X + R(q) s_b, v_b = V + omega x (r_b - X) (Sec. 1.2);
//  - friction coupling F_b = -gamma (v_b - u(r_b)) + f_s, Eq.
//    (latticeboltzmannfriction) in Sec. 1.1, with u trilinearly interpolated
//    from the 8 surrounding nodes and -F_b spread back onto the same nodes
//    with the same weights, so the exchange conserves momentum; bead forces
//    and torques summed onto the body (Sec. 2.3).
#include "lb_couple.cuh"

namespace lbk {

namespace {

// Step prologue in one launch: thread 0 of blocks [0, nb) finishes the
// previous step's body (second half kick) if asked and starts this step's
// (half kick, drift, rotation); every thread also clears nodes of the
// flagged 4x4x4 tiles of this step's spread-force buffer.
template <typename T>
__global__ void k_step_pre(Body *bodies, int nb, int finish_prev, T *F, int *tiles, const int *tlist,
                           const int *tcount, Geom g, int ntx, int nty, Recorder rec, double dt, const double *ext) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // one body per block, so the FP64 work of the bodies spreads over SMs;
    // a private copy means one read and one write of the record
    if (threadIdx.x == 0 && blockIdx.x < nb) {
        Body B = bodies[blockIdx.x];
        if (finish_prev) kick2(B, dt);
        if (ext) {                     // this step's external force and torque (host-written, mapped)
            const int b = blockIdx.x;
            for (int a = 0; a < 3; ++a) {
                B.F_ext[a] = ext[3 * b + a];
                B.T_ext[a] = ext[3 * nb + 3 * b + a];
            }
        }
        kick_drift(B, dt);
        bodies[blockIdx.x] = B;
        record_body(rec, B, blockIdx.x, nb);
    }
    if (!tiles) return;
    // one thread per (listed tile, node of the tile): zero the force, drop the flag
    const long long total = 64LL * (*tcount);
    for (long long i = t; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int tile = tlist[i >> 6];
        const int l = (int)(i & 63);
        const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
        const int x = 4 * tx + (l & 3), y = 4 * ty + ((l >> 2) & 3), z = 4 * tz + (l >> 4);
        if (x < g.nx && y < g.ny && z < g.nz) {
            const long long n = nidx(g, x, y, z);
            F[n] = T(0);
            F[g.N + n] = T(0);
            F[2 * g.N + n] = T(0);
        }
        if (l == 0) tiles[tile] = 0;
    }
}

// The end of a group of steps in one launch: the last step's second half
// kick (one body per block) and the advance of the device step counter;
// with `out` (host-mapped) also every body's force and torque totals and the
// device error word, so the host reads them without a copy.
__global__ void k_finish(Body *bodies, int nb, double dt, unsigned long long *step, unsigned int by, double *out,
                         const int *err) {
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    if (b < nb) {
        Body B = bodies[b];
        kick2(B, dt);
        bodies[b] = B;
        if (out)
            for (int a = 0; a < 3; ++a) {
                out[6 * b + a] = B.F_tot[a];
                out[6 * b + 3 + a] = B.T_tot[a];
            }
    }
    if (b == 0) {
        *step += by;
        if (out) out[6 * nb] = err ? (double)*err : 0.0;
    }
}

// Between two MD substeps of one LB step: the finished substep's second half
// kick, the next substep's first half kick and drift (and the trajectory
// record after the last substep's drift).
__global__ void k_substep(Body *bodies, int nb, double dt, Recorder rec) {
    const int b = blockIdx.x;
    if (threadIdx.x == 0 && b < nb) {
        Body B = bodies[b];
        kick2(B, dt);
        kick_drift(B, dt);
        bodies[b] = B;
        record_body(rec, B, b, nb);
    }
}

__global__ void k_wall_beads(const WallBeads w, Body *bodies, const double *s, const int *bead_body, int nbeads) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nbeads) wall_bead_body(w, bodies, s, bead_body, k);
}

// threads per block of the body prologue when it runs beside a fluid kernel
#ifndef LB_PRE_BLOCK
#define LB_PRE_BLOCK 256
#endif

// register cap of the FP32 coupling kernel (resident CTAs of 128 per SM:
// 65536 / (128 x cap))
#ifndef LB_COUPLE_REGS
#define LB_COUPLE_REGS 64
#endif
template <typename T>
__global__ void __launch_bounds__(128) __maxnreg__(sizeof(T) == 4 ? LB_COUPLE_REGS : 255) k_couple(const CoupleArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t >> 3;
    couple_bead<T>(a, k, k, t & 7, threadIdx.x & 31, k < a.nbeads);
}

}  // namespace

cudaError_t launch_step_pre(Body *b, int nbodies, bool finish_prev, void *F, bool fp32, int *tiles, const int *tlist,
                            const int *tcount, int list_cap, const Geom &g, int ntx, int nty, const Recorder &rec,
                            cudaStream_t s, double dt, const double *ext, bool alone) {
    // one block per body, and for the tile clearing (grid-stride) at most a
    // quarter of the SMs' worth of blocks when the kernel runs beside the
    // fluid kernel of the previous step, whose blocks it would otherwise
    // displace (measured on GB300 at 256^3 with 64 bodies: fluid kernel
    // 0.4372 ms against 0.4392 with a full-GPU grid, the step 0.4620 against
    // 0.4641); 8 blocks per SM when nothing runs beside it (the first step of
    // a group, e.g. every step of a one-step-per-call control loop)
    static const int sms = [] {     // initialised once, thread-safe
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || n <= 0)
            n = 152;
        return n;
    }();
    long long n = 64LL * list_cap;
    const int bs = alone ? 256 : LB_PRE_BLOCK;
    const long long cap = (alone ? 8LL * sms : (long long)(sms + 3) / 4) * bs;
    if (n > cap) n = cap;
    unsigned grid = (unsigned)((n + bs - 1) / bs);
    if (grid < (unsigned)nbodies) grid = (unsigned)nbodies;
    if (fp32) k_step_pre<float><<<grid, bs, 0, s>>>(b, nbodies, finish_prev ? 1 : 0, (float *)F, tiles, tlist, tcount, g, ntx, nty, rec, dt, ext);
    else k_step_pre<double><<<grid, bs, 0, s>>>(b, nbodies, finish_prev ? 1 : 0, (double *)F, tiles, tlist, tcount, g, ntx, nty, rec, dt, ext);
    return cudaGetLastError();
}

cudaError_t launch_couple(const CoupleArgs &a, cudaStream_t s) {
    if (a.nbeads <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((8LL * a.nbeads + 127) / 128);
    if (a.fp32) k_couple<float><<<grid, 128, 0, s>>>(a);
    else k_couple<double><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wall_beads(const WallBeads &w, Body *b, const double *s, const int *bead_body, int nbeads,
                              cudaStream_t st) {
    if (!w.on || nbeads <= 0) return cudaSuccess;
    k_wall_beads<<<(nbeads + 127) / 128, 128, 0, st>>>(w, b, s, bead_body, nbeads);
    return cudaGetLastError();
}

cudaError_t launch_finish(Body *b, int nbodies, double dt, unsigned long long *step, unsigned int by, cudaStream_t s,
                          double *out, const int *err) {
    k_finish<<<nbodies > 0 ? nbodies : 1, 32, 0, s>>>(b, nbodies > 0 ? nbodies : 0, dt, step, by, out, err);
    return cudaGetLastError();
}

cudaError_t launch_substep(Body *b, int nbodies, double dt, const Recorder &rec, cudaStream_t s) {
    if (nbodies <= 0) return cudaSuccess;
    k_substep<<<nbodies, 32, 0, s>>>(b, nbodies, dt, rec);
    return cudaGetLastError();
}

}  // namespace lbk
