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

__global__ void k_kick2(Body *bodies, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) kick2(bodies[b]);
}

template <typename T>
__global__ void __launch_bounds__(128) k_couple(const CoupleArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t >> 3;
    couple_bead<T>(a, k, k, t & 7, threadIdx.x & 31, k < a.nbeads);
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
