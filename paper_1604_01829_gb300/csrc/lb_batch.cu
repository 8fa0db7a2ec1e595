// Batched lattices: many independent LB + raspberry instances of uneven size
// advanced together (one launch per kernel per step for all instances; the
// step sequence replayed from a CUDA graph).
//
// Each instance is the same step as a single lattice (Sec. 1.1 collision
// and streaming, Eq. (latticeboltzmannfriction) coupling, Sec. 2.3 bodies
// and pore walls of Ustach & Faller, arXiv:1604.01829); only the
// scheduling differs. All populations live in one pool (instance k at
// element offset off_k, its own plane stride N_k); the fluid kernel walks a
// flattened list of equal work tiles (TS consecutive nodes of one instance)
// with a persistent grid or one CTA per tile, so uneven instances
// load-balance by construction. Tile size, blocks per SM and the tile-to-CTA
// order are chosen by a measuring autotuner on a snapshot of the state,
// restored afterwards.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_collide.cuh"
#include "lb_couple.cuh"

// register caps of the FP32 fluid kernel per parity (resident CTAs of 128
// threads per SM: 65536 / (128 x cap), rounded down)
#ifndef LB_BATCH_REGS_EVEN
#define LB_BATCH_REGS_EVEN 64
#endif
#ifndef LB_BATCH_REGS_ODD
#define LB_BATCH_REGS_ODD 64
#endif

namespace lbk {

struct BInst {
    Geom g;
    uint32_t mx, my;             // ceil(2^32 / nx), ceil(2^32 / ny) for exact quotients (fastdiv)
    int fastdiv;                 // 1 when n * nx and (n / nx) * ny stay below 2^32 for every node
    long long off;               // element offset of plane 0 in the population pool
    long long ps;                // population plane stride (elements): the node count rounded up
                                 // to 32 (dense), or the fluid node count rounded up to 32 (compact
                                 // pore layout), so that every plane starts on a 128-byte line
    long long fs;                // force-pool plane stride: the node count rounded up to 32
    int cmode;                   // 1: compact pore layout (g.cmap, g.cnbr), from the first upload on
    long long foff;              // offset of this instance's [3][N] block in a force pool
    long long toff;              // offset of its tile flags
    // work items of the fluid kernel: all N nodes of a periodic instance; the
    // fluid nodes only of a pore instance, as (position across the axis j,
    // coordinate along it a): node = fluid[loff + j] + a * astride, with j
    // fastest (a fastest for an x-axis pore, so that x stays contiguous)
    long long loff;              // offset in the fluid-position pool, -1: no compaction
    uint32_t nwork;              // work items
    uint32_t ncs, nax, astride;  // fluid positions across the axis, nodes along it, node stride along it
    uint32_t mw;                 // ceil(2^32 / divisor) for exact quotients when wfast
    int wfast;
    int ntx, nty, ntz;
    uint32_t key0, key1, instance;
    double rho0, gamma, noise_amp;
    float gamma_f, noise_amp_f;
    float noise_amp_sub_f;       // noise_amp x sqrt(MD substeps), rounded to FP32 (FP32 coupling)
    double pore_R;
    WallBeads wall;              // pore-wall beads
    double gd[3];                // uniform force density
    float gf[3];
    CollParams<double> pd;
    CollParams<float> pf;
};

struct BatchArgs {
    const BInst *inst;
    const int *tile_start;       // n + 1: first work tile of each instance
    const int *tile_inst;        // instance of each work tile
    int n, ntiles, chunk, order;
    CollParams<double> pd;       // collision constants shared by all instances (COMMON kernels)
    CollParams<float> pf;
    void *pool;
    const void *F;               // spread force of this step (pool, storage precision), nullptr without bodies
    const int *tiles;
    const uint32_t *fluid;       // fluid positions across the axis of the pore instances (BInst::loff)
    const unsigned long long *step_base;
    uint32_t step_off;
    // index checks of checked builds (-DLB_CHECKS): the error word and the
    // extents of the shared tables (other builds compile the checks out)
    int *err;
    long long nfluid, ttot;
};

namespace {

// Odd-step loads and stores of one fluid node of a compact pore instance,
// with the pore axis AX known at compile time so that each link's in-plane
// direction and shift along the axis are constants: the node's 8 in-plane
// neighbours come in one 16-byte load (rec), then per link one compare and
// one address. m = the node's compact index, j its position across the axis,
// l its coordinate along the axis (nl nodes), sj / sa the compact strides of
// the position across and along the axis.
__device__ __forceinline__ int nbr_of(const uint4 &rec, int d) {
    const uint32_t w = d < 2 ? rec.x : (d < 4 ? rec.y : (d < 6 ? rec.z : rec.w));
    return (int)((d & 1) ? (w >> 16) : (w & 0xFFFFu));
}

template <int AX>
__device__ __forceinline__ void axis_parts(int i, int &u, int &v, int &al) {
    if (AX == 2) { u = cx(i); v = cy(i); al = cz(i); }
    else if (AX == 1) { u = cx(i); v = cz(i); al = cy(i); }
    else { u = cy(i); v = cz(i); al = cx(i); }
}

template <int AX, typename T, typename R>
__device__ __forceinline__ void compact_odd_load(const T *P, uint32_t base, uint32_t N, const uint4 &rec,
                                                 uint32_t j, uint32_t l, uint32_t nl, uint32_t sj, uint32_t sa,
                                                 uint32_t m, R (&f)[19], int *err) {
    // along-axis part of the upstream node x - c_i for c_i's component -1, 0, +1
    const uint32_t o[3] = {(l + 1 == nl ? 0 : l + 1) * sa, l * sa, (l == 0 ? nl - 1 : l - 1) * sa};
    f[0] = P[base + chk(m, N, err)];
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        int u, v, al;
        axis_parts<AX>(i, u, v, al);
        const int js = (u == 0 && v == 0) ? (int)j : nbr_of(rec, dir8(-u, -v));
        const uint32_t idx = js == 0xFFFF ? (uint32_t)i * N + m : (uint32_t)opp(i) * N + (uint32_t)js * sj + o[al + 1];
        f[i] = P[base + chk(idx, 19LL * N, err)];
    }
}

template <int AX, typename T, typename R>
__device__ __forceinline__ void compact_odd_store(T *P, uint32_t base, uint32_t N, const uint4 &rec,
                                                  uint32_t j, uint32_t l, uint32_t nl, uint32_t sj, uint32_t sa,
                                                  uint32_t m, const R (&f)[19], int *err) {
    // along-axis part of the downstream node x + c_i for c_i's component -1, 0, +1
    const uint32_t o[3] = {(l == 0 ? nl - 1 : l - 1) * sa, l * sa, (l + 1 == nl ? 0 : l + 1) * sa};
    P[base + chk(m, N, err)] = f[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        int u, v, al;
        axis_parts<AX>(i, u, v, al);
        const int jd = (u == 0 && v == 0) ? (int)j : nbr_of(rec, dir8(u, v));
        // a wall downstream returns the population into this node's opposite slot
        const uint32_t idx = jd == 0xFFFF ? (uint32_t)opp(i) * N + m : (uint32_t)i * N + (uint32_t)jd * sj + o[al + 1];
        P[base + chk(idx, 19LL * N, err)] = f[i];
    }
}

template <typename T, int COLL, bool NOISE, bool ODD, bool COMMON>
__global__ void __maxnreg__(sizeof(T) == 4 ? (ODD ? LB_BATCH_REGS_ODD : LB_BATCH_REGS_EVEN) : 255)
    k_batch_collide(const BatchArgs a) {
    using R = T;
    constexpr bool DEV = sizeof(T) == 4;
    for (int it = 0;; ++it) {
        int t;
        if (a.order == 0) t = blockIdx.x + it * gridDim.x;
        else {
            if (it >= a.chunk) break;
            t = blockIdx.x * a.chunk + it;
        }
        if (t >= a.ntiles) break;
        const int k = chk(__ldg(a.tile_inst + t), a.n, a.err);
        const BInst &I = a.inst[k];
        const Geom g = I.g;
        const uint32_t N = (uint32_t)I.ps;          // population plane stride
        const uint32_t w = (uint32_t)(t - __ldg(a.tile_start + k)) * blockDim.x + threadIdx.x;
        if (w >= I.nwork) continue;
        // a pore instance stores its fluid nodes only (compact layout): work
        // item w is compact node w, at position j across the axis and l along
        // it; n is the node's index in the dense numbering (coordinates,
        // forces, noise counter)
        const bool compact = I.cmode != 0;
        uint32_t n = w, j = 0, l = 0;
        if (compact) {
            const uint32_t d = g.pore_axis == 0 ? I.nax : I.ncs;
            const uint32_t q = I.wfast ? __umulhi(w, I.mw) : w / d;
            const uint32_t rm = w - q * d;
            j = g.pore_axis == 0 ? q : rm;
            l = g.pore_axis == 0 ? rm : q;
            n = __ldg(a.fluid + chk(I.loff + j, a.nfluid, a.err)) + l * I.astride;
        }
        uint32_t r, z;
        if (I.fastdiv) {
            r = __umulhi(n, I.mx);
            z = __umulhi(r, I.my);
        } else {
            r = n / (uint32_t)g.nx;
            z = r / (uint32_t)g.ny;
        }
        const int x = (int)(n - r * (uint32_t)g.nx), y = (int)(r - z * (uint32_t)g.ny);
        // 32-bit element indices into the pool (the pool holds < 2^32 elements)
        T *P = static_cast<T *>(a.pool);
        const uint32_t base = (uint32_t)I.off;
        const int nxy = g.nx * g.ny;
        const int xo[3] = {x == 0 ? g.nx - 1 : x - 1, x, x == g.nx - 1 ? 0 : x + 1};
        const int yo[3] = {(y == 0 ? g.ny - 1 : y - 1) * g.nx, y * g.nx, (y == g.ny - 1 ? 0 : y + 1) * g.nx};
        const int zo[3] = {((int)z == 0 ? g.nz - 1 : (int)z - 1) * nxy, (int)z * nxy,
                           ((int)z == g.nz - 1 ? 0 : (int)z + 1) * nxy};
        auto at = [&](int i, uint32_t node) -> T & { return P[base + (uint32_t)i * N + chk(node, N, a.err)]; };
        R f[19];
        if (!ODD) {
            const uint32_t m = compact ? w : n;
#pragma unroll
            for (int i = 0; i < 19; ++i) f[i] = at(i, m);
        } else if (!compact) {
            f[0] = at(0, n);
#pragma unroll
            for (int i = 1; i < 19; ++i) f[i] = at(opp(i), (uint32_t)(xo[1 - cx(i)] + yo[1 - cy(i)] + zo[1 - cz(i)]));
        } else {
            // the upstream node x - c_i: its compact position from the
            // neighbour table, -1 for a wall node (the population bounced back)
            const uint4 rec = __ldg(reinterpret_cast<const uint4 *>(g.cnbr) + chk(j, (long long)I.ncs, a.err));
            const uint32_t nl = I.nax, sj = (uint32_t)g.csj, sa = (uint32_t)g.csa;
            if (g.pore_axis == 2) compact_odd_load<2>(P, base, N, rec, j, l, nl, sj, sa, w, f, a.err);
            else if (g.pore_axis == 1) compact_odd_load<1>(P, base, N, rec, j, l, nl, sj, sa, w, f, a.err);
            else compact_odd_load<0>(P, base, N, rec, j, l, nl, sj, sa, w, f, a.err);
        }
        R Fx, Fy, Fz;
        if constexpr (DEV) { Fx = I.gf[0]; Fy = I.gf[1]; Fz = I.gf[2]; }
        else { Fx = I.gd[0]; Fy = I.gd[1]; Fz = I.gd[2]; }
        if (a.tiles && a.tiles[chk(I.toff + tile_of(x, y, (int)z, I.ntx, I.nty), a.ttot, a.err)]) {
            const T *Fn = static_cast<const T *>(a.F) + I.foff;
            const size_t FS = (size_t)I.fs;
            Fx += Fn[chk((long long)n, (long long)FS, a.err)];
            Fy += Fn[FS + n];
            Fz += Fn[2 * FS + n];
        }
        uint32_t step = 0;
        if (NOISE) step = (uint32_t)(*a.step_base) + a.step_off;
        const uint2 key = make_uint2(I.key0, I.key1);
        if constexpr (DEV) collide<R, true, COLL, NOISE>(f, Fx, Fy, Fz, COMMON ? a.pf : I.pf, key, I.instance, n, step);
        else collide<R, false, COLL, NOISE>(f, Fx, Fy, Fz, COMMON ? a.pd : I.pd, key, I.instance, n, step);
        // re-read the plane layout for the stores instead of keeping 19 plane
        // offsets live across the collision (register pressure)
        const uint32_t base2 = *(const volatile uint32_t *)&a.inst[k].off;
        const uint32_t N2 = *(const volatile uint32_t *)&a.inst[k].ps;
        auto at2 = [&](int i, uint32_t node) -> T & { return P[base2 + (uint32_t)i * N2 + chk(node, N2, a.err)]; };
        if (!ODD) {
            const uint32_t m = compact ? w : n;
#pragma unroll
            for (int i = 0; i < 19; ++i) at2(opp(i), m) = f[i];
        } else if (!compact) {
            at2(0, n) = f[0];
#pragma unroll
            for (int i = 1; i < 19; ++i) at2(i, (uint32_t)(xo[1 + cx(i)] + yo[1 + cy(i)] + zo[1 + cz(i)])) = f[i];
        } else {
            // the downstream node x + c_i; a wall there returns the population
            // into this node's opposite slot (halfway bounce-back)
            const int axis2 = *(const volatile int *)&a.inst[k].g.pore_axis;
            const uint16_t *cnb = *(const uint16_t *const volatile *)&a.inst[k].g.cnbr;
            const uint32_t nl = *(const volatile uint32_t *)&a.inst[k].nax;
            const uint4 rec = __ldg(reinterpret_cast<const uint4 *>(cnb) + chk(j, (long long)a.inst[k].ncs, a.err));
            const uint32_t sj = (uint32_t)*(const volatile int *)&a.inst[k].g.csj;
            const uint32_t sa = (uint32_t)*(const volatile int *)&a.inst[k].g.csa;
            if (axis2 == 2) compact_odd_store<2>(P, base2, N2, rec, j, l, nl, sj, sa, w, f, a.err);
            else if (axis2 == 1) compact_odd_store<1>(P, base2, N2, rec, j, l, nl, sj, sa, w, f, a.err);
            else compact_odd_store<0>(P, base2, N2, rec, j, l, nl, sj, sa, w, f, a.err);
        }
    }
}

struct BatchCouple {
    const BInst *inst;
    const void *pool;
    bool fp32, odd;
    const void *Fprev;
    void *Fcur;
    int *tiles_cur;
    int *tlist;
    int *tcount;
    const double *s;
    const float *sf;
    const int *bead_body;
    const int *bead_rng;          // bead index within its own lattice
    const int *bead_inst;         // instance of each bead
    int ninst;
    Body *bodies;
    double *F_bead;
    int nbeads;
    const unsigned long long *step_base;
    uint32_t step_off;
    int *err;                     // index checks of checked builds, as BatchArgs
    int list_cap, nbodies;
    double dt, noise_scale;       // MD substep length 1/n; bead noise amplitude factor sqrt(n)
    float dt_f;                  // dt rounded to FP32
    uint32_t call;                // Philox call word of the bead noise: 4 + substep
};

// 1: lb_batch_step launches every step eagerly instead of replaying the
// captured two-step graph
#ifndef LB_BATCH_EAGER
#define LB_BATCH_EAGER 0
#endif

#ifndef LB_BATCH_COUPLE_REGS
#define LB_BATCH_COUPLE_REGS 64
#endif
template <typename T>
__global__ void __maxnreg__(sizeof(T) == 4 ? LB_BATCH_COUPLE_REGS : 255) k_batch_couple(const BatchCouple b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t >> 3;
    const bool active = k < b.nbeads;
    // lanes of inactive groups borrow bead 0's instance (they do no work)
    const int kk = active ? k : 0;
    const BInst &I = b.inst[chk(b.bead_inst[kk], b.ninst, b.err)];
    CoupleArgs a{};
    a.g = I.g;
    a.g.N = I.fs;                 // force planes (and dense population planes): the padded node count
    a.f = static_cast<const T *>(b.pool) + I.off;
    a.fp32 = b.fp32;
    a.odd = b.odd;
    // the FP32 coupling reads the FP32 copies only (no FP64 work per thread)
    if constexpr (sizeof(T) == 8) {
        a.rho0 = I.rho0;
        a.gamma = I.gamma;
        a.noise_amp = I.noise_amp * b.noise_scale;
        a.dt = b.dt;
    }
    a.rho0_f = I.pf.rho0;
    a.gforce = I.gd;
    a.gforce_f = I.gf;
    a.Fprev = static_cast<const T *>(b.Fprev) + I.foff;
    a.Fcur = static_cast<T *>(b.Fcur) + I.foff;
    a.tiles_cur = b.tiles_cur + I.toff;
    a.tlist = b.tlist;
    a.tcount = b.tcount;
    a.tile_base = (int)I.toff;
    a.ntx = I.ntx;
    a.nty = I.nty;
    a.s = b.s;
    a.sf = b.sf;
    a.gamma_f = I.gamma_f;
    a.noise_amp_f = I.noise_amp_sub_f;
    a.bead_body = b.bead_body;
    a.bodies = b.bodies;
    a.F_bead = b.F_bead;
    a.nbeads = b.nbeads;
    a.err = b.err;
    a.ntiles = (long long)I.ntx * I.nty * I.ntz;
    a.list_cap = b.list_cap;
    a.nbodies = b.nbodies;
    a.dt_f = b.dt_f;
    a.call = b.call;
    a.key0 = I.key0;
    a.key1 = I.key1;
    a.instance = I.instance;
    a.step_base = b.step_base;
    a.step_off = b.step_off;
    couple_bead<T>(a, k, active ? b.bead_rng[k] : 0, t & 7, threadIdx.x & 31, active);
}

// pore-wall beads of each bead's instance (one thread per bead)
__global__ void k_batch_wall(const BInst *inst, Body *bodies, const double *s, const int *bead_body, int nbeads,
                             int nbodies, int *err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nbeads) return;
    const BInst &I = inst[bodies[chk(bead_body[k], nbodies, err)].inst];
    if (!I.wall.on) return;
    const WallBeads w = I.wall;
    wall_bead_body(w, bodies, s, bead_body, k);
}

// previous step's second half kick (optional), this step's kick and drift,
// and the clearing of every flagged tile of this step's force pool
template <typename T>
__global__ void k_batch_pre(Body *bodies, int nb, int finish_prev, T *F, int *tiles, const int *tlist,
                            const int *tcount, const BInst *inst, const long long *flag_start, int n,
                            Recorder rec, int list_cap, long long ttot, int *err, double dt) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (threadIdx.x == 0 && blockIdx.x < nb) {     // one body per block
        Body B = bodies[blockIdx.x];
        if (finish_prev) kick2(B, dt);
        kick_drift(B, dt);
        bodies[blockIdx.x] = B;
        record_body(rec, B, blockIdx.x, nb);
    }
    if (!tiles) return;
    // one thread per (listed tile, node of the tile)
    const long long total = 64LL * (*tcount);
    for (long long i = t; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long gt = chk((long long)tlist[chk(i >> 6, list_cap, err)], ttot, err);
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (flag_start[mid] <= gt) lo = mid; else hi = mid;
        }
        const BInst &I = inst[lo];
        const int lt = (int)(gt - flag_start[lo]);
        const int l = (int)(i & 63);
        const int tx = lt % I.ntx, ty = (lt / I.ntx) % I.nty, tz = lt / (I.ntx * I.nty);
        const int x = 4 * tx + (l & 3), y = 4 * ty + ((l >> 2) & 3), z = 4 * tz + (l >> 4);
        if (x < I.g.nx && y < I.g.ny && z < I.g.nz) {
            T *Fi = F + I.foff;
            const long long nn = nidx(I.g, x, y, z);
            Fi[nn] = T(0);
            Fi[I.fs + nn] = T(0);
            Fi[2 * I.fs + nn] = T(0);
        }
        if (l == 0) tiles[gt] = 0;
    }
}

template <typename T>
__global__ void k_batch_gather(const T *A, Geom g, long long Nn, bool odd, double rho0, double *out) {
    // g.N is the plane stride of the pool, Nn the node count (the output's plane length)
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= Nn) return;
    const int x = (int)(n % g.nx);
    const long long r = n / g.nx;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    // wall nodes hold no populations (compact layout) or stale ones: they
    // read as fluid at rest
    const bool wall = is_wall(g, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const T v = wall ? (sizeof(T) == 4 ? T(0) : T(wq(i) * rho0))
                         : (g.cmap ? compact_load_pre(A, g, x, y, z, i, odd) : load_pre(A, g, x, y, z, n, i, odd));
        out[(long long)i * Nn + n] = sizeof(T) == 4 ? (double)v + wq(i) * rho0 : (double)v;
    }
}

template <typename T>
__global__ void k_batch_scatter(T *A, Geom g, long long Nn, bool odd, double rho0, const double *in) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= Nn) return;
    const int x = (int)(n % g.nx);
    const long long r = n / g.nx;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    if (is_wall(g, x, y, z)) return;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const double v = in[(long long)i * Nn + n];
        const T tv = sizeof(T) == 4 ? (T)(v - wq(i) * rho0) : (T)v;
        if (g.cmap) compact_store_pre(A, g, x, y, z, i, odd, tv);
        else store_pre(A, g, x, y, z, n, i, odd, tv);
    }
}

template <typename T>
__global__ void k_batch_init(T *A, long long N, double rho0) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
#pragma unroll
    for (int i = 0; i < 19; ++i) A[(long long)i * N + n] = sizeof(T) == 4 ? T(0) : T(wq(i) * rho0);
}

}  // namespace
}  // namespace lbk

using lbk::BInst;
using lbk::Body;

struct lb_batch_ctx {
    std::vector<lb_params> p;
    int n = 0;
    bool fp32 = false;
    int collision = 0;
    bool noise = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the prologue of step k + 1 runs on this stream beside the fluid kernel
    // of step k (see launch_step)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<BInst> hinst;
    std::vector<long long> flag_start;      // n + 1
    std::vector<long long> nfluid;
    long long Ntot = 0, Ttot = 0, Ftot = 0;  // padded plane strides summed (pool sizes)
    long long Nnodes = 0;                    // nodes of all instances
    void *pool = nullptr;
    void *Fbuf[2] = {nullptr, nullptr};     // force pools, storage precision
    int *tiles[2] = {nullptr, nullptr};
    int *tlist[2] = {nullptr, nullptr};
    int *tcount[2] = {nullptr, nullptr};
    int list_cap = 0;
    BInst *dinst = nullptr;
    int *dtile_start = nullptr;
    int *dtile_inst = nullptr;
    size_t tile_inst_cap = 0;
    bool common = false;                    // all instances share their collision constants
    long long *dflag_start = nullptr;
    unsigned long long *step_dev = nullptr;
    long long step = 0;
    // bodies
    std::vector<Body> hb;
    std::vector<double> hs;
    std::vector<int> hbody_of, hbead_rng, hbead_inst;
    std::vector<std::vector<int>> inst_bodies;     // body ids per instance
    std::vector<int> inst_beads;                   // beads per instance so far
    Body *db = nullptr;
    double *ds = nullptr;
    float *dsf = nullptr;
    std::vector<float> hsf;
    int *dbody_of = nullptr, *dbead_rng = nullptr;
    int *dbead_inst = nullptr;              // instance of each bead (the coupling's first lookup)
    double *dFbead = nullptr;
    bool uploaded = false;
    // schedule
    int TS = 128, bpsm = 8, order = 0, ntiles = 0, sms = 0;
    int resident[2] = {0, 0};               // resident CTAs per SM of the even / odd fluid kernel at TS threads
    // graph of two steps
    cudaGraphExec_t gexec = nullptr;
    bool any_wall = false;                  // some instance has pore-wall beads
    // fluid positions (BInst::loff) of the pore instances and their compact
    // layout's position map and neighbour table (Geom::cmap, Geom::cnbr)
    int *dcmap = nullptr;
    uint16_t *dcnbr = nullptr;
    uint32_t *dfluid = nullptr;
    // trajectory recorder ([rec_cap][nbodies][7], records k >= rec_k0)
    double *rec = nullptr;
    int rec_every = 0, rec_cap = 0;
    long long rec_k0 = 0;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double timed_ms = 0.0;
    long long timed_n = 0;
    size_t dev_bytes = 0;
    std::string err;
    // device error word of the index checks (checked builds) and its pinned
    // host copy; extents of the wall-mask and fluid-position tables
    int *derr = nullptr;
    int *herr = nullptr;
    int nsub = 1;                           // MD substeps per LB step (shared by the instances)
    long long nfluidpos = 0;
};

namespace {

thread_local std::string g_batch_error;

lb_status bfail(lb_batch_ctx *h, lb_status s, const std::string &m) {
    if (h) h->err = m;
    else g_batch_error = m;
    return s;
}

#define BCUDA(h, call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return bfail((h), LB_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

template <typename P>
lb_status balloc(lb_batch_ctx *h, P **ptr, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)ptr, bytes < 16 ? 16 : bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return bfail(h, LB_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    h->dev_bytes += bytes;
    return LB_OK;
}

void fill_coll(const lb_params &p, BInst &I) {
    static const double bk[19] = {1.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9,
                                  1.0 / 9, 2.0 / 3, 2.0 / 3, 2.0 / 3, 2.0 / 9, 2.0 / 9, 2.0 / 9, 2.0, 4.0 / 3,
                                  4.0 / 9};
    auto rate = [&](int k) {
        return k == 4 ? p.gamma_bulk : (k <= 9 ? p.gamma_shear : (k <= 15 ? p.gamma_odd : p.gamma_even));
    };
    I.pd.rho0 = p.rho0;
    I.pd.omega = 1.0 / p.tau;
    for (int k = 4; k <= 9; ++k) {
        const double c = (1.0 / 36.0) / bk[k], g = rate(k);
        I.pd.ke[k - 4] = c * (1.0 - g);
        I.pd.km[k - 4] = c * g;
        I.pd.ks[k - 4] = c * 0.5 * (1.0 + g);
    }
    for (int k = 10; k <= 18; ++k) I.pd.kg[k - 10] = (1.0 / 36.0) / bk[k] * rate(k);
    for (int k = 4; k <= 18; ++k) {
        const double g = rate(k);
        const double sig = (p.collision == 1 && p.kT > 0.0) ? std::sqrt(3.0 * p.kT * bk[k] * (1.0 - g * g)) : 0.0;
        I.pd.kn[k - 4] = (1.0 / 36.0) / bk[k] * sig * 3.4641016151377544;
    }
    I.pf.rho0 = (float)I.pd.rho0;
    I.pf.omega = (float)I.pd.omega;
    for (int k = 0; k < 6; ++k) {
        I.pf.ke[k] = (float)I.pd.ke[k];
        I.pf.km[k] = (float)I.pd.km[k];
        I.pf.ks[k] = (float)I.pd.ks[k];
    }
    for (int k = 0; k < 9; ++k) I.pf.kg[k] = (float)I.pd.kg[k];
    for (int k = 0; k < 15; ++k) I.pf.kn[k] = (float)(I.pd.kn[k] * 2.3283064365386963e-10);
}

lb_status validate(const lb_params &p) {
    if (p.nx < 2 || p.ny < 2 || p.nz < 2) return LB_ERR_ARG;
    if ((double)p.nx * p.ny * p.nz > 2.0e9) return LB_ERR_ARG;
    if (p.collision == 0 && !(p.tau > 0.5)) return LB_ERR_ARG;
    if (p.collision == 1) {
        const double r[4] = {p.gamma_shear, p.gamma_bulk, p.gamma_odd, p.gamma_even};
        for (double v : r)
            if (!(v > -1.0 && v < 1.0)) return LB_ERR_ARG;
    }
    if (!(p.rho0 > 0.0) || !(p.kT >= 0.0) || !(p.gamma_bead >= 0.0)) return LB_ERR_ARG;
    if (!std::isfinite(p.rho0) || !std::isfinite(p.kT) || !std::isfinite(p.gamma_bead)) return LB_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p.body_force[a])) return LB_ERR_ARG;
    if (p.kT > 0.0 && p.collision == 0) return LB_ERR_ARG;
    if (p.md_substeps < 0 || p.md_substeps > 4) return LB_ERR_ARG;
    return LB_OK;
}

void compute_g(const lb_batch_ctx *h, int k, double g[3]) {
    const lb_params &p = h->p[k];
    for (int a = 0; a < 3; ++a) g[a] = p.body_force[a];
    if (p.compensate_force && h->nfluid[k] > 0)
        for (int b : h->inst_bodies[k])
            if (h->hb[b].fixed != 1)
                for (int a = 0; a < 3; ++a) g[a] -= h->hb[b].F_ext[a] / (double)h->nfluid[k];
}

lb_status rebuild_schedule(lb_batch_ctx *h) {
    std::vector<int> ts(h->n + 1, 0);
    long long acc = 0;
    for (int k = 0; k < h->n; ++k) {
        ts[k] = (int)acc;
        acc += ((long long)h->hinst[k].nwork + h->TS - 1) / h->TS;
    }
    ts[h->n] = (int)acc;
    if (acc > 2000000000LL) return bfail(h, LB_ERR_ARG, "too many work tiles");
    h->ntiles = (int)acc;
    std::vector<int> ti((size_t)acc);
    for (int k = 0; k < h->n; ++k)
        for (int t = ts[k]; t < ts[k + 1]; ++t) ti[t] = k;
    if ((size_t)acc > h->tile_inst_cap) {
        if (h->dtile_inst) { cudaFree(h->dtile_inst); h->dtile_inst = nullptr; }
        lb_status s = balloc(h, &h->dtile_inst, sizeof(int) * (size_t)acc);
        if (s != LB_OK) return s;
        h->tile_inst_cap = (size_t)acc;
    }
    BCUDA(h, cudaMemcpyAsync(h->dtile_start, ts.data(), sizeof(int) * (h->n + 1), cudaMemcpyHostToDevice, h->stream));
    BCUDA(h, cudaMemcpyAsync(h->dtile_inst, ti.data(), sizeof(int) * (size_t)acc, cudaMemcpyHostToDevice, h->stream));
    BCUDA(h, cudaStreamSynchronize(h->stream));
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    // resident CTAs of the even- and odd-step fluid kernels at this tile size
    // (their register counts differ): each parity's persistent grid never
    // exceeds its own, so every CTA runs concurrently
    for (int odd = 0; odd < 2; ++odd) {
        int occ = 0;
        cudaError_t e;
#define BOCC(T, C, NZ, O)                                                                                           \
        e = h->common ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lbk::k_batch_collide<T, C, NZ, O, true>, h->TS, 0) \
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lbk::k_batch_collide<T, C, NZ, O, false>, h->TS, 0)
#define BOCC2(T, C, NZ) do { if (odd) BOCC(T, C, NZ, true); else BOCC(T, C, NZ, false); } while (0)
        if (h->fp32) {
            if (h->collision == 0) BOCC2(float, 0, false);
            else if (h->noise) BOCC2(float, 1, true);
            else BOCC2(float, 1, false);
        } else {
            if (h->collision == 0) BOCC2(double, 0, false);
            else if (h->noise) BOCC2(double, 1, true);
            else BOCC2(double, 1, false);
        }
#undef BOCC2
#undef BOCC
        if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
        h->resident[odd] = occ > 0 ? occ : 1;
    }
    return LB_OK;
}

lb_status upload(lb_batch_ctx *h) {
    if (h->uploaded) return LB_OK;
    // fluid positions across the axis of each pore instance: the fluid
    // kernel's work items are its fluid nodes only, and from here on the
    // instance stores only those (compact layout, converted in place below)
    std::vector<uint32_t> fl;
    std::vector<int> cm;
    std::vector<uint16_t> cn;
    std::vector<long long> cmap_off, cnbr_off;
    for (int k = 0; k < h->n; ++k) {
        BInst &I = h->hinst[k];
        if (I.g.pore_axis < 0) continue;
        const int ax = I.g.pore_axis;
        const int na = ax == 0 ? I.g.ny : I.g.nx, nb = ax == 2 ? I.g.ny : I.g.nz;   // across, first fastest
        I.loff = (long long)fl.size();
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                const long long da = 2LL * a + 1 - na, db = 2LL * b + 1 - nb;
                if (da * da + db * db >= I.g.pore_t) continue;          // wall node (same test as the kernels)
                const long long node = ax == 2 ? a + (long long)I.g.nx * b
                                     : (ax == 1 ? a + (long long)I.g.nx * I.g.ny * b
                                                : (long long)I.g.nx * (a + (long long)I.g.ny * b));
                fl.push_back((uint32_t)node);
            }
        I.ncs = (uint32_t)((long long)fl.size() - I.loff);
        if (I.ncs >= 0xFFFF)
            return bfail(h, LB_ERR_ARG, "instance " + std::to_string(k) + ": a batched pore's cross-section holds at "
                                        "most 65534 fluid positions (the compact layout indexes them in 16 bits)");
        // compact layout: dense position across the axis -> compact position
        // (-1 for a wall), and the 9 in-plane neighbours of each compact
        // position (periodic across the box, -1 where the neighbour is a wall)
        const long long coff = (long long)cm.size();
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                const long long da = 2LL * a + 1 - na, db = 2LL * b + 1 - nb;
                cm.push_back(da * da + db * db >= I.g.pore_t ? -1 : 0);
            }
        int jc = 0;
        for (long long q = coff; q < (long long)cm.size(); ++q)
            if (cm[q] >= 0) cm[q] = jc++;
        const long long noff = (long long)cn.size();
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                if (cm[coff + a + (long long)na * b] < 0) continue;
                uint16_t rec[8];
                for (int v = -1; v <= 1; ++v)
                    for (int u = -1; u <= 1; ++u) {
                        if (u == 0 && v == 0) continue;
                        const int a2 = (a + u + na) % na, b2 = (b + v + nb) % nb;
                        const int q = cm[coff + a2 + (long long)na * b2];
                        rec[lbk::dir8(u, v)] = q < 0 ? (uint16_t)0xFFFF : (uint16_t)q;
                    }
                cn.insert(cn.end(), rec, rec + 8);
            }
        cmap_off.push_back(coff);
        cnbr_off.push_back(noff);
        I.nax = (uint32_t)(ax == 0 ? I.g.nx : (ax == 1 ? I.g.ny : I.g.nz));
        I.astride = (uint32_t)(ax == 0 ? 1 : (ax == 1 ? I.g.nx : I.g.nx * I.g.ny));
        I.nwork = I.ncs * I.nax;
        const uint32_t d = ax == 0 ? I.nax : I.ncs;
        I.mw = d > 1 ? (uint32_t)((0x100000000ULL + d - 1) / d) : 0u;
        // exact while w * d < 2^32 for every work item w
        I.wfast = (d > 1 && (double)I.nwork * d < 4294967296.0) ? 1 : 0;
    }
    h->nfluidpos = (long long)fl.size();
    if (!fl.empty()) {
        lb_status s = balloc(h, &h->dfluid, sizeof(uint32_t) * fl.size());
        if (s != LB_OK) return s;
        if ((s = balloc(h, &h->dcmap, sizeof(int) * cm.size())) != LB_OK) return s;
        if ((s = balloc(h, &h->dcnbr, sizeof(uint16_t) * cn.size())) != LB_OK) return s;
        BCUDA(h, cudaMemcpyAsync(h->dfluid, fl.data(), sizeof(uint32_t) * fl.size(), cudaMemcpyHostToDevice,
                                 h->stream));
        BCUDA(h, cudaMemcpyAsync(h->dcmap, cm.data(), sizeof(int) * cm.size(), cudaMemcpyHostToDevice, h->stream));
        BCUDA(h, cudaMemcpyAsync(h->dcnbr, cn.data(), sizeof(uint16_t) * cn.size(), cudaMemcpyHostToDevice, h->stream));
        // convert each pore instance to the compact layout in place (its
        // region keeps its dense size): the populations in the dense layout
        // (step 0, even parity) go out through the gather and come back
        // through the compact scatter
        long long nmax = 0;
        for (int k = 0; k < h->n; ++k)
            if (h->hinst[k].g.pore_axis >= 0) nmax = std::max(nmax, h->hinst[k].g.N);
        double *tmp = nullptr;
        if (cudaMalloc((void **)&tmp, sizeof(double) * 19 * (size_t)nmax) != cudaSuccess) {
            cudaGetLastError();
            return bfail(h, LB_ERR_OOM, "no device memory to convert the pore instances' layout");
        }
        int pi = 0;
        for (int k = 0; k < h->n && s == LB_OK; ++k) {
            BInst &I = h->hinst[k];
            if (I.g.pore_axis < 0) continue;
            const long long N = I.g.N;
            const unsigned grid = (unsigned)((N + 255) / 256);
            lbk::Geom gd = I.g;
            gd.N = I.ps;
            gd.cmap = nullptr;
            if (h->fp32) lbk::k_batch_gather<float><<<grid, 256, 0, h->stream>>>((const float *)h->pool + I.off, gd, N, false, h->p[k].rho0, tmp);
            else lbk::k_batch_gather<double><<<grid, 256, 0, h->stream>>>((const double *)h->pool + I.off, gd, N, false, h->p[k].rho0, tmp);
            I.cmode = 1;
            I.ps = ((long long)I.ncs * I.nax + 31) / 32 * 32;
            I.g.cmap = h->dcmap + cmap_off[pi];
            I.g.cnbr = h->dcnbr + cnbr_off[pi];
            I.g.cps = I.ps;
            I.g.csj = I.g.pore_axis == 0 ? (int)I.nax : 1;
            I.g.csa = I.g.pore_axis == 0 ? 1 : (int)I.ncs;
            ++pi;
            lbk::Geom gc = I.g;
            gc.N = I.ps;
            if (h->fp32) {
                lbk::k_batch_init<float><<<(unsigned)((I.ps + 255) / 256), 256, 0, h->stream>>>((float *)h->pool + I.off, I.ps, h->p[k].rho0);
                lbk::k_batch_scatter<float><<<grid, 256, 0, h->stream>>>((float *)h->pool + I.off, gc, N, false, h->p[k].rho0, tmp);
            } else {
                lbk::k_batch_init<double><<<(unsigned)((I.ps + 255) / 256), 256, 0, h->stream>>>((double *)h->pool + I.off, I.ps, h->p[k].rho0);
                lbk::k_batch_scatter<double><<<grid, 256, 0, h->stream>>>((double *)h->pool + I.off, gc, N, false, h->p[k].rho0, tmp);
            }
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) s = bfail(h, LB_ERR_CUDA, std::string("compact layout: ") + cudaGetErrorString(e));
        }
        const cudaError_t e = cudaStreamSynchronize(h->stream);
        cudaFree(tmp);
        if (s != LB_OK) return s;
        if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("compact layout: ") + cudaGetErrorString(e));
        if ((s = rebuild_schedule(h)) != LB_OK) return s;   // tile counts follow the work items
    }
    // instance table with final body forces / compensation
    for (int k = 0; k < h->n; ++k) {
        double g[3];
        compute_g(h, k, g);
        for (int a = 0; a < 3; ++a) {
            h->hinst[k].gd[a] = g[a];
            h->hinst[k].gf[a] = (float)g[a];
        }
    }
    BCUDA(h, cudaMemcpyAsync(h->dinst, h->hinst.data(), sizeof(BInst) * h->n, cudaMemcpyHostToDevice, h->stream));
    const int nb = (int)h->hb.size(), nbeads = (int)h->hbody_of.size();
    lb_status s;
    if (nb > 0) {
        if ((s = balloc(h, &h->db, sizeof(Body) * nb)) != LB_OK) return s;
        if ((s = balloc(h, &h->ds, sizeof(double) * 3 * (size_t)nbeads)) != LB_OK) return s;
        if ((s = balloc(h, &h->dsf, sizeof(float) * 3 * (size_t)nbeads)) != LB_OK) return s;
        if ((s = balloc(h, &h->dbody_of, sizeof(int) * (size_t)nbeads)) != LB_OK) return s;
        if ((s = balloc(h, &h->dbead_rng, sizeof(int) * (size_t)nbeads)) != LB_OK) return s;
        if ((s = balloc(h, &h->dbead_inst, sizeof(int) * (size_t)std::max(nbeads, 1))) != LB_OK) return s;
        if ((s = balloc(h, &h->dFbead, sizeof(double) * 3 * (size_t)nbeads)) != LB_OK) return s;
        BCUDA(h, cudaMemcpyAsync(h->db, h->hb.data(), sizeof(Body) * nb, cudaMemcpyHostToDevice, h->stream));
        if (nbeads > 0) {
            BCUDA(h, cudaMemcpyAsync(h->ds, h->hs.data(), sizeof(double) * 3 * nbeads, cudaMemcpyHostToDevice, h->stream));
            h->hsf.assign(h->hs.begin(), h->hs.end());
            BCUDA(h, cudaMemcpyAsync(h->dsf, h->hsf.data(), sizeof(float) * 3 * nbeads, cudaMemcpyHostToDevice, h->stream));
            BCUDA(h, cudaMemcpyAsync(h->dbody_of, h->hbody_of.data(), sizeof(int) * nbeads, cudaMemcpyHostToDevice, h->stream));
            BCUDA(h, cudaMemcpyAsync(h->dbead_rng, h->hbead_rng.data(), sizeof(int) * nbeads, cudaMemcpyHostToDevice, h->stream));
            h->hbead_inst.resize(nbeads);
            for (int j = 0; j < nbeads; ++j) h->hbead_inst[j] = h->hb[h->hbody_of[j]].inst;
            BCUDA(h, cudaMemcpyAsync(h->dbead_inst, h->hbead_inst.data(), sizeof(int) * nbeads, cudaMemcpyHostToDevice, h->stream));
        }
        const size_t fb = (h->fp32 ? sizeof(float) : sizeof(double)) * 3 * (size_t)h->Ftot;
        h->list_cap = (int)std::min<long long>(h->Ttot, 8LL * std::max(nbeads, 1));
        for (int k = 0; k < 2; ++k) {
            if ((s = balloc(h, &h->Fbuf[k], fb)) != LB_OK) return s;
            if ((s = balloc(h, &h->tiles[k], sizeof(int) * (size_t)h->Ttot)) != LB_OK) return s;
            if ((s = balloc(h, &h->tlist[k], sizeof(int) * (size_t)h->list_cap)) != LB_OK) return s;
            if ((s = balloc(h, &h->tcount[k], sizeof(int))) != LB_OK) return s;
            BCUDA(h, cudaMemsetAsync(h->Fbuf[k], 0, fb, h->stream));
            BCUDA(h, cudaMemsetAsync(h->tiles[k], 0, sizeof(int) * (size_t)h->Ttot, h->stream));
            BCUDA(h, cudaMemsetAsync(h->tcount[k], 0, sizeof(int), h->stream));
        }
    }
    BCUDA(h, cudaStreamSynchronize(h->stream));
    h->uploaded = true;
    return LB_OK;
}

// Step k of a group. With bodies, its prologue (kick and drift, clearing of
// the force tiles of step k - 2) runs on the side stream: it needs the
// coupling of step k - 1 (body sums, and the force buffer it clears is the one
// that coupling read as the previous step's) but nothing the fluid kernel of
// step k - 1 reads or writes, so it is forked after that coupling (`more`: a
// step of the same group follows) and joined before the coupling of step k.
// Steps timed kernel by kernel (lb_batch_set_timing) keep it on the main
// stream, so that the fluid kernel's events time it alone.
lb_status launch_step(lb_batch_ctx *h, int k, bool finish_prev, bool record, bool more) {
    const bool side = !h->timing;
    cudaStream_t ps = side ? h->side : h->stream;
    const bool odd = ((h->step + k) & 1) != 0;
    const int cur = (int)((h->step + k) & 1), prev = cur ^ 1;
    const int nb = (int)h->hb.size(), nbeads = (int)h->hbody_of.size();
    const bool coupled = nb > 0 && nbeads > 0;
    const int nsub = h->nsub;
    const double dt = 1.0 / nsub;
    if (nb > 0) {
        // with MD substeps the record is taken after the last substep's drift
        const lbk::Recorder rec{nsub == 1 ? h->rec : nullptr, h->rec_every, h->rec_cap, h->step_dev, (uint32_t)k};
        const long long nthreads = std::min<long long>(64LL * h->list_cap, 152LL * 2048);
        const unsigned pg = std::max<unsigned>((unsigned)((nthreads + 255) / 256), (unsigned)nb);
        if (k == 0 && side) {
            BCUDA(h, cudaEventRecord(h->ev_fork, h->stream));
            BCUDA(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        }
        if (h->fp32)
            lbk::k_batch_pre<float><<<pg, 256, 0, ps>>>(
                h->db, nb, finish_prev ? 1 : 0, coupled ? (float *)h->Fbuf[cur] : nullptr,
                coupled ? h->tiles[cur] : nullptr, h->tlist[cur], h->tcount[cur], h->dinst, h->dflag_start, h->n,
                rec, h->list_cap, h->Ttot, h->derr, dt);
        else
            lbk::k_batch_pre<double><<<pg, 256, 0, ps>>>(
                h->db, nb, finish_prev ? 1 : 0, coupled ? (double *)h->Fbuf[cur] : nullptr,
                coupled ? h->tiles[cur] : nullptr, h->tlist[cur], h->tcount[cur], h->dinst, h->dflag_start, h->n,
                rec, h->list_cap, h->Ttot, h->derr, dt);
        BCUDA(h, cudaGetLastError());
        if (coupled) BCUDA(h, cudaMemsetAsync(h->tcount[cur], 0, sizeof(int), ps));
        if (side) {
            BCUDA(h, cudaEventRecord(h->ev_join, h->side));
            BCUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
        }
    }
    if (coupled) {
        lbk::BatchCouple c{};
        c.inst = h->dinst;
        c.pool = h->pool;
        c.fp32 = h->fp32;
        c.odd = odd;
        c.Fprev = h->Fbuf[prev];
        c.Fcur = h->Fbuf[cur];
        c.tiles_cur = h->tiles[cur];
        c.tlist = h->tlist[cur];
        c.tcount = h->tcount[cur];
        c.s = h->ds;
        c.sf = h->dsf;
        c.bead_body = h->dbody_of;
        c.bead_rng = h->dbead_rng;
        c.bead_inst = h->dbead_inst;
        c.ninst = h->n;
        c.bodies = h->db;
        c.F_bead = h->dFbead;
        c.nbeads = nbeads;
        c.step_base = h->step_dev;
        c.step_off = (uint32_t)k;
        c.err = h->derr;
        c.list_cap = h->list_cap;
        c.nbodies = nb;
        // bead noise of variance 2 kT gamma / dt per substep (Philox call 4 + substep)
        c.dt = dt;
        c.noise_scale = std::sqrt((double)nsub);
        c.dt_f = (float)dt;
        const unsigned grid = (unsigned)((8LL * nbeads + 127) / 128);
        for (int sub = 0; sub < nsub; ++sub) {
            if (sub > 0) {   // bodies move by dt between the couplings of one LB step
                const lbk::Recorder rec{sub == nsub - 1 ? h->rec : nullptr, h->rec_every, h->rec_cap, h->step_dev,
                                        (uint32_t)k};
                BCUDA(h, lbk::launch_substep(h->db, nb, dt, rec, h->stream));
            }
            c.call = 4u + (uint32_t)sub;
            if (h->fp32) lbk::k_batch_couple<float><<<grid, 128, 0, h->stream>>>(c);
            else lbk::k_batch_couple<double><<<grid, 128, 0, h->stream>>>(c);
            BCUDA(h, cudaGetLastError());
            if (h->any_wall) {
                lbk::k_batch_wall<<<(nbeads + 127) / 128, 128, 0, h->stream>>>(h->dinst, h->db, h->ds, h->dbody_of,
                                                                              nbeads, nb, h->derr);
                BCUDA(h, cudaGetLastError());
            }
        }
    }
    if (nb > 0 && more && side) {               // the next prologue may start now
        BCUDA(h, cudaEventRecord(h->ev_fork, h->stream));
        BCUDA(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    }
    lbk::BatchArgs a{};
    a.inst = h->dinst;
    a.tile_start = h->dtile_start;
    a.tile_inst = h->dtile_inst;
    a.n = h->n;
    a.ntiles = h->ntiles;
    a.pd = h->hinst[0].pd;
    a.pf = h->hinst[0].pf;
    const int res = h->resident[odd ? 1 : 0];
    int grid = h->sms * std::min(h->bpsm, res > 0 ? res : h->bpsm);
    if (h->order == 2) grid = h->ntiles;    // one CTA per tile, round-robin loop runs once
    if (grid > h->ntiles) grid = h->ntiles;
    if (grid < 1) grid = 1;
    a.order = h->order == 1 ? 1 : 0;
    a.chunk = (h->ntiles + grid - 1) / grid;
    a.pool = h->pool;
    a.fluid = h->dfluid;
    a.F = coupled ? h->Fbuf[cur] : nullptr;
    a.tiles = coupled ? h->tiles[cur] : nullptr;
    a.step_base = h->step_dev;
    a.step_off = (uint32_t)k;
    a.err = h->derr;
    a.nfluid = h->nfluidpos;
    a.ttot = h->Ttot;
    if (record) BCUDA(h, cudaEventRecord(h->ev[h->ev_used], h->stream));
#define BLAUNCH(T, C, NZ)                                                                                   \
    do {                                                                                                    \
        if (h->common) {                                                                                    \
            if (odd) lbk::k_batch_collide<T, C, NZ, true, true><<<grid, h->TS, 0, h->stream>>>(a);          \
            else lbk::k_batch_collide<T, C, NZ, false, true><<<grid, h->TS, 0, h->stream>>>(a);             \
        } else {                                                                                            \
            if (odd) lbk::k_batch_collide<T, C, NZ, true, false><<<grid, h->TS, 0, h->stream>>>(a);         \
            else lbk::k_batch_collide<T, C, NZ, false, false><<<grid, h->TS, 0, h->stream>>>(a);            \
        }                                                                                                   \
    } while (0)
    if (h->fp32) {
        if (h->collision == 0) BLAUNCH(float, 0, false);
        else if (h->noise) BLAUNCH(float, 1, true);
        else BLAUNCH(float, 1, false);
    } else {
        if (h->collision == 0) BLAUNCH(double, 0, false);
        else if (h->noise) BLAUNCH(double, 1, true);
        else BLAUNCH(double, 1, false);
    }
#undef BLAUNCH
    BCUDA(h, cudaGetLastError());
    if (record) {
        BCUDA(h, cudaEventRecord(h->ev[h->ev_used + 1], h->stream));
        h->ev_used += 2;
    }
    return LB_OK;
}

lb_status finish_steps(lb_batch_ctx *h, int nsteps) {
    const int nb = (int)h->hb.size();
    BCUDA(h, lbk::launch_finish(h->db, nb, 1.0 / h->nsub, h->step_dev, (unsigned)nsteps, h->stream));
    return LB_OK;
}

lb_status eager_steps(lb_batch_ctx *h, int nsteps) {
    for (int k = 0; k < nsteps; ++k) {
        bool rec = false;
        if (h->timing) {
            if (h->ev_used + 2 > h->ev.size())
                for (int e = 0; e < 256; ++e) {
                    cudaEvent_t ev;
                    BCUDA(h, cudaEventCreate(&ev));
                    h->ev.push_back(ev);
                }
            rec = true;
        }
        lb_status s = launch_step(h, k, k > 0, rec, k + 1 < nsteps);
        if (s != LB_OK) return s;
    }
    lb_status s = finish_steps(h, nsteps);
    h->step += nsteps;
    return s;
}

// two steps (even, odd) + second half kick + counter advance, as one graph
lb_status ensure_graph(lb_batch_ctx *h) {
    if (h->gexec) return LB_OK;
    cudaGraph_t graph = nullptr;
    BCUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    lb_status s = launch_step(h, 0, false, false, true);
    if (s == LB_OK) s = launch_step(h, 1, true, false, false);
    if (s == LB_OK) s = finish_steps(h, 2);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (s != LB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return LB_OK;
}

lb_status check(lb_batch_ctx *h, int k) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (k < 0 || k >= h->n) return bfail(h, LB_ERR_ARG, "instance index out of range");
    return LB_OK;
}

}  // namespace

extern "C" {

const char *lb_batch_last_error(lb_batch_handle h) { return h ? h->err.c_str() : g_batch_error.c_str(); }

lb_status lb_batch_create(const lb_params *params, int n, void *cuda_stream, lb_batch_handle *out) {
    if (!params || n <= 0 || !out) return bfail(nullptr, LB_ERR_ARG, "need n >= 1 parameter sets");
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (validate(params[k]) != LB_OK) return bfail(nullptr, LB_ERR_ARG, "invalid parameters for instance " + std::to_string(k));
        if (params[k].precision != params[0].precision || params[k].collision != params[0].collision ||
            (params[k].kT > 0.0) != (params[0].kT > 0.0) ||
            std::max(params[k].md_substeps, 1) != std::max(params[0].md_substeps, 1))
            return bfail(nullptr, LB_ERR_ARG,
                         "all instances must share precision, collision type, noise on/off and MD substeps");
    }
    if (params[0].precision != 32 && params[0].precision != 64) return bfail(nullptr, LB_ERR_ARG, "precision must be 32 or 64");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return bfail(nullptr, LB_ERR_CUDA, "no CUDA device");
    }
    lb_batch_ctx *h = new (std::nothrow) lb_batch_ctx();
    if (!h) return bfail(nullptr, LB_ERR_OOM, "host allocation failed");
    h->p.assign(params, params + n);
    h->n = n;
    h->fp32 = params[0].precision == 32;
    h->collision = params[0].collision;
    h->noise = params[0].collision == 1 && params[0].kT > 0.0;
    h->nsub = std::max(params[0].md_substeps, 1);
    h->hinst.resize(n);
    h->flag_start.assign(n + 1, 0);
    h->nfluid.assign(n, 0);
    h->inst_bodies.resize(n);
    h->inst_beads.assign(n, 0);
    long long off = 0, foff = 0, toff = 0;
    for (int k = 0; k < n; ++k) {
        const lb_params &p = params[k];
        BInst &I = h->hinst[k];
        std::memset(&I, 0, sizeof(I));
        I.g.nx = p.nx; I.g.ny = p.ny; I.g.nz = p.nz;
        I.g.N = (long long)p.nx * p.ny * p.nz;
        I.g.pore_axis = -1;
        I.loff = -1;
        I.nwork = (uint32_t)I.g.N;
        I.off = off;
        I.foff = foff;
        I.toff = toff;
        I.ntx = (p.nx + 3) / 4; I.nty = (p.ny + 3) / 4; I.ntz = (p.nz + 3) / 4;
        I.key0 = (uint32_t)p.seed;
        I.key1 = (uint32_t)(p.seed >> 32);
        I.instance = p.instance;
        I.rho0 = p.rho0;
        I.gamma = p.gamma_bead;
        I.noise_amp = p.kT > 0.0 ? std::sqrt(2.0 * p.kT * p.gamma_bead) : 0.0;
        I.gamma_f = (float)I.gamma;
        I.noise_amp_f = (float)I.noise_amp;
        I.noise_amp_sub_f = (float)(I.noise_amp * std::sqrt((double)h->nsub));
        fill_coll(p, I);
        I.mx = (uint32_t)((0x100000000ULL + p.nx - 1) / p.nx);
        I.my = (uint32_t)((0x100000000ULL + p.ny - 1) / p.ny);
        // exact while n * nx < 2^32 and (n / nx) * ny < 2^32 for all n < N
        I.fastdiv = ((double)I.g.N * p.nx < 4294967296.0 && (double)(I.g.N / p.nx) * p.ny < 4294967296.0) ? 1 : 0;
        h->flag_start[k] = toff;
        h->nfluid[k] = I.g.N;
        I.ps = (I.g.N + 31) / 32 * 32;
        I.fs = I.ps;
        h->Nnodes += I.g.N;
        off += 19 * I.ps;
        foff += 3 * I.fs;
        toff += (long long)I.ntx * I.nty * I.ntz;
    }
    h->flag_start[n] = toff;
    if (off >= 4294967296LL) {
        delete h;
        return bfail(nullptr, LB_ERR_ARG, "a batch holds at most 2^32 population values (19 per node)");
    }
    h->common = true;
    for (int k = 1; k < n; ++k)
        if (std::memcmp(&h->hinst[k].pd, &h->hinst[0].pd, sizeof(h->hinst[0].pd)) != 0) h->common = false;
    h->Ntot = off / 19;
    h->Ftot = foff / 3;
    h->Ttot = toff;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
    else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete h; return bfail(nullptr, LB_ERR_CUDA, "cudaStreamCreate failed"); }
        h->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        g_batch_error = std::string("side stream: ") + cudaGetErrorString(e);
        lb_batch_destroy(h);
        return LB_ERR_CUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t es = h->fp32 ? 4 : 8;
    lb_status s;
    if ((s = balloc(h, &h->pool, es * 19 * (size_t)h->Ntot)) != LB_OK ||
        (s = balloc(h, &h->dinst, sizeof(BInst) * n)) != LB_OK ||
        (s = balloc(h, &h->dtile_start, sizeof(int) * (n + 1))) != LB_OK ||
        (s = balloc(h, &h->dflag_start, sizeof(long long) * (n + 1))) != LB_OK ||
        (s = balloc(h, &h->step_dev, sizeof(unsigned long long))) != LB_OK ||
        (s = balloc(h, &h->derr, sizeof(int))) != LB_OK) {
        g_batch_error = h->err;
        lb_batch_destroy(h);
        return s;
    }
    if (cudaMallocHost((void **)&h->herr, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        h->herr = nullptr;
        g_batch_error = "no pinned host memory for the error word";
        lb_batch_destroy(h);
        return LB_ERR_OOM;
    }
    e = cudaMemsetAsync(h->step_dev, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->dflag_start, h->flag_start.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, h->stream);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        const BInst &I = h->hinst[k];
        if (h->fp32) lbk::k_batch_init<float><<<(unsigned)((I.ps + 255) / 256), 256, 0, h->stream>>>((float *)h->pool + I.off, I.ps, h->p[k].rho0);
        else lbk::k_batch_init<double><<<(unsigned)((I.ps + 255) / 256), 256, 0, h->stream>>>((double *)h->pool + I.off, I.ps, h->p[k].rho0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        g_batch_error = std::string("batch init: ") + cudaGetErrorString(e);
        lb_batch_destroy(h);
        return LB_ERR_CUDA;
    }
    if ((s = rebuild_schedule(h)) != LB_OK) {
        g_batch_error = h->err;
        lb_batch_destroy(h);
        return s;
    }
    *out = h;
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch_handle h) {
    if (!h) return LB_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    void *bufs[] = {h->pool, h->Fbuf[0], h->Fbuf[1], h->tiles[0], h->tiles[1], h->tlist[0], h->tlist[1], h->tcount[0],
                    h->tcount[1], h->dinst, h->dtile_start, h->dtile_inst,
                    h->dflag_start, h->step_dev, h->db, h->ds, h->dsf, h->dbody_of, h->dbead_rng, h->dbead_inst, h->dFbead, h->rec, h->dcmap, h->dcnbr, h->dfluid,
                    h->derr};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (h->herr) cudaFreeHost(h->herr);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return LB_OK;
}

lb_status lb_batch_set_pore(lb_batch_handle h, int k, double radius, int axis) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    if (h->uploaded || h->step > 0) return bfail(h, LB_ERR_STATE, "pores must be set before the first step");
    if (axis < 0 || axis > 2 || !(radius > 0.0)) return bfail(h, LB_ERR_ARG, "bad pore");
    BInst &I = h->hinst[k];
    const double t = std::ceil(4.0 * (radius * radius));
    I.g.pore_axis = axis;
    I.g.pore_t = (long long)t;
    I.pore_R = radius;
    I.wall = lbk::WallBeads{};
    const double inner = std::sqrt(t) - 2.0 * std::sqrt(2.0) - 0.01;
    I.g.pore_in = inner > 0 ? (long long)std::floor(inner * inner) : 0;
    const int na = axis == 0 ? I.g.ny : I.g.nx, nb = axis == 2 ? I.g.ny : I.g.nz;
    const int nl = axis == 0 ? I.g.nx : (axis == 1 ? I.g.ny : I.g.nz);
    long long c = 0;
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < na; ++a) {
            const long long da = 2LL * a + 1 - na, db = 2LL * b + 1 - nb;
            if (da * da + db * db < I.g.pore_t) ++c;
        }
    h->nfluid[k] = c * nl;
    return LB_OK;
}

lb_status lb_batch_set_pore_beads(lb_batch_handle h, int k, double spacing, double r_pore_bead, double r_bead,
                                  double epsilon) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    if (h->uploaded) return bfail(h, LB_ERR_STATE, "pore beads must be set before the first step");
    BInst &I = h->hinst[k];
    if (I.g.pore_axis < 0) return bfail(h, LB_ERR_STATE, "lb_batch_set_pore_beads needs a pore");
    if (spacing == 0.0) {
        I.wall = lbk::WallBeads{};
        return LB_OK;
    }
    if (!lbk::make_wall_beads(I.g, I.pore_R, spacing, r_pore_bead, r_bead, epsilon, I.wall))
        return bfail(h, LB_ERR_ARG, "spacing > 0, radii >= 0 with a positive sum, epsilon >= 0");
    h->any_wall = true;
    return LB_OK;
}

lb_status lb_batch_add_raspberry(lb_batch_handle h, int k, const double *beads, int nbeads, const double X[3],
                                 const double q[4], double mass, const double inertia[3], const double F_ext[3],
                                 const double T_ext[3], int fixed, int *body_id) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    if (h->uploaded) return bfail(h, LB_ERR_STATE, "bodies must be added before the first step");
    if (nbeads < 0 || (nbeads > 0 && !beads) || !X || !q || !inertia || !(mass > 0.0) ||
        !(inertia[0] > 0 && inertia[1] > 0 && inertia[2] > 0))
        return bfail(h, LB_ERR_ARG, "bad raspberry arguments");
    const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(qn > 0.0) || !std::isfinite(qn)) return bfail(h, LB_ERR_ARG, "quaternion must be non-zero");
    if (!lbk::all_finite(beads, 3 * nbeads) || !lbk::all_finite(X, 3) || !lbk::all_finite(&mass, 1) ||
        !lbk::all_finite(inertia, 3) || !lbk::all_finite(F_ext, 3) || !lbk::all_finite(T_ext, 3))
        return bfail(h, LB_ERR_ARG, "non-finite bead offset, position, mass, inertia or external force");
    Body b{};
    for (int a = 0; a < 3; ++a) {
        b.X[a] = X[a];
        b.I[a] = inertia[a];
        b.F_ext[a] = F_ext ? F_ext[a] : 0.0;
        b.T_ext[a] = T_ext ? T_ext[a] : 0.0;
    }
    for (int a = 0; a < 4; ++a) b.q[a] = q[a] / qn;
    b.mass = mass;
    b.inv_mass = 1.0 / mass;
    for (int a = 0; a < 3; ++a) b.inv_I[a] = 1.0 / inertia[a];
    if (fixed < 0 || fixed > 2) return bfail(h, LB_ERR_ARG, "fixed must be 0, 1 or 2");
    b.fixed = fixed;
    b.inst = k;
    const int id = (int)h->hb.size();
    h->hb.push_back(b);
    for (int j = 0; j < 3 * nbeads; ++j) h->hs.push_back(beads[j]);
    for (int j = 0; j < nbeads; ++j) {
        h->hbody_of.push_back(id);
        h->hbead_rng.push_back(h->inst_beads[k] + j);
    }
    h->inst_beads[k] += nbeads;
    if (body_id) *body_id = (int)h->inst_bodies[k].size();
    h->inst_bodies[k].push_back(id);
    return LB_OK;
}

lb_status lb_batch_step(lb_batch_handle h, int nsteps) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (nsteps < 0) return bfail(h, LB_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return LB_OK;
    lb_status s = upload(h);
    if (s != LB_OK) return s;
    if (h->timing || LB_BATCH_EAGER) return eager_steps(h, nsteps);
    if (h->step & 1) {
        if ((s = eager_steps(h, 1)) != LB_OK) return s;
        --nsteps;
    }
    const int pairs = nsteps / 2;
    if (pairs > 0) {
        if ((s = ensure_graph(h)) != LB_OK) return s;
        for (int r = 0; r < pairs; ++r) BCUDA(h, cudaGraphLaunch(h->gexec, h->stream));
        h->step += 2LL * pairs;
    }
    if (nsteps & 1) return eager_steps(h, 1);
    return LB_OK;
}

lb_status lb_batch_record_bodies(lb_batch_handle h, int every, int capacity) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (every < 0 || (every > 0 && capacity < 1)) return bfail(h, LB_ERR_ARG, "every >= 0 and capacity >= 1");
    if (every > 0 && h->hb.empty()) return bfail(h, LB_ERR_ARG, "no bodies to record");
    if (h->rec) {
        BCUDA(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->rec);
        h->dev_bytes -= sizeof(double) * 7 * (size_t)h->rec_cap * h->hb.size();
        h->rec = nullptr;
    }
    h->rec_every = h->rec_cap = 0;
    if (h->gexec) {                        // the captured steps hold the old recorder
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    if (every == 0) return LB_OK;
    lb_status s = upload(h);               // the body set is fixed from here on
    if (s != LB_OK) return s;
    if ((s = balloc(h, &h->rec, sizeof(double) * 7 * (size_t)capacity * h->hb.size())) != LB_OK) return s;
    h->rec_every = every;
    h->rec_cap = capacity;
    h->rec_k0 = h->step / every + 1;
    return LB_OK;
}

lb_status lb_batch_get_trajectory(lb_batch_handle h, int k, int body, int max_records, long long *steps, double *X,
                                  double *q, int *count) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    if (!count || max_records < 0) return bfail(h, LB_ERR_ARG, "count must not be NULL, max_records >= 0");
    if (body < 0 || body >= (int)h->inst_bodies[k].size()) return bfail(h, LB_ERR_ARG, "bad body id");
    cudaError_t e = lbk::copy_records(h->rec, h->rec_every, h->rec_cap, h->rec_k0, h->step, (int)h->hb.size(),
                                      h->inst_bodies[k][body], max_records, steps, X, q, count, h->stream);
    if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("lb_batch_get_trajectory: ") + cudaGetErrorString(e));
    return LB_OK;
}

namespace {

// Synchronises the stream (completing the copies the caller queued) and
// returns LB_ERR_STATE once if an index check of a checked build failed
// since the last check (the word is then cleared).
lb_status bcheck_device(lb_batch_ctx *h) {
    BCUDA(h, cudaMemcpyAsync(h->herr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    BCUDA(h, cudaStreamSynchronize(h->stream));
    if (*h->herr & 2) {
        BCUDA(h, cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream));
        return bfail(h, LB_ERR_STATE, "an index check of the checked build failed (an index outside its array)");
    }
    return LB_OK;
}

}  // namespace

lb_status lb_batch_forces(lb_batch_handle h, int k, int body, double F[3], double T[3]) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    if (body < 0 || body >= (int)h->inst_bodies[k].size()) return bfail(h, LB_ERR_ARG, "bad body id");
    const int id = h->inst_bodies[k][body];
    if (!h->uploaded) {
        for (int a = 0; a < 3; ++a) { if (F) F[a] = 0; if (T) T[a] = 0; }
        return LB_OK;
    }
    if (F) BCUDA(h, cudaMemcpyAsync(F, &h->db[id].F_tot[0], 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (T) BCUDA(h, cudaMemcpyAsync(T, &h->db[id].T_tot[0], 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return bcheck_device(h);
}

lb_status lb_batch_get_body(lb_batch_handle h, int k, int body, double X[3], double V[3], double q[4], double w[3]) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    if (body < 0 || body >= (int)h->inst_bodies[k].size()) return bfail(h, LB_ERR_ARG, "bad body id");
    const int id = h->inst_bodies[k][body];
    Body b = h->hb[id];
    if (h->uploaded) {
        BCUDA(h, cudaMemcpyAsync(&b, &h->db[id], sizeof(Body), cudaMemcpyDeviceToHost, h->stream));
        if ((s = bcheck_device(h)) != LB_OK) return s;
    }
    for (int a = 0; a < 3; ++a) {
        if (X) X[a] = b.X[a];
        if (V) V[a] = b.V[a];
        if (w) w[a] = b.w[a];
    }
    if (q) for (int a = 0; a < 4; ++a) q[a] = b.q[a];
    return LB_OK;
}

namespace {
// an instance's geometry with N the plane stride of the pool (population I/O)
lbk::Geom pool_geom(const BInst &I) {
    lbk::Geom g = I.g;
    g.N = I.ps;
    return g;
}
}  // namespace

lb_status lb_batch_get_populations(lb_batch_handle h, int k, double *host, size_t n) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    const BInst &I = h->hinst[k];
    if (!host || n != 19 * (size_t)I.g.N) return bfail(h, LB_ERR_ARG, "buffer must hold 19*N doubles");
    double *tmp = nullptr;
    if ((s = balloc(h, &tmp, sizeof(double) * n)) != LB_OK) return s;
    h->dev_bytes -= sizeof(double) * n;
    const bool odd = (h->step & 1) != 0;
    const unsigned grid = (unsigned)((I.g.N + 255) / 256);
    if (h->fp32) lbk::k_batch_gather<float><<<grid, 256, 0, h->stream>>>((const float *)h->pool + I.off, pool_geom(I), I.g.N, odd, h->p[k].rho0, tmp);
    else lbk::k_batch_gather<double><<<grid, 256, 0, h->stream>>>((const double *)h->pool + I.off, pool_geom(I), I.g.N, odd, h->p[k].rho0, tmp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("lb_batch_get_populations: ") + cudaGetErrorString(e));
    return bcheck_device(h);
}

lb_status lb_batch_set_populations(lb_batch_handle h, int k, const double *host, size_t n) {
    lb_status s = check(h, k);
    if (s != LB_OK) return s;
    const BInst &I = h->hinst[k];
    if (!host || n != 19 * (size_t)I.g.N) return bfail(h, LB_ERR_ARG, "buffer must hold 19*N doubles");
    double *tmp = nullptr;
    if ((s = balloc(h, &tmp, sizeof(double) * n)) != LB_OK) return s;
    h->dev_bytes -= sizeof(double) * n;
    const bool odd = (h->step & 1) != 0;
    const unsigned grid = (unsigned)((I.g.N + 255) / 256);
    cudaError_t e = cudaMemcpyAsync(tmp, host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        if (h->fp32) lbk::k_batch_scatter<float><<<grid, 256, 0, h->stream>>>((float *)h->pool + I.off, pool_geom(I), I.g.N, odd, h->p[k].rho0, tmp);
        else lbk::k_batch_scatter<double><<<grid, 256, 0, h->stream>>>((double *)h->pool + I.off, pool_geom(I), I.g.N, odd, h->p[k].rho0, tmp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bfail(h, LB_ERR_CUDA, std::string("lb_batch_set_populations: ") + cudaGetErrorString(e));
    return LB_OK;
}

lb_status lb_batch_set_schedule(lb_batch_handle h, int tile_nodes, int blocks_per_sm, int order) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    // the persistent grid is capped at the CTAs that are resident at once (at
    // most 2048 threads per SM; fewer as the registers allow)
    if ((tile_nodes != 64 && tile_nodes != 128 && tile_nodes != 256) || blocks_per_sm < 1 ||
        blocks_per_sm * tile_nodes > 2048 || order < 0 || order > 2)
        return bfail(h, LB_ERR_ARG, "tile_nodes 64/128/256, blocks_per_sm * tile_nodes <= 2048, order 0/1/2");
    h->TS = tile_nodes;
    h->bpsm = blocks_per_sm;
    h->order = order;
    return rebuild_schedule(h);
}

lb_status lb_batch_autotune(lb_batch_handle h, int trial_steps, int chosen[3], double *best_ms_per_step) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (trial_steps < 2) trial_steps = 2;
    trial_steps &= ~1;   // keep the parity
    lb_status s = upload(h);
    if (s != LB_OK) return s;
    // snapshot of everything a step changes
    const size_t es = h->fp32 ? 4 : 8;
    const size_t pbytes = es * 19 * (size_t)h->Ntot;
    const int nb = (int)h->hb.size();
    void *snap = nullptr;
    Body *bsnap = nullptr;
    void *fsnap[2] = {nullptr, nullptr};
    int *tsnap[2] = {nullptr, nullptr};
    int *lsnap[2] = {nullptr, nullptr};
    const size_t fbytes = (h->fp32 ? sizeof(float) : sizeof(double)) * 3 * (size_t)h->Ftot;
    if (cudaMalloc(&snap, pbytes) != cudaSuccess) { cudaGetLastError(); return bfail(h, LB_ERR_OOM, "no room for the autotune snapshot"); }
    bool ok = true;
    if (nb > 0) {
        ok = cudaMalloc((void **)&bsnap, sizeof(Body) * nb) == cudaSuccess;
        for (int k = 0; k < 2 && ok; ++k)
            ok = cudaMalloc((void **)&fsnap[k], fbytes) == cudaSuccess &&
                 cudaMalloc((void **)&tsnap[k], sizeof(int) * (size_t)h->Ttot) == cudaSuccess &&
                 cudaMalloc((void **)&lsnap[k], sizeof(int) * ((size_t)h->list_cap + 1)) == cudaSuccess;
    }
    auto release = [&]() {
        cudaFree(snap);
        if (bsnap) cudaFree(bsnap);
        for (int k = 0; k < 2; ++k) {
            if (fsnap[k]) cudaFree(fsnap[k]);
            if (tsnap[k]) cudaFree(tsnap[k]);
            if (lsnap[k]) cudaFree(lsnap[k]);
        }
    };
    if (!ok) { cudaGetLastError(); release(); return bfail(h, LB_ERR_OOM, "no room for the autotune snapshot"); }
    auto copy_state = [&](bool save) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(save ? snap : h->pool, save ? h->pool : snap, pbytes, cudaMemcpyDeviceToDevice, h->stream);
        if (nb > 0 && e == cudaSuccess) {
            e = cudaMemcpyAsync(save ? (void *)bsnap : (void *)h->db, save ? (void *)h->db : (void *)bsnap, sizeof(Body) * nb, cudaMemcpyDeviceToDevice, h->stream);
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                e = cudaMemcpyAsync(save ? (void *)fsnap[k] : (void *)h->Fbuf[k], save ? (void *)h->Fbuf[k] : (void *)fsnap[k], fbytes, cudaMemcpyDeviceToDevice, h->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(save ? (void *)tsnap[k] : (void *)h->tiles[k], save ? (void *)h->tiles[k] : (void *)tsnap[k], sizeof(int) * (size_t)h->Ttot, cudaMemcpyDeviceToDevice, h->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(save ? (void *)lsnap[k] : (void *)h->tlist[k], save ? (void *)h->tlist[k] : (void *)lsnap[k], sizeof(int) * (size_t)h->list_cap, cudaMemcpyDeviceToDevice, h->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(save ? (void *)(lsnap[k] + h->list_cap) : (void *)h->tcount[k], save ? (void *)h->tcount[k] : (void *)(lsnap[k] + h->list_cap), sizeof(int), cudaMemcpyDeviceToDevice, h->stream);
            }
        }
        return e;
    };
    unsigned long long step_saved = 0;
    cudaError_t e = copy_state(true);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&step_saved, h->step_dev, sizeof(step_saved), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { release(); return bfail(h, LB_ERR_CUDA, std::string("autotune snapshot: ") + cudaGetErrorString(e)); }
    const long long step_host = h->step;
    const bool timing = h->timing;
    h->timing = false;
    // trial steps record nothing (the ring keeps the simulation's records;
    // each schedule change drops the captured graph, so no trial graph
    // outlives this)
    double *rec_saved = h->rec;
    h->rec = nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int tiles[3] = {64, 128, 256};
    double best = 1e30;
    int bt = h->TS, bb = h->bpsm, bo = h->order;
    for (int ts : tiles)
        for (int bps = 2; bps * ts <= 2048; bps *= 2)
            for (int order = 0; order < 3; ++order) {
                if (order == 2 && bps != 2) continue;     // blocks_per_sm unused: one trial per tile size
                if ((s = lb_batch_set_schedule(h, ts, bps, order)) != LB_OK) break;
                // warm-up pair, then timed pairs
                if ((s = lb_batch_step(h, 2)) != LB_OK) break;
                cudaEventRecord(e0, h->stream);
                if ((s = lb_batch_step(h, trial_steps)) != LB_OK) break;
                cudaEventRecord(e1, h->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / trial_steps < best) { best = ms / trial_steps; bt = ts; bb = bps; bo = order; }
                // restore
                e = copy_state(false);
                if (e == cudaSuccess) e = cudaMemcpyAsync(h->step_dev, &step_saved, sizeof(step_saved), cudaMemcpyHostToDevice, h->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
                h->step = step_host;
                if (e != cudaSuccess) { s = bfail(h, LB_ERR_CUDA, std::string("autotune restore: ") + cudaGetErrorString(e)); break; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    h->timing = timing;
    h->rec = rec_saved;
    if (s != LB_OK) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        return s;
    }
    s = lb_batch_set_schedule(h, bt, bb, bo);
    if (chosen) { chosen[0] = bt; chosen[1] = bb; chosen[2] = bo; }
    if (best_ms_per_step) *best_ms_per_step = best;
    return s;
}

namespace {

struct BatchCkptHeader {
    char magic[8];
    int n, precision, collision, nbodies, nbeads, list_cap;
    long long Ntot, Ftot, Ttot, step;
    unsigned long long geometry;      // FNV-1a of every instance's sizes, pore, seed and instance number
    unsigned long long body_bytes, total;
};

unsigned long long batch_geometry_hash(const lb_batch_ctx *h) {
    unsigned long long x = 1469598103934665603ULL;
    auto mix = [&](const void *v, size_t nbytes) {
        const unsigned char *c = static_cast<const unsigned char *>(v);
        for (size_t k = 0; k < nbytes; ++k) x = (x ^ c[k]) * 1099511628211ULL;
    };
    for (int k = 0; k < h->n; ++k) {
        const BInst &I = h->hinst[k];
        const long long v[6] = {I.g.nx, I.g.ny, I.g.nz, I.g.pore_axis, (long long)I.g.pore_t,
                                (long long)h->p[k].seed};
        mix(v, sizeof(v));
        mix(&h->p[k].instance, sizeof(h->p[k].instance));
        mix(&I.pore_R, sizeof(I.pore_R));
    }
    return x;
}

// the sections of a batch checkpoint: device pointer and bytes, in file order
std::vector<std::pair<void *, size_t>> batch_ckpt_sections(lb_batch_ctx *h) {
    std::vector<std::pair<void *, size_t>> v;
    const size_t es = h->fp32 ? 4 : 8;
    v.push_back({h->pool, 19 * es * (size_t)h->Ntot});
    const int nb = (int)h->hb.size(), nbeads = (int)h->hbody_of.size();
    if (nb > 0) {
        v.push_back({h->db, sizeof(Body) * nb});
        if (nbeads > 0) v.push_back({h->dFbead, sizeof(double) * 3 * (size_t)nbeads});
        for (int k = 0; k < 2; ++k) {
            v.push_back({h->Fbuf[k], 3 * es * (size_t)h->Ftot});
            v.push_back({h->tiles[k], sizeof(int) * (size_t)h->Ttot});
            if (h->list_cap > 0) v.push_back({h->tlist[k], sizeof(int) * (size_t)h->list_cap});
            v.push_back({h->tcount[k], sizeof(int)});
        }
    }
    return v;
}

BatchCkptHeader batch_ckpt_header(lb_batch_ctx *h) {
    BatchCkptHeader c{};
    std::memcpy(c.magic, "LBBCKP1", 8);
    c.n = h->n;
    c.precision = h->fp32 ? 32 : 64;
    c.collision = h->collision;
    c.nbodies = (int)h->hb.size();
    c.nbeads = (int)h->hbody_of.size();
    c.list_cap = h->list_cap;
    c.Ntot = h->Ntot;
    c.Ftot = h->Ftot;
    c.Ttot = h->Ttot;
    c.step = h->step;
    c.geometry = batch_geometry_hash(h);
    c.body_bytes = sizeof(Body);
    size_t total = sizeof(BatchCkptHeader);
    for (auto &sec : batch_ckpt_sections(h)) total += sec.second;
    c.total = total;
    return c;
}

}  // namespace

lb_status lb_batch_checkpoint_size(lb_batch_handle h, size_t *bytes) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (!bytes) return bfail(h, LB_ERR_ARG, "null argument");
    lb_status s = upload(h);
    if (s != LB_OK) return s;
    *bytes = (size_t)batch_ckpt_header(h).total;
    return LB_OK;
}

lb_status lb_batch_checkpoint_save(lb_batch_handle h, void *host, size_t bytes) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (!host) return bfail(h, LB_ERR_ARG, "null buffer");
    lb_status s = upload(h);
    if (s != LB_OK) return s;
    const BatchCkptHeader c = batch_ckpt_header(h);
    if (bytes < c.total) return bfail(h, LB_ERR_ARG, "buffer smaller than lb_batch_checkpoint_size");
    char *p = static_cast<char *>(host);
    std::memcpy(p, &c, sizeof(c));
    p += sizeof(c);
    for (auto &sec : batch_ckpt_sections(h)) {
        BCUDA(h, cudaMemcpyAsync(p, sec.first, sec.second, cudaMemcpyDeviceToHost, h->stream));
        p += sec.second;
    }
    BCUDA(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

lb_status lb_batch_checkpoint_load(lb_batch_handle h, const void *host, size_t bytes) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (!host || bytes < sizeof(BatchCkptHeader)) return bfail(h, LB_ERR_ARG, "buffer too small for a checkpoint");
    BatchCkptHeader c;
    std::memcpy(&c, host, sizeof(c));
    if (std::memcmp(c.magic, "LBBCKP1", 8) != 0) return bfail(h, LB_ERR_ARG, "not a batch checkpoint of this library");
    lb_status s = upload(h);
    if (s != LB_OK) return s;
    const BatchCkptHeader mine = batch_ckpt_header(h);
    if (c.n != mine.n || c.precision != mine.precision || c.collision != mine.collision ||
        c.nbodies != mine.nbodies || c.nbeads != mine.nbeads || c.list_cap != mine.list_cap ||
        c.Ntot != mine.Ntot || c.Ftot != mine.Ftot || c.Ttot != mine.Ttot || c.geometry != mine.geometry ||
        c.body_bytes != mine.body_bytes || c.total != mine.total)
        return bfail(h, LB_ERR_STATE, "the checkpoint was taken from a batch with other instances or bodies");
    if (bytes < c.total) return bfail(h, LB_ERR_ARG, "buffer shorter than the checkpoint");
    if (h->gexec) {                        // the captured steps start from the saved parity again
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    const char *p = static_cast<const char *>(host) + sizeof(c);
    for (auto &sec : batch_ckpt_sections(h)) {
        BCUDA(h, cudaMemcpyAsync(sec.first, p, sec.second, cudaMemcpyHostToDevice, h->stream));
        p += sec.second;
    }
    const unsigned long long st = (unsigned long long)c.step;
    BCUDA(h, cudaMemcpyAsync(h->step_dev, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
    BCUDA(h, cudaStreamSynchronize(h->stream));
    h->step = c.step;
    return LB_OK;
}

lb_status lb_batch_info(lb_batch_handle h, long long *total_nodes, long long *step, int schedule[3]) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    if (total_nodes) *total_nodes = h->Nnodes;
    if (step) *step = h->step;
    if (schedule) { schedule[0] = h->TS; schedule[1] = h->bpsm; schedule[2] = h->order; }
    return LB_OK;
}

lb_status lb_batch_set_timing(lb_batch_handle h, int on) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    h->timing = on != 0;
    return LB_OK;
}

lb_status lb_batch_kernel_time(lb_batch_handle h, double *total_ms, long long *launches) {
    if (!h) return bfail(nullptr, LB_ERR_ARG, "null handle");
    BCUDA(h, cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float ms = 0.f;
        BCUDA(h, cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
        h->timed_ms += ms;
        h->timed_n += 1;
    }
    h->ev_used = 0;
    if (total_ms) *total_ms = h->timed_ms;
    if (launches) *launches = h->timed_n;
    h->timed_ms = 0.0;
    h->timed_n = 0;
    return LB_OK;
}

}  // extern "C"
