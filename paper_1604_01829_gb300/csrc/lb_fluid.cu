// Fluid kernels: the fused collide-and-stream step (Sec. 1.1 of Ustach &
// Faller, arXiv:1604.01829: streaming along the velocity links, relaxation
// towards equilibrium with one (BGK) or many (MRT) rates, optional thermal
// noise, bounce-back at boundary nodes) plus population I/O and reductions.
//
// Layout: structure of arrays, plane i of the 19 populations at f + i*N,
// node index x + nx (y + ny z), x fastest, so each warp touches 32
// consecutive elements per plane. One buffer, streamed in place with the AA
// pattern: on an even step a node reads and writes only its own 19 slots
// (writing each post-collision population into the slot of the opposite
// link); on an odd step it reads the 19 slots its neighbours wrote and
// writes its results into the neighbours' slots. Every slot is read and
// written by the same thread within a launch, so no second buffer and no
// synchronisation is needed. Halfway bounce-back on an odd step replaces a
// read from (write to) a wall neighbour by a read from (write to) the own
// opposite slot.
//
// FP32 storage holds d_i = f_i - w_i rho0 and computes in FP32; all moments
// but the density are unchanged by the shift, so only rho = rho0 + sum d_i
// and the zeroth reconstruction coefficient see it.
#include <algorithm>
#include <cmath>

#include "lb_collide.cuh"

// Minimum resident blocks of 128 threads per SM requested for the FP32
// collide kernels (caps their registers; FP64 kernels are not capped):
// 8 blocks (64 registers) without noise, 7 (72 registers) with it, where the
// Philox state needs the room (measured on GB300 at 256^3 with noise: 0.439 ms
// per launch at 7 blocks, 0.452 at 8, 0.458 at 6, 0.488 at 5; without noise
// 0.415 ms at 8, 0.419 at 7).
#ifndef LB_CS_MINB
#define LB_CS_MINB 8
#endif
#ifndef LB_CS_MINB_NOISE
#define LB_CS_MINB_NOISE 7
#endif

namespace lbk {

namespace {

// ------------------------------------------------------------ pore wall masks
__constant__ signed char kC[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                       {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                       {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                       {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

// One thread per position across the pore axis (the wall test ignores the
// coordinate along it): bit 31 if the node is a wall node, else bit i for
// every link whose upstream node x - c_i is a wall node.
__global__ void k_build_masks(Geom g, uint32_t *out, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (g.chan) {                        // channel walls: the mask depends on y only
        uint32_t m = 0;
        for (int i = 1; i < 19; ++i) {
            const int ys = t - kC[i][1];
            if (ys < 0 || ys >= g.ny) m |= 1u << i;
        }
        out[t] = m;
        return;
    }
    int x = 0, y = 0, z = 0;
    if (g.pore_axis == 2) { x = t % g.nx; y = t / g.nx; }
    else if (g.pore_axis == 1) { x = t % g.nx; z = t / g.nx; }
    else { y = t % g.ny; z = t / g.ny; }
    if (pore_r2(g, x, y, z) >= g.pore_t) {
        out[t] = 1u << 31;
        return;
    }
    uint32_t m = 0;
    for (int i = 1; i < 19; ++i) {
        const int xs = wrapm(x - kC[i][0], g.nx), ys = wrapm(y - kC[i][1], g.ny), zs = wrapm(z - kC[i][2], g.nz);
        if (pore_r2(g, xs, ys, zs) >= g.pore_t) m |= 1u << i;
    }
    out[t] = m;
}

__device__ __forceinline__ uint32_t pore_section_index(const Geom &g, int x, int y, int z) {
    if (g.chan) return (uint32_t)y;
    return g.pore_axis == 2 ? (uint32_t)x + (uint32_t)g.nx * (uint32_t)y
         : (g.pore_axis == 1 ? (uint32_t)x + (uint32_t)g.nx * (uint32_t)z : (uint32_t)y + (uint32_t)g.ny * (uint32_t)z);
}

// ------------------------------------------------------- collide and stream

template <typename T, int COLL, bool NOISE, bool ODD, bool PORE, bool OOP = false>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (NOISE ? LB_CS_MINB_NOISE : LB_CS_MINB) : 1)
    k_collide_stream(const FluidArgs a) {
    using R = T;
    constexpr bool DEV = sizeof(T) == 4;
    const Geom &g = a.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    T *A = static_cast<T *>(a.f);
    const long long N = g.N;
    const unsigned n = (unsigned)x + (unsigned)g.nx * ((unsigned)y + (unsigned)g.ny * (unsigned)z);

    uint32_t wmask = 0;                      // bit i: the upstream node x - c_i is a wall node
    if (PORE) {
        wmask = __ldg(a.masks + pore_section_index(g, x, y, z));
        if (wmask >> 31) return;             // wall node: holds no fluid
    }

    // Neighbour node n + (dx, dy, dz) with periodic wrap (32-bit; the node
    // count is limited to 2^31 at creation), from per-axis wrapped offsets.
    // Without noise, a row whose y and z are away from the box faces (all but
    // 4 rows in 256 at 256^3) takes a form that wraps only in x: n plus a
    // per-link constant plus one of two x corrections, so three values stay
    // live through the collision instead of nine (measured on GB300: 3.5 %
    // faster without noise, slower with it, where the Philox state competes
    // for the same registers).
    const int nx = g.nx, nxy = g.nx * g.ny;
    const int xo[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int yo[3] = {(y == 0 ? g.ny - 1 : y - 1) * nx, y * nx, (y == g.ny - 1 ? 0 : y + 1) * nx};
    const int zo[3] = {(z == 0 ? g.nz - 1 : z - 1) * nxy, z * nxy, (z == g.nz - 1 ? 0 : z + 1) * nxy};
    const bool row_in = !NOISE && y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1;
    const int wxm = x == 0 ? nx : 0, wxp = x == nx - 1 ? -nx : 0;
    auto nb_in = [&](int dx, int dy, int dz) -> unsigned {
        return (unsigned)((int)n + (dx < 0 ? wxm : (dx > 0 ? wxp : 0)) + (dx + dy * nx + dz * nxy));
    };
    auto nb_any = [&](int dx, int dy, int dz) -> unsigned {
        return (unsigned)(xo[1 + dx] + yo[1 + dy] + zo[1 + dz]);
    };
    auto plane = [&](int i) { return static_cast<T *>(a.plane[i]); };
    // stores: in place, or (OOP) into the output planes
    T *AO = OOP ? static_cast<T *>(a.out[0]) : A;
    auto oplane = [&](int i) { return static_cast<T *>(OOP ? a.out[i] : a.plane[i]); };

    R f[19];
    // odd step: population i arrives from the upstream node n - c_i, where it
    // sits in the opposite slot; halfway bounce-back takes the population that
    // left towards a wall (plus the moving-wall term of a channel wall upstream)
    auto load_odd = [&](auto nb) {
        f[0] = A[n];
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (PORE && ((wmask >> i) & 1u))
                f[i] = g.chan ? (R)((double)plane(i)[n] + chan_term(g, cy(i) > 0 ? 0 : 1, i)) : (R)plane(i)[n];
            else
                f[i] = plane(opp(i))[chk(nb(-cx(i), -cy(i), -cz(i)), N, a.err)];
        }
    };
    if (!ODD) {
#pragma unroll
        for (int i = 0; i < 19; ++i) f[i] = plane(i)[chk(n, N, a.err)];
    } else if (row_in) {
        load_odd(nb_in);
    } else {
        load_odd(nb_any);
    }

    R Fx, Fy, Fz;
    if constexpr (sizeof(R) == 4) {
        Fx = __ldg(a.gforce_f); Fy = __ldg(a.gforce_f + 1); Fz = __ldg(a.gforce_f + 2);
    } else {
        Fx = __ldg(a.gforce); Fy = __ldg(a.gforce + 1); Fz = __ldg(a.gforce + 2);
    }
    if (a.tiles && a.tiles[tile_of(x, y, z, a.ntx, a.nty)]) {
        const T *Fn = static_cast<const T *>(a.Fn);
        Fx += Fn[n];
        Fy += Fn[N + n];
        Fz += Fn[2 * N + n];
    }
    uint32_t step = 0;
    if (NOISE) step = (uint32_t)(*a.step_base) + a.step_off;

    const uint2 key = make_uint2(a.key0, a.key1);
    if constexpr (sizeof(R) == 4) collide<R, DEV, COLL, NOISE>(f, Fx, Fy, Fz, a.pf, key, a.instance, (uint32_t)n, step);
    else collide<R, DEV, COLL, NOISE>(f, Fx, Fy, Fz, a.pd, key, a.instance, (uint32_t)n, step);

    // odd step: f*_i goes to the downstream node n + c_i, the upstream node of
    // link opp(i) there; a wall downstream returns it into the own slot
    auto store_odd = [&](auto nb) {
        AO[n] = f[0];
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (PORE && ((wmask >> opp(i)) & 1u))
                oplane(opp(i))[n] = g.chan ? (T)((double)f[i] - chan_term(g, cy(i) < 0 ? 0 : 1, i)) : (T)f[i];
            else oplane(i)[chk(nb(cx(i), cy(i), cz(i)), N, a.err)] = f[i];
        }
    };
    if (!ODD) {
#pragma unroll
        for (int i = 0; i < 19; ++i) oplane(opp(i))[chk(n, N, a.err)] = f[i];
    } else if (row_in) {
        store_odd(nb_in);
    } else {
        store_odd(nb_any);
    }
}

template <typename T, int COLL, bool NOISE, bool OOP = false>
cudaError_t launch_cs_t(const FluidArgs &a, bool odd, dim3 block, cudaStream_t s) {
    const dim3 grid((a.g.nx + block.x - 1) / block.x, (a.g.ny + block.y - 1) / block.y, a.g.nz);
    const bool pore = a.g.pore_axis >= 0 || a.g.chan;       // bounded: per-position wall masks
    if (odd) {
        if (pore) k_collide_stream<T, COLL, NOISE, true, true, OOP><<<grid, block, 0, s>>>(a);
        else k_collide_stream<T, COLL, NOISE, true, false, OOP><<<grid, block, 0, s>>>(a);
    } else {
        if (pore) k_collide_stream<T, COLL, NOISE, false, true, OOP><<<grid, block, 0, s>>>(a);
        else k_collide_stream<T, COLL, NOISE, false, false, OOP><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ population I/O
template <typename T>
__global__ void k_init(T *f, long long N, double rho0) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
#pragma unroll
    for (int i = 0; i < 19; ++i) f[(long long)i * N + n] = sizeof(T) == 4 ? T(0) : T(wq(i) * rho0);
}

__device__ __forceinline__ void decode(const Geom &g, long long n, int &x, int &y, int &z) {
    x = (int)(n % g.nx);
    const long long r = n / g.nx;
    y = (int)(r % g.ny);
    z = (int)(r / g.ny);
}

template <typename T>
__global__ void k_gather(const T *f, Geom g, bool odd, double rho0, double *out) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    int x, y, z;
    decode(g, n, x, y, z);
    const bool wall = is_wall(g, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const T v = wall ? f[(long long)i * g.N + n] : load_pre(f, g, x, y, z, n, i, odd);
        out[(long long)i * g.N + n] = sizeof(T) == 4 ? (double)v + wq(i) * rho0 : (double)v;
    }
}

template <typename T>
__global__ void k_scatter(T *f, Geom g, bool odd, double rho0, const double *in) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    int x, y, z;
    decode(g, n, x, y, z);
    if (is_wall(g, x, y, z)) return;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const double v = in[(long long)i * g.N + n];
        store_pre(f, g, x, y, z, n, i, odd, sizeof(T) == 4 ? (T)(v - wq(i) * rho0) : (T)v);
    }
}

template <typename T>
__global__ void k_sample(const T *f, Geom g, bool odd, double rho0, const long long *nodes, int count,
                         double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const long long n = nodes[k];
    if (n < 0 || n >= g.N) {
        for (int i = 0; i < 19; ++i) out[19LL * k + i] = __longlong_as_double(0x7FF8000000000000LL);
        return;
    }
    int x, y, z;
    decode(g, n, x, y, z);
    const bool wall = is_wall(g, x, y, z);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const T v = wall ? f[(long long)i * g.N + n] : load_pre(f, g, x, y, z, n, i, odd);
        out[19LL * k + i] = sizeof(T) == 4 ? (double)v + wq(i) * rho0 : (double)v;
    }
}

// Sum over fluid nodes of (f, c f) in FP64: per-block partials, then one block.
template <typename T>
__global__ void __launch_bounds__(256) k_moments(const T *f, Geom g, bool odd, double *partials) {
    double s[4] = {0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        decode(g, n, x, y, z);
        if (is_wall(g, x, y, z)) continue;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double v = (double)load_pre(f, g, x, y, z, n, i, odd);
            s[0] += v;
            if (cx(i)) s[1] += cx(i) * v;
            if (cy(i)) s[2] += cy(i) * v;
            if (cz(i)) s[3] += cz(i) * v;
        }
    }
    __shared__ double red[4][256];
#pragma unroll
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) partials[4LL * blockIdx.x + c] = red[c][0];
}

// FP32 deviations in a periodic box: every population sits in exactly one
// slot of one node, in slot i on an even step count and in slot opp(i) of
// the upstream node on an odd one, so mass and momentum are plane sums:
// M = sum over all slots, P = +/- sum_i c_i (sum of plane i). One coalesced
// pass; each thread sums four nodes' 19 values in FP32 (deviations of
// O(1e-2): rounding ~1e-9 per partial) and accumulates the partials in FP64.
__global__ void __launch_bounds__(256) k_moments_periodic_f32(const float *f, long long N, bool odd,
                                                            double *partials) {
    double s[4] = {0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    while (n < N) {
        float p[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < 4 && n < N; ++k, n += stride) {
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                const float v = __ldcs(f + (long long)i * N + n);
                p[0] += v;
                if (cx(i)) p[1] += cx(i) * v;
                if (cy(i)) p[2] += cy(i) * v;
                if (cz(i)) p[3] += cz(i) * v;
            }
        }
        s[0] += (double)p[0];
        for (int c = 1; c < 4; ++c) s[c] += odd ? -(double)p[c] : (double)p[c];
    }
    __shared__ double red[4][256];
#pragma unroll
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) partials[4LL * blockIdx.x + c] = red[c][0];
}

__global__ void __launch_bounds__(256) k_moments_final(const double *partials, int nblocks, double *out) {
    __shared__ double red[4][256];
    double s[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] += partials[4LL * b + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) out[c] = red[c][0];
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_init(void *f, bool fp32, long long N, double rho0, cudaStream_t s) {
    if (fp32) k_init<float><<<blocks_for(N, 256), 256, 0, s>>>((float *)f, N, rho0);
    else k_init<double><<<blocks_for(N, 256), 256, 0, s>>>((double *)f, N, rho0);
    return cudaGetLastError();
}

cudaError_t launch_collide_stream(const FluidArgs &a, bool fp32, int collision, bool noise, bool odd,
                                  dim3 block, cudaStream_t s) {
    if (fp32) {
        if (collision == 0) return launch_cs_t<float, 0, false>(a, odd, block, s);
        if (noise) return launch_cs_t<float, 1, true>(a, odd, block, s);
        return launch_cs_t<float, 1, false>(a, odd, block, s);
    }
    if (collision == 0) return launch_cs_t<double, 0, false>(a, odd, block, s);
    if (noise) return launch_cs_t<double, 1, true>(a, odd, block, s);
    return launch_cs_t<double, 1, false>(a, odd, block, s);
}

cudaError_t launch_collide_stream_oop(const FluidArgs &a, bool fp32, int collision, bool odd, dim3 block,
                                      cudaStream_t s) {
    if (fp32) {
        if (collision == 0) return launch_cs_t<float, 0, false, true>(a, odd, block, s);
        return launch_cs_t<float, 1, false, true>(a, odd, block, s);
    }
    if (collision == 0) return launch_cs_t<double, 0, false, true>(a, odd, block, s);
    return launch_cs_t<double, 1, false, true>(a, odd, block, s);
}

bool make_wall_beads(const Geom &g, double pore_R, double spacing, double r_pore_bead, double r_bead, double eps,
                     WallBeads &w) {
    w = WallBeads{};
    if (g.pore_axis < 0 || !(spacing > 0.0) || !(r_pore_bead >= 0.0) || !(r_bead >= 0.0) ||
        !(r_pore_bead + r_bead > 0.0) || !(eps >= 0.0) || !std::isfinite(spacing) || !std::isfinite(eps))
        return false;
    const int n[3] = {g.nx, g.ny, g.nz};
    const int ax = g.pore_axis, a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
    const double twopi = 6.283185307179586;
    w.on = 1;
    w.axis = ax;
    w.Rc = pore_R + r_pore_bead;
    w.L = n[ax];
    w.cu = 0.5 * n[a1];
    w.cv = 0.5 * n[a2];
    w.ntheta = std::max(3, (int)std::lround(twopi * w.Rc / spacing));
    w.nrow = std::max(1, (int)std::lround(w.L / spacing));
    const double sigma = r_pore_bead + r_bead;
    w.sigma2 = sigma * sigma;
    w.rcut2 = std::pow(2.0, 1.0 / 3.0) * w.sigma2;
    w.eps = eps;
    // a bead at radius rho >= Rc - rcut is at distance >= 2 sqrt(rho Rc) sin(dphi / 2)
    // from a wall bead dphi away around the axis, and >= |dz| along it
    const double rcut = std::sqrt(w.rcut2), rmin = w.Rc - rcut;
    const double x = rmin > 0.0 ? rcut / (2.0 * std::sqrt(rmin * w.Rc)) : 2.0;
    w.wt = x >= 1.0 ? w.ntheta : (int)std::ceil(2.0 * std::asin(x) * w.ntheta / twopi + 0.5) + 1;
    w.wz = (int)std::ceil(rcut / (w.L / w.nrow) + 0.5) + 1;
    return true;
}

long long pore_section_size(const Geom &g) {
    if (g.chan) return g.ny;
    return g.pore_axis == 2 ? (long long)g.nx * g.ny
         : (g.pore_axis == 1 ? (long long)g.nx * g.nz : (long long)g.ny * g.nz);
}

cudaError_t launch_build_masks(const Geom &g, uint32_t *out, cudaStream_t s) {
    const int n = (int)pore_section_size(g);
    k_build_masks<<<(n + 255) / 256, 256, 0, s>>>(g, out, n);
    return cudaGetLastError();
}

cudaError_t launch_gather(const void *f, bool fp32, const Geom &g, bool odd, double rho0, double *out,
                          cudaStream_t s) {
    if (fp32) k_gather<float><<<blocks_for(g.N, 256), 256, 0, s>>>((const float *)f, g, odd, rho0, out);
    else k_gather<double><<<blocks_for(g.N, 256), 256, 0, s>>>((const double *)f, g, odd, rho0, out);
    return cudaGetLastError();
}

cudaError_t launch_scatter(void *f, bool fp32, const Geom &g, bool odd, double rho0, const double *in,
                           cudaStream_t s) {
    if (fp32) k_scatter<float><<<blocks_for(g.N, 256), 256, 0, s>>>((float *)f, g, odd, rho0, in);
    else k_scatter<double><<<blocks_for(g.N, 256), 256, 0, s>>>((double *)f, g, odd, rho0, in);
    return cudaGetLastError();
}

cudaError_t launch_sample(const void *f, bool fp32, const Geom &g, bool odd, double rho0,
                          const long long *nodes, int count, double *out, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (fp32) k_sample<float><<<blocks_for(count, 128), 128, 0, s>>>((const float *)f, g, odd, rho0, nodes, count, out);
    else k_sample<double><<<blocks_for(count, 128), 128, 0, s>>>((const double *)f, g, odd, rho0, nodes, count, out);
    return cudaGetLastError();
}

cudaError_t launch_moments(const void *f, bool fp32, const Geom &g, bool odd, double *partials,
                           int nblocks, double *out4, cudaStream_t s) {
    if (fp32 && g.pore_axis < 0 && !g.chan)
        k_moments_periodic_f32<<<nblocks, 256, 0, s>>>((const float *)f, g.N, odd, partials);
    else if (fp32) k_moments<float><<<nblocks, 256, 0, s>>>((const float *)f, g, odd, partials);
    else k_moments<double><<<nblocks, 256, 0, s>>>((const double *)f, g, odd, partials);
    k_moments_final<<<1, 256, 0, s>>>(partials, nblocks, out4);
    return cudaGetLastError();
}

}  // namespace lbk
