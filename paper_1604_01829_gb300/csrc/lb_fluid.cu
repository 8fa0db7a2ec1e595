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
#include "lb_internal.h"

namespace lbk {

namespace {

// ---------------------------------------------------------------- collision
// Post-collision populations of one node, in place. Force F = uniform + spread
// bead force; u = (j + F/2) / rho (Guo forcing); MRT in the orthogonal
// D3Q19 moment basis 1, c, c^2-1, 3cx^2-c^2, cy^2-cz^2, cxcy, cycz, czcx,
// (3c^2-5)c, (cy^2-cz^2)cx, (cz^2-cx^2)cy, (cx^2-cy^2)cz, 3c^4-6c^2+1,
// (2c^2-3)(3cx^2-c^2), (2c^2-3)(cy^2-cz^2), with norms b_k = sum w e_k^2.
template <typename R, bool DEV, int COLL, bool NOISE>
__device__ __forceinline__ void collide(R (&f)[19], R Fx, R Fy, R Fz, const CollParams<R> &a,
                                        const FluidArgs &fa, uint32_t node, uint32_t step) {
    const R s1 = f[1] + f[2], d1 = f[1] - f[2];
    const R s3 = f[3] + f[4], d3 = f[3] - f[4];
    const R s5 = f[5] + f[6], d5 = f[5] - f[6];
    const R s7 = f[7] + f[8], d7 = f[7] - f[8];
    const R s9 = f[9] + f[10], d9 = f[9] - f[10];
    const R s11 = f[11] + f[12], d11 = f[11] - f[12];
    const R s13 = f[13] + f[14], d13 = f[13] - f[14];
    const R s15 = f[15] + f[16], d15 = f[15] - f[16];
    const R s17 = f[17] + f[18], d17 = f[17] - f[18];
    const R Sax = s1 + s3 + s5;
    const R Sxy = s7 + s9, Sxz = s11 + s13, Syz = s15 + s17;
    const R Sd = Sxy + Sxz + Syz;
    const R m0 = f[0] + Sax + Sd;                      // rho, or rho - rho0 for deviations
    const R rho = DEV ? a.rho0 + m0 : m0;
    const R jx = d1 + d7 + d9 + d11 + d13;
    const R jy = d3 + d7 - d9 + d15 + d17;
    const R jz = d5 + d11 - d13 + d15 - d17;
    R ir;
    if constexpr (sizeof(R) == 4) ir = __frcp_rn(rho); else ir = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * ir;
    const R uy = (jy + R(0.5) * Fy) * ir;
    const R uz = (jz + R(0.5) * Fz) * ir;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R uu = ux * ux + uy * uy + uz * uz;
    constexpr R w0 = R(1.0 / 3.0), w1 = R(1.0 / 18.0), w2 = R(1.0 / 36.0);

    if (COLL == 0) {
        // BGK: f* = f - (f - f_eq)/tau + (1 - 1/(2 tau)) w [3(c-u) + 9 (c.u) c].F
        const R om = a.omega, h = R(1) - R(0.5) * om;
        const R base = DEV ? m0 : rho;                 // w rho (or w (rho - rho0)) coefficient of '1'
        const R k2 = R(1.5) * uu;
        // rest population
        f[0] = f[0] - om * (f[0] - w0 * (base - rho * k2)) + h * w0 * (R(-3) * uF);
        auto pair = [&](int i, R cu, R cF, R w) {
            const R e = w * (base + rho * (R(4.5) * cu * cu - k2));
            const R o = w * rho * R(3) * cu;
            const R se = w * (R(9) * cu * cF - R(3) * uF);
            const R so = w * R(3) * cF;
            f[i] = f[i] - om * (f[i] - (e + o)) + h * (se + so);
            f[i + 1] = f[i + 1] - om * (f[i + 1] - (e - o)) + h * (se - so);
        };
        pair(1, ux, Fx, w1);
        pair(3, uy, Fy, w1);
        pair(5, uz, Fz, w1);
        pair(7, ux + uy, Fx + Fy, w2);
        pair(9, ux - uy, Fx - Fy, w2);
        pair(11, ux + uz, Fx + Fz, w2);
        pair(13, ux - uz, Fx - Fz, w2);
        pair(15, uy + uz, Fy + Fz, w2);
        pair(17, uy - uz, Fy - Fz, w2);
        return;
    }

    // MRT: non-conserved moments
    R m4 = Sd - f[0];
    R m5 = R(2) * s1 - s3 - s5 + Sxy + Sxz - R(2) * Syz;
    R m6 = s3 - s5 + Sxy - Sxz;
    R m7 = s7 - s9, m8 = s15 - s17, m9 = s11 - s13;
    R m10 = R(-2) * d1 + d7 + d9 + d11 + d13;
    R m11 = R(-2) * d3 + d7 - d9 + d15 + d17;
    R m12 = R(-2) * d5 + d11 - d13 + d15 - d17;
    R m13 = d7 + d9 - d11 - d13;
    R m14 = -d7 + d9 + d15 + d17;
    R m15 = d11 - d13 - d15 + d17;
    R m16 = f[0] - R(2) * Sax + Sd;
    R m17 = -(R(2) * s1 - s3 - s5) + Sxy + Sxz - R(2) * Syz;
    R m18 = -(s3 - s5) + Sxy - Sxz;

    // equilibrium stress moments and Guo source moments
    const R gb = a.gb, gs = a.gs, go = a.go, ge = a.ge;
    const R hb = R(0.5) * (R(1) + gb), hs = R(0.5) * (R(1) + gs);
    {
        const R e4 = rho * uu;
        const R e5 = rho * (R(2) * ux * ux - uy * uy - uz * uz);
        const R e6 = rho * (uy * uy - uz * uz);
        const R e7 = rho * ux * uy, e8 = rho * uy * uz, e9 = rho * uz * ux;
        m4 = e4 + gb * (m4 - e4) + hb * (R(2) * uF);
        m5 = e5 + gs * (m5 - e5) + hs * (R(2) * (R(2) * ux * Fx - uy * Fy - uz * Fz));
        m6 = e6 + gs * (m6 - e6) + hs * (R(2) * (uy * Fy - uz * Fz));
        m7 = e7 + gs * (m7 - e7) + hs * (ux * Fy + uy * Fx);
        m8 = e8 + gs * (m8 - e8) + hs * (uy * Fz + uz * Fy);
        m9 = e9 + gs * (m9 - e9) + hs * (uz * Fx + ux * Fz);
    }
    m10 *= go; m11 *= go; m12 *= go; m13 *= go; m14 *= go; m15 *= go;
    m16 *= ge; m17 *= ge; m18 *= ge;

    if (NOISE) {
        // 15 non-conserved modes, variance 3 rho kT b_k (1 - g_k^2)
        const uint2 key = make_uint2(fa.key0, fa.key1);
        const uint4 r0 = philox4x32_10(make_uint4(node, step, fa.instance, 0u), key);
        const uint4 r1 = philox4x32_10(make_uint4(node, step, fa.instance, 1u), key);
        const uint4 r2 = philox4x32_10(make_uint4(node, step, fa.instance, 2u), key);
        const uint4 r3 = philox4x32_10(make_uint4(node, step, fa.instance, 3u), key);
        const R sr = sqrt(rho);
        auto xi = [](uint32_t v) -> R {
            if constexpr (sizeof(R) == 8) return unit_uniform_d(v); else return unit_uniform_f(v);
        };
        m4 += sr * a.sig[0] * xi(r0.x);
        m5 += sr * a.sig[1] * xi(r0.y);
        m6 += sr * a.sig[2] * xi(r0.z);
        m7 += sr * a.sig[3] * xi(r0.w);
        m8 += sr * a.sig[4] * xi(r1.x);
        m9 += sr * a.sig[5] * xi(r1.y);
        m10 += sr * a.sig[6] * xi(r1.z);
        m11 += sr * a.sig[7] * xi(r1.w);
        m12 += sr * a.sig[8] * xi(r2.x);
        m13 += sr * a.sig[9] * xi(r2.y);
        m14 += sr * a.sig[10] * xi(r2.z);
        m15 += sr * a.sig[11] * xi(r2.w);
        m16 += sr * a.sig[12] * xi(r3.x);
        m17 += sr * a.sig[13] * xi(r3.y);
        m18 += sr * a.sig[14] * xi(r3.z);
    }

    // back to populations: f*_i = w_i sum_k e_k(c_i) m*_k / b_k
    const R a0 = m0;
    const R a1 = R(3) * (jx + Fx), a2 = R(3) * (jy + Fy), a3 = R(3) * (jz + Fz);
    const R a4 = R(1.5) * m4, a5 = R(0.75) * m5, a6 = R(2.25) * m6;
    const R a7 = R(9) * m7, a8 = R(9) * m8, a9 = R(9) * m9;
    const R a10 = R(1.5) * m10, a11 = R(1.5) * m11, a12 = R(1.5) * m12;
    const R a13 = R(4.5) * m13, a14 = R(4.5) * m14, a15 = R(4.5) * m15;
    const R a16 = R(0.5) * m16, a17 = R(0.75) * m17, a18 = R(2.25) * m18;

    f[0] = w0 * (a0 - a4 + a16);
    {
        const R E = a0 + R(2) * a5 - R(2) * a16 - R(2) * a17, O = a1 - R(2) * a10;
        f[1] = w1 * (E + O); f[2] = w1 * (E - O);
    }
    {
        const R E = a0 - a5 + a6 - R(2) * a16 + a17 - a18, O = a2 - R(2) * a11;
        f[3] = w1 * (E + O); f[4] = w1 * (E - O);
    }
    {
        const R E = a0 - a5 - a6 - R(2) * a16 + a17 + a18, O = a3 - R(2) * a12;
        f[5] = w1 * (E + O); f[6] = w1 * (E - O);
    }
    const R Ed = a0 + a4 + a16;
    {
        const R E = Ed + a5 + a6 + a7 + a17 + a18, O = a1 + a2 + a10 + a11 + a13 - a14;
        f[7] = w2 * (E + O); f[8] = w2 * (E - O);
    }
    {
        const R E = Ed + a5 + a6 - a7 + a17 + a18, O = a1 - a2 + a10 - a11 + a13 + a14;
        f[9] = w2 * (E + O); f[10] = w2 * (E - O);
    }
    {
        const R E = Ed + a5 - a6 + a9 + a17 - a18, O = a1 + a3 + a10 + a12 - a13 + a15;
        f[11] = w2 * (E + O); f[12] = w2 * (E - O);
    }
    {
        const R E = Ed + a5 - a6 - a9 + a17 - a18, O = a1 - a3 + a10 - a12 - a13 - a15;
        f[13] = w2 * (E + O); f[14] = w2 * (E - O);
    }
    {
        const R E = Ed - R(2) * a5 + a8 - R(2) * a17, O = a2 + a3 + a11 + a12 + a14 - a15;
        f[15] = w2 * (E + O); f[16] = w2 * (E - O);
    }
    {
        const R E = Ed - R(2) * a5 - a8 - R(2) * a17, O = a2 - a3 + a11 - a12 + a14 + a15;
        f[17] = w2 * (E + O); f[18] = w2 * (E - O);
    }
}

// ------------------------------------------------------- collide and stream
template <typename T, int COLL, bool NOISE, bool ODD, bool PORE>
__global__ void __launch_bounds__(128) k_collide_stream(const FluidArgs a) {
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

    bool near_wall = false;
    if (PORE) {
        const long long r2 = pore_r2(g, x, y, z);
        if (r2 >= g.pore_t) return;          // wall node: holds no fluid
        near_wall = r2 >= g.pore_in;         // some neighbour may be a wall node
    }

    // neighbour offsets with periodic wrap: node = xo[dx] + yo[dy] + zo[dz]
    // (32-bit; the node count is limited to 2^31 at creation)
    const int nxy = g.nx * g.ny;
    const int xo[3] = {x == 0 ? g.nx - 1 : x - 1, x, x == g.nx - 1 ? 0 : x + 1};
    const int yo[3] = {(y == 0 ? g.ny - 1 : y - 1) * g.nx, y * g.nx, (y == g.ny - 1 ? 0 : y + 1) * g.nx};
    const int zo[3] = {(z == 0 ? g.nz - 1 : z - 1) * nxy, z * nxy, (z == g.nz - 1 ? 0 : z + 1) * nxy};
    const unsigned N32 = (unsigned)N;
    auto plane = [&](int i) { return A + (size_t)i * N32; };

    R f[19];
    if (!ODD) {
#pragma unroll
        for (int i = 0; i < 19; ++i) f[i] = plane(i)[n];
    } else {
        f[0] = A[n];
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const unsigned src = (unsigned)(xo[1 - cx(i)] + yo[1 - cy(i)] + zo[1 - cz(i)]);
            if (PORE && near_wall) {
                int xs = xo[1 - cx(i)], ys = (y - cy(i) + g.ny) % g.ny, zs = (z - cz(i) + g.nz) % g.nz;
                if (pore_r2(g, xs, ys, zs) >= g.pore_t) { f[i] = plane(i)[n]; continue; }
            }
            f[i] = plane(opp(i))[src];
        }
    }

    R Fx, Fy, Fz;
    if constexpr (sizeof(R) == 4) {
        Fx = __ldg(a.gforce_f); Fy = __ldg(a.gforce_f + 1); Fz = __ldg(a.gforce_f + 2);
    } else {
        Fx = __ldg(a.gforce); Fy = __ldg(a.gforce + 1); Fz = __ldg(a.gforce + 2);
    }
    if (a.tiles && a.tiles[tile_of(x, y, z, a.ntx, a.nty)]) {
        Fx += (R)a.Fn[n];
        Fy += (R)a.Fn[N + n];
        Fz += (R)a.Fn[2 * N + n];
    }
    uint32_t step = 0;
    if (NOISE) step = (uint32_t)(*a.step_base) + a.step_off;

    if constexpr (sizeof(R) == 4) collide<R, DEV, COLL, NOISE>(f, Fx, Fy, Fz, a.pf, a, (uint32_t)n, step);
    else collide<R, DEV, COLL, NOISE>(f, Fx, Fy, Fz, a.pd, a, (uint32_t)n, step);

    if (!ODD) {
#pragma unroll
        for (int i = 0; i < 19; ++i) plane(opp(i))[n] = f[i];
    } else {
        A[n] = f[0];
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            const unsigned dst = (unsigned)(xo[1 + cx(i)] + yo[1 + cy(i)] + zo[1 + cz(i)]);
            if (PORE && near_wall) {
                int xd = xo[1 + cx(i)], yd = (y + cy(i) + g.ny) % g.ny, zd = (z + cz(i) + g.nz) % g.nz;
                if (pore_r2(g, xd, yd, zd) >= g.pore_t) { plane(opp(i))[n] = f[i]; continue; }
            }
            plane(i)[dst] = f[i];
        }
    }
}

template <typename T, int COLL, bool NOISE>
cudaError_t launch_cs_t(const FluidArgs &a, bool odd, dim3 block, cudaStream_t s) {
    const dim3 grid((a.g.nx + block.x - 1) / block.x, (a.g.ny + block.y - 1) / block.y, a.g.nz);
    const bool pore = a.g.pore_axis >= 0;
    if (odd) {
        if (pore) k_collide_stream<T, COLL, NOISE, true, true><<<grid, block, 0, s>>>(a);
        else k_collide_stream<T, COLL, NOISE, true, false><<<grid, block, 0, s>>>(a);
    } else {
        if (pore) k_collide_stream<T, COLL, NOISE, false, true><<<grid, block, 0, s>>>(a);
        else k_collide_stream<T, COLL, NOISE, false, false><<<grid, block, 0, s>>>(a);
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

__global__ void k_advance(unsigned long long *step, unsigned int by) { *step += by; }

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
    if (fp32) k_moments<float><<<nblocks, 256, 0, s>>>((const float *)f, g, odd, partials);
    else k_moments<double><<<nblocks, 256, 0, s>>>((const double *)f, g, odd, partials);
    k_moments_final<<<1, 256, 0, s>>>(partials, nblocks, out4);
    return cudaGetLastError();
}

cudaError_t launch_advance(unsigned long long *step, unsigned int by, cudaStream_t s) {
    k_advance<<<1, 1, 0, s>>>(step, by);
    return cudaGetLastError();
}

}  // namespace lbk
