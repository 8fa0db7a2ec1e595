// Device-side building blocks of the LB + raspberry-coupling step (sm_103a).
//
// D3Q19 velocity set, Philox4x32-10, node indexing with periodic wrap, the
// analytic cylindrical-pore wall test and the parity-aware population access
// of the in-place (AA) streaming pattern.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbk {

// ----------------------------------------------------------------- lattice
// D3Q19 (Sec. 1.1 "discrete velocity links"): 0 rest; 1-6 axis links
// +x -x +y -y +z -z; 7-18 face diagonals, each followed by its opposite:
// (+x+y)(-x-y) (+x-y)(-x+y) (+x+z)(-x-z) (+x-z)(-x+z) (+y+z)(-y-z) (+y-z)(-y+z).
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
// opposite link: odd i pairs with i + 1
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wq(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// Each round: two 32x32->64 products (one wide multiply each), two
// three-input XORs; the key schedule is the same for every thread.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y,
                       (uint32_t)p0);
    }
    return c;
}

// Zero-mean unit-variance uniform variate from 32 random bits:
// sqrt(12) ((x + 1/2) 2^-32 - 1/2).
__device__ __forceinline__ double unit_uniform_d(uint32_t x) {
    return 3.4641016151377544 * (((double)x + 0.5) * 2.3283064365386963e-10 - 0.5);
}
// The centred 16-bit variate (h + 1/2) 2^-16 - 1/2 (times sqrt(12) for unit
// variance), exact in one FMA: h 2^-16 and 2^-17 - 1/2 are exact in FP64.
__device__ __forceinline__ double centred16_d(uint32_t h) {
    return fma((double)h, 0x1p-16, 0x1p-17 - 0.5);
}
__device__ __forceinline__ float unit_uniform_f(uint32_t x) {
    // (x - 2^31 + 1/2) 2^-32 with one integer-to-float conversion
    return 3.4641016151377544f * (((float)(int32_t)(x ^ 0x80000000u) + 0.5f) * 2.3283064365386963e-10f);
}

// ------------------------------------------------------------------ geometry
struct Geom {
    int nx, ny, nz;
    long long N;        // nodes = stride between population planes
    int pore_axis;      // -1: periodic box without walls
    long long pore_t;   // wall iff (2a+1-na)^2 + (2b+1-nb)^2 >= pore_t (a, b: coordinates across the axis)
    long long pore_in;  // below this the node and all its neighbours are fluid
    int chan;           // 1: moving walls at y = -1/2 and y = ny - 1/2, the box not periodic in y
    const double *wchan;  // device, chan: [2][19] bounce-back terms 6 w_i rho0 (c_i . u_wall) of the
                          // lower and upper wall, then [2][3] the wall velocities
    // Compact layout of a pore (batched pore instances; nullptr: the dense
    // layout): only fluid nodes are stored. A node at position p across the
    // axis (p = a + na b, (a, b) = (x, y), (x, z) or (y, z) for an axis z, y
    // or x) and coordinate l along it has index m = cmap[p] * csj + l * csa in
    // planes cps apart; cnbr[8 j + dir8(u, v)] is the compact position of the
    // in-plane neighbour (a + u, b + v) of compact position j (periodic),
    // 0xFFFF if that is a wall node: one 16-byte record per position, read
    // by one vector load.
    const int *cmap;
    const uint16_t *cnbr;
    long long cps;
    int csj, csa;
};

__device__ __forceinline__ int wrapm(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Index check of checked builds (-DLB_CHECKS, a stand-in for a memory
// sanitizer): an index outside [0, n) is replaced by 0, an in-bounds access,
// and bit 2 of the device error word is set (the host reports LB_ERR_STATE).
// Other builds return the index unchanged.
template <typename I>
__device__ __forceinline__ I chk(I i, long long n, int *err) {
#ifdef LB_CHECKS
    if ((long long)i < 0 || (long long)i >= n) {
        if (err) atomicOr(err, 2);
        return I(0);
    }
#endif
    return i;
}

__device__ __forceinline__ long long nidx(const Geom &g, int x, int y, int z) {
    return (long long)x + (long long)g.nx * ((long long)y + (long long)g.ny * z);
}

// squared doubled distance from the pore axis of the node centre
__device__ __forceinline__ long long pore_r2(const Geom &g, int x, int y, int z) {
    int a, b, na, nb;
    if (g.pore_axis == 0) { a = y; b = z; na = g.ny; nb = g.nz; }
    else if (g.pore_axis == 1) { a = x; b = z; na = g.nx; nb = g.nz; }
    else { a = x; b = y; na = g.nx; nb = g.ny; }
    const long long da = 2 * a + 1 - na, db = 2 * b + 1 - nb;
    return da * da + db * db;
}

__device__ __forceinline__ bool is_wall(const Geom &g, int x, int y, int z) {
    return g.pore_axis >= 0 && pore_r2(g, x, y, z) >= g.pore_t;
}

// Bounce-back term of a population of link i returning from the moving wall
// on `side` (0 lower, 1 upper): f_i = f*_opp(i) + 6 w_i rho0 (c_i . u_wall).
__device__ __forceinline__ double chan_term(const Geom &g, int side, int i) { return g.wchan[19 * side + i]; }

// Pre-collision population i of node (x,y,z) under the AA pattern.
// Even step count: stored in place, A[i][n]. Odd step count: the neighbour
// upstream holds it in the opposite slot, A[opp i][n - c_i]; if that
// neighbour is a wall node the population bounced back into A[i][n] (plus
// the moving-wall term when the wall is a channel wall).
template <typename T>
__device__ __forceinline__ T load_pre(const T *A, const Geom &g, int x, int y, int z, long long n,
                                      int i, bool odd) {
    if (!odd || i == 0) return A[(long long)i * g.N + n];
    const int yr = y - cy(i);
    if (g.chan && (yr < 0 || yr >= g.ny))
        return (T)((double)A[(long long)i * g.N + n] + chan_term(g, yr < 0 ? 0 : 1, i));
    const int xs = wrapm(x - cx(i), g.nx), ys = wrapm(yr, g.ny), zs = wrapm(z - cz(i), g.nz);
    if (is_wall(g, xs, ys, zs)) return A[(long long)i * g.N + n];
    return A[(long long)opp(i) * g.N + nidx(g, xs, ys, zs)];
}

// Store of population i so that the next load_pre returns it (inverse map).
template <typename T>
__device__ __forceinline__ void store_pre(T *A, const Geom &g, int x, int y, int z, long long n,
                                          int i, bool odd, T v) {
    if (!odd || i == 0) { A[(long long)i * g.N + n] = v; return; }
    const int yr = y - cy(i);
    if (g.chan && (yr < 0 || yr >= g.ny)) {
        A[(long long)i * g.N + n] = (T)((double)v - chan_term(g, yr < 0 ? 0 : 1, i));
        return;
    }
    const int xs = wrapm(x - cx(i), g.nx), ys = wrapm(yr, g.ny), zs = wrapm(z - cz(i), g.nz);
    if (is_wall(g, xs, ys, zs)) { A[(long long)i * g.N + n] = v; return; }
    A[(long long)opp(i) * g.N + nidx(g, xs, ys, zs)] = v;
}

// Slot of the in-plane direction (u, v) != (0, 0) in a position's record of
// 8 neighbours (compact layout).
__host__ __device__ constexpr int dir8(int u, int v) {
    return (u + 1) + 3 * (v + 1) < 4 ? (u + 1) + 3 * (v + 1) : (u + 1) + 3 * (v + 1) - 1;
}

// In-plane components (u, v) and the component along the pore axis of link
// i, for the compact layout.
__device__ __forceinline__ void link_axes(int axis, int i, int &u, int &v, int &al) {
    if (axis == 2) { u = cx(i); v = cy(i); al = cz(i); }
    else if (axis == 1) { u = cx(i); v = cz(i); al = cy(i); }
    else { u = cy(i); v = cz(i); al = cx(i); }
}

// Compact index of fluid node (x, y, z) and its position j across the axis
// and coordinate l along it.
__device__ __forceinline__ long long compact_node(const Geom &g, int x, int y, int z, int &j, int &l) {
    int a, b, na;
    if (g.pore_axis == 2) { a = x; b = y; na = g.nx; l = z; }
    else if (g.pore_axis == 1) { a = x; b = z; na = g.nx; l = y; }
    else { a = y; b = z; na = g.ny; l = x; }
    j = g.cmap[a + na * b];
    return (long long)j * g.csj + (long long)l * g.csa;
}

// load_pre and store_pre for the compact layout (fluid node (x, y, z)).
template <typename T>
__device__ __forceinline__ T compact_load_pre(const T *A, const Geom &g, int x, int y, int z, int i, bool odd) {
    int j, l;
    const long long m = compact_node(g, x, y, z, j, l);
    if (!odd || i == 0) return A[(long long)i * g.cps + m];
    int u, v, al;
    link_axes(g.pore_axis, i, u, v, al);
    const int js = (u == 0 && v == 0) ? j : (int)g.cnbr[8 * j + dir8(-u, -v)];
    if (js == 0xFFFF) return A[(long long)i * g.cps + m];
    const int nl = g.pore_axis == 2 ? g.nz : (g.pore_axis == 1 ? g.ny : g.nx);
    const int ls = wrapm(l - al, nl);
    return A[(long long)opp(i) * g.cps + (long long)js * g.csj + (long long)ls * g.csa];
}

template <typename T>
__device__ __forceinline__ void compact_store_pre(T *A, const Geom &g, int x, int y, int z, int i, bool odd, T val) {
    int j, l;
    const long long m = compact_node(g, x, y, z, j, l);
    if (!odd || i == 0) { A[(long long)i * g.cps + m] = val; return; }
    int u, v, al;
    link_axes(g.pore_axis, i, u, v, al);
    const int js = (u == 0 && v == 0) ? j : (int)g.cnbr[8 * j + dir8(-u, -v)];
    if (js == 0xFFFF) { A[(long long)i * g.cps + m] = val; return; }
    const int nl = g.pore_axis == 2 ? g.nz : (g.pore_axis == 1 ? g.ny : g.nx);
    const int ls = wrapm(l - al, nl);
    A[(long long)opp(i) * g.cps + (long long)js * g.csj + (long long)ls * g.csa] = val;
}

// 4x4x4 tiles flag where bead forces were spread
__device__ __forceinline__ long long tile_of(int x, int y, int z, int ntx, int nty) {
    return (long long)(x >> 2) + (long long)ntx * ((long long)(y >> 2) + (long long)nty * (z >> 2));
}

}  // namespace lbk
