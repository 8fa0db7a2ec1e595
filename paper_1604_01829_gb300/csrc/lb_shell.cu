// Raspberry shell construction on the GPU (Ustach & Faller, arXiv:1604.01829,
// Sec. 2.1 and the SI section "Details for ellipsoidal raspberry
// construction").
//
// Beads of one shell relax on an ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1
// under two forces: a harmonic pull -2k (r - r_s) towards the nearest surface
// point r_s, and pairwise WCA repulsion between the beads of the shell. The
// nearest point follows from the normal condition r - r_s = (t/2) grad S(r_s),
// i.e. r_s = (x a^2/(t + a^2), ...) (Eq. (xtoxs)), with t the root of
// F(t) = sum (x a/(t + a^2))^2 - 1 (Eq. (bisection) read without its printed
// "+1", which contradicts Eq. (xtoxs)). F decreases for t > -m^2 (m the
// smallest semi-axis); the root lies in [-m^2 + m |x_m|, a_max |r|], where the
// term of the smallest axis alone is 1 at the lower end and F <= 0 at the
// upper end. The paper stops its bisection at |F| < 1e-6; here the bracket is
// halved a fixed number of times (64 in FP64, 40 in FP32), which is tighter.
// Integration: damped leapfrog with unit mass, v <- (1 - eta dt) v + dt F,
// r <- r + dt v.
//
// Design: one thread block per shell, the shell's positions and velocities in
// shared memory (structure of arrays, 6 n values: 192 KB for 4096 beads in
// FP64), each thread owning up to 4 beads. A step reads every position once per owned
// bead group (shared-memory broadcast: all lanes of a warp read the same j),
// then, after a barrier, each thread moves its beads. Shells are independent,
// so many of them fill the GPU in one launch.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lb.h"
#include "lb_device.cuh"

namespace lbk {

namespace {

constexpr int kShellThreads = 1024;
constexpr int kMaxCells = 4096;                     // cells per shell at most
constexpr int kCellsFrom = 256;                     // automatic pair search: cell list from this many beads
constexpr double kWcaCut = 1.122462048309373;      // 2^(1/6)

template <typename R>
struct ShellArgs {
    const double *axes;       // [nshells][3]
    const int *count;         // [nshells]
    const long long *offset;  // [nshells] first bead of each shell
    double *xyz;              // [total][3], in and out
    int max_count;            // largest shell (shared-memory extent)
    R k2;                     // 2k
    R sig2, rc2, eps24;       // sigma^2, (2^(1/6) sigma)^2, 24 epsilon
    R dt, damp;               // dt, 1 - eta dt
    long long steps;
    int project_final;
    // cell list (CELLS kernels): per shell the grid g[3] over the box
    // [-L, L) per axis (L = box[3 s + q]) with cells of size >= the WCA range
    const int *cgrid;         // [nshells][3]
    const double *cbox;       // [nshells][3] half-widths L
    int max_cells;            // largest grid (shared-memory extent)
    int *err;                 // index checks of checked builds (LB_CHECKS): bit 2 on failure
};

__device__ __forceinline__ float rdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return a / b; }

// Nearest surface point of (x, y, z): bisection for the root of F(t).
template <typename R>
__device__ __forceinline__ void surface_point(R x, R y, R z, R a, R b, R c, R &sx, R &sy, R &sz) {
    constexpr int H = sizeof(R) == 8 ? 64 : 40;
    const R m = fmin(a, fmin(b, c));
    R xm = R(0);
    if (a == m) xm = fmax(xm, fabs(x));
    if (b == m) xm = fmax(xm, fabs(y));
    if (c == m) xm = fmax(xm, fabs(z));
    R lo = -m * m + m * xm;
    R hi = fmax(a, fmax(b, c)) * sqrt(x * x + y * y + z * z);
    if (hi < lo) hi = lo;
    const R a2 = a * a, b2 = b * b, c2 = c * c, xa = x * a, yb = y * b, zc = z * c;
    for (int it = 0; it < H; ++it) {
        const R mid = R(0.5) * (lo + hi);
        const R u = rdiv(xa, mid + a2), v = rdiv(yb, mid + b2), w = rdiv(zc, mid + c2);
        if (u * u + v * v + w * w - R(1) > R(0)) lo = mid;
        else hi = mid;
    }
    const R t = R(0.5) * (lo + hi);
    const R da = t + a2, db = t + b2, dc = t + c2;
    // a denominator vanishes only when the bracket collapsed onto -m^2 (a bead
    // on the medial set inside, without a unique nearest point): component 0
    sx = da > R(0) ? rdiv(x * a2, da) : R(0);
    sy = db > R(0) ? rdiv(y * b2, db) : R(0);
    sz = dc > R(0) ? rdiv(z * c2, dc) : R(0);
}

// Block-wide exclusive scan of cnt[0..C) into start[0..C] (start[C] = total),
// resetting cnt to 0 (it then serves as the fill cursor). wsum: 32 ints.
__device__ __forceinline__ void scan_cells(int *cnt, int *start, int C, int *wsum) {
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (C + T - 1) / T;
    const int c0 = min(C, tid * per), c1 = min(C, c0 + per);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += cnt[c];
    int v = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < ((T + 31) >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int base = v - sum + (warp > 0 ? wsum[warp - 1] : 0);
    for (int c = c0; c < c1; ++c) {
        start[c] = base;
        base += cnt[c];
        cnt[c] = 0;
    }
    if (tid == T - 1) start[C] = base;
}

// One block per shell. CELLS: pair search through a cell list rebuilt every
// step (counting sort by cell, beads of a cell in index order, so results do
// not depend on the order of the atomics); a step in which a bead lies
// outside the grid's box searches all pairs instead. Without CELLS every
// step tests all pairs, summed in index order.
template <typename R, int BPT, bool CELLS>
__global__ void __launch_bounds__(kShellThreads) k_relax_shells(const ShellArgs<R> a) {
    extern __shared__ unsigned char smem_raw[];
    R *px = reinterpret_cast<R *>(smem_raw);
    R *py = px + a.max_count;
    R *pz = py + a.max_count;
    R *vx = pz + a.max_count;              // velocities
    R *vy = vx + a.max_count;
    R *vz = vy + a.max_count;
    int *bcell = reinterpret_cast<int *>(vz + a.max_count);   // CELLS: cell of each bead
    int *sorted = bcell + a.max_count;                        // bead indices by cell
    int *cnt = sorted + a.max_count;                          // per cell count / cursor
    int *start = cnt + a.max_cells;                           // per cell first slot (+1)
    __shared__ int wsum[32];
    const int s = blockIdx.x;
    const int n = a.count[s];
    double *X = a.xyz + 3 * a.offset[s];
    const R ax = (R)a.axes[3 * s], ay = (R)a.axes[3 * s + 1], az = (R)a.axes[3 * s + 2];
    int gx = 1, gy = 1, gz = 1, C = 1;
    R Lx = R(0), Ly = R(0), Lz = R(0), ihx = R(0), ihy = R(0), ihz = R(0);
    if (CELLS) {
        gx = a.cgrid[3 * s]; gy = a.cgrid[3 * s + 1]; gz = a.cgrid[3 * s + 2];
        C = gx * gy * gz;
        Lx = (R)a.cbox[3 * s]; Ly = (R)a.cbox[3 * s + 1]; Lz = (R)a.cbox[3 * s + 2];
        ihx = (R)gx / (R(2) * Lx); ihy = (R)gy / (R(2) * Ly); ihz = (R)gz / (R(2) * Lz);
        for (int c = threadIdx.x; c < C; c += blockDim.x) cnt[c] = 0;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        px[i] = (R)X[3 * i];
        py[i] = (R)X[3 * i + 1];
        pz[i] = (R)X[3 * i + 2];
        vx[i] = vy[i] = vz[i] = R(0);
    }
    __syncthreads();

    for (long long step = 0; step < a.steps; ++step) {
        R xi[BPT], yi[BPT], zi[BPT], fx[BPT], fy[BPT], fz[BPT];
        int id[BPT];
        bool outside = false;
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int i = threadIdx.x + b * blockDim.x;
            id[b] = i < n ? i : -1;
            xi[b] = yi[b] = zi[b] = fx[b] = fy[b] = fz[b] = R(0);
            if (i < n) {
                xi[b] = px[i];
                yi[b] = py[i];
                zi[b] = pz[i];
                if (CELLS) {
                    const int cx = (int)floor((xi[b] + Lx) * ihx), cy = (int)floor((yi[b] + Ly) * ihy),
                              cz = (int)floor((zi[b] + Lz) * ihz);
                    if (cx < 0 || cx >= gx || cy < 0 || cy >= gy || cz < 0 || cz >= gz) {
                        outside = true;
                        bcell[i] = -1;
                    } else {
                        const int c = chk(cx + gx * (cy + gy * cz), C, a.err);
                        bcell[i] = c;
                        atomicAdd(&cnt[c], 1);
                    }
                }
                R sx, sy, sz;
                surface_point(xi[b], yi[b], zi[b], ax, ay, az, sx, sy, sz);
                fx[b] = -a.k2 * (xi[b] - sx);
                fy[b] = -a.k2 * (yi[b] - sy);
                fz[b] = -a.k2 * (zi[b] - sz);
            }
        }
        auto pair = [&](int b, int j) {
            const R dx = xi[b] - px[j], dy = yi[b] - py[j], dz = zi[b] - pz[j];
            const R r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < a.rc2 && j != id[b]) {
                const R s2 = rdiv(a.sig2, r2);
                const R s6 = s2 * s2 * s2;
                const R fm = rdiv(a.eps24 * (R(2) * s6 * s6 - s6), r2);
                fx[b] += fm * dx;
                fy[b] += fm * dy;
                fz[b] += fm * dz;
            }
        };
        bool use_cells = false;
        if (CELLS) {
            use_cells = !__syncthreads_or(outside);
            if (use_cells) {
                scan_cells(cnt, start, C, wsum);
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x)
                    sorted[chk(start[bcell[i]] + atomicAdd(&cnt[bcell[i]], 1), n, a.err)] = i;
                __syncthreads();
                // beads of each cell in index order (few per cell: insertion sort)
                for (int c = threadIdx.x; c < C; c += blockDim.x) {
                    for (int k = start[c] + 1; k < start[c + 1]; ++k) {
                        const int v = sorted[k];
                        int m = k - 1;
                        while (m >= start[c] && sorted[m] > v) {
                            sorted[m + 1] = sorted[m];
                            --m;
                        }
                        sorted[m + 1] = v;
                    }
                }
                __syncthreads();
            } else {
                for (int c = threadIdx.x; c < C; c += blockDim.x) cnt[c] = 0;
            }
        }
        if (use_cells) {
            // WCA over the 27 cells around each bead (cells are at least as wide as the range)
#pragma unroll
            for (int b = 0; b < BPT; ++b) {
                if (id[b] < 0) continue;
                const int c = bcell[id[b]];
                const int cx = c % gx, cy = (c / gx) % gy, cz = c / (gx * gy);
                for (int dz = -1; dz <= 1; ++dz) {
                    const int z = cz + dz;
                    if (z < 0 || z >= gz) continue;
                    for (int dy = -1; dy <= 1; ++dy) {
                        const int y = cy + dy;
                        if (y < 0 || y >= gy) continue;
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int x = cx + dx;
                            if (x < 0 || x >= gx) continue;
                            const int cc = x + gx * (y + gy * z);
                            for (int k = start[cc]; k < start[cc + 1]; ++k) pair(b, chk(sorted[k], n, a.err));
                        }
                    }
                }
            }
        } else {
            // pairwise WCA, summed over j in index order (one read of j for all owned beads)
            for (int j = 0; j < n; ++j) {
                const R xj = px[j], yj = py[j], zj = pz[j];
#pragma unroll
                for (int b = 0; b < BPT; ++b) {
                    const R dx = xi[b] - xj, dy = yi[b] - yj, dz = zi[b] - zj;
                    const R r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < a.rc2 && j != id[b] && id[b] >= 0) {
                        const R s2 = rdiv(a.sig2, r2);
                        const R s6 = s2 * s2 * s2;
                        const R fm = rdiv(a.eps24 * (R(2) * s6 * s6 - s6), r2);
                        fx[b] += fm * dx;
                        fy[b] += fm * dy;
                        fz[b] += fm * dz;
                    }
                }
            }
        }
        __syncthreads();   // every thread has read every position of this step
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int i = id[b];
            if (i < 0) continue;
            const R ux = a.damp * vx[i] + a.dt * fx[b];
            const R uy = a.damp * vy[i] + a.dt * fy[b];
            const R uz = a.damp * vz[i] + a.dt * fz[b];
            vx[i] = ux;
            vy[i] = uy;
            vz[i] = uz;
            px[i] = xi[b] + a.dt * ux;
            py[i] = yi[b] + a.dt * uy;
            pz[i] = zi[b] + a.dt * uz;
        }
        if (CELLS && use_cells)
            for (int c = threadIdx.x; c < C; c += blockDim.x) cnt[c] = 0;
        __syncthreads();   // positions of the next step are complete
    }

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        R x = px[i], y = py[i], z = pz[i];
        if (a.project_final) {
            R sx, sy, sz;
            surface_point(x, y, z, ax, ay, az, sx, sy, sz);
            x = sx;
            y = sy;
            z = sz;
        }
        X[3 * i] = (double)x;
        X[3 * i + 1] = (double)y;
        X[3 * i + 2] = (double)z;
    }
}

size_t shell_smem(size_t rsize, int max_count, int max_cells, bool cells) {
    return 6 * rsize * (size_t)max_count + (cells ? sizeof(int) * (2 * (size_t)max_count + 2 * (size_t)max_cells + 1) : 0);
}

template <typename R, int BPT, bool CELLS>
cudaError_t launch_shells_t(const ShellArgs<R> &a, int nshells, int threads, cudaStream_t s) {
    const size_t smem = shell_smem(sizeof(R), a.max_count, a.max_cells, CELLS);
    cudaError_t e = cudaFuncSetAttribute(k_relax_shells<R, BPT, CELLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_relax_shells<R, BPT, CELLS><<<nshells, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_shells(ShellArgs<R> a, const lb_shell_params &p, int nshells, bool cells, cudaStream_t s) {
    a.k2 = (R)(2.0 * p.k_surface);
    a.sig2 = (R)(p.sigma * p.sigma);
    a.rc2 = (R)(kWcaCut * kWcaCut * p.sigma * p.sigma);
    a.eps24 = (R)(24.0 * p.epsilon);
    a.dt = (R)p.dt;
    a.damp = (R)(1.0 - p.eta * p.dt);
    a.steps = p.steps;
    a.project_final = p.project_final;
    // beads per thread: 1, 2 or 4; threads a multiple of the warp
    const int bpt = a.max_count <= kShellThreads ? 1 : (a.max_count <= 2 * kShellThreads ? 2 : 4);
    int threads = (a.max_count + bpt - 1) / bpt;
    threads = ((threads + 31) / 32) * 32;
    if (cells) {
        if (bpt == 1) return launch_shells_t<R, 1, true>(a, nshells, threads, s);
        if (bpt == 2) return launch_shells_t<R, 2, true>(a, nshells, threads, s);
        return launch_shells_t<R, 4, true>(a, nshells, threads, s);
    }
    if (bpt == 1) return launch_shells_t<R, 1, false>(a, nshells, threads, s);
    if (bpt == 2) return launch_shells_t<R, 2, false>(a, nshells, threads, s);
    return launch_shells_t<R, 4, false>(a, nshells, threads, s);
}

}  // namespace

}  // namespace lbk

extern "C" lb_status lb_relax_shells(int nshells, const double *axes, const int *counts, double *xyz,
                                     const lb_shell_params *p, void *cuda_stream, char *err, size_t err_len) {
    auto fail = [&](lb_status st, const std::string &m) {
        if (err && err_len) {
            std::strncpy(err, m.c_str(), err_len - 1);
            err[err_len - 1] = 0;
        }
        return st;
    };
    if (!axes || !counts || !xyz || !p) return fail(LB_ERR_ARG, "null pointer");
    if (nshells < 1 || nshells > 65535) return fail(LB_ERR_ARG, "nshells must be in [1, 65535]");
    if (p->precision != 32 && p->precision != 64) return fail(LB_ERR_ARG, "precision must be 32 or 64");
    if (!(p->k_surface > 0.0) || !(p->sigma > 0.0) || !(p->epsilon > 0.0) || !(p->dt > 0.0) || !(p->eta >= 0.0) ||
        !(p->eta * p->dt <= 2.0) || p->steps < 0 || !std::isfinite(p->k_surface) || !std::isfinite(p->sigma) ||
        !std::isfinite(p->epsilon) || !std::isfinite(p->dt) || !std::isfinite(p->eta))
        return fail(LB_ERR_ARG, "need k, sigma, epsilon, dt > 0, eta >= 0, eta dt <= 2 and steps >= 0");
    if (p->pair_search < 0 || p->pair_search > 2) return fail(LB_ERR_ARG, "pair_search must be 0, 1 or 2");
    std::vector<long long> off(nshells);
    long long total = 0;
    int max_count = 0;
    for (int s = 0; s < nshells; ++s) {
        if (counts[s] < 1 || counts[s] > LB_SHELL_MAX_BEADS)
            return fail(LB_ERR_ARG, "every shell needs 1 to LB_SHELL_MAX_BEADS (4096) beads");
        for (int q = 0; q < 3; ++q)
            if (!(axes[3 * s + q] > 0.0) || !std::isfinite(axes[3 * s + q]))
                return fail(LB_ERR_ARG, "semi-axes must be positive and finite");
        off[s] = total;
        total += counts[s];
        if (counts[s] > max_count) max_count = counts[s];
    }
    for (long long i = 0; i < 3 * total; ++i)
        if (!std::isfinite(xyz[i])) return fail(LB_ERR_ARG, "initial positions must be finite");

    // cell grids: per axis the box [-L, L), L = 1.25 a + 1, cut into cells at
    // least as wide as the WCA range, at most kMaxCells cells per shell
    const double rc = lbk::kWcaCut * p->sigma;
    std::vector<int> grid((size_t)3 * nshells);
    std::vector<double> box((size_t)3 * nshells);
    int max_cells = 1;
    for (int s = 0; s < nshells; ++s) {
        long long g[3];
        for (int q = 0; q < 3; ++q) {
            box[3 * s + q] = 1.25 * axes[3 * s + q] + 1.0;
            g[q] = std::max(1LL, (long long)std::floor(2.0 * box[3 * s + q] / rc));
            g[q] = std::min(g[q], 4096LL);
        }
        while (g[0] * g[1] * g[2] > lbk::kMaxCells) {
            const int q = g[0] >= g[1] && g[0] >= g[2] ? 0 : (g[1] >= g[2] ? 1 : 2);
            g[q] = std::max(1LL, (g[q] * 7) / 8);
        }
        for (int q = 0; q < 3; ++q) grid[3 * s + q] = (int)g[q];
        max_cells = std::max(max_cells, (int)(g[0] * g[1] * g[2]));
    }
    const size_t rsize = p->precision == 64 ? sizeof(double) : sizeof(float);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
    const bool cells_fit = lbk::shell_smem(rsize, max_count, max_cells, true) <= (size_t)optin;
    if (p->pair_search == 2 && !cells_fit)
        return fail(LB_ERR_ARG, "the cell list does not fit in shared memory for this shell size and precision");
    if (lbk::shell_smem(rsize, max_count, 1, false) > (size_t)optin)
        return fail(LB_ERR_ARG, "the shell does not fit in shared memory at this precision");
    // automatic: the cell list pays off when a block per shell is latency-bound
    // (few shells for the SMs) or the shells are large; many small shells fill
    // the GPU and are faster testing all pairs (measured on GB300)
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 1;
    const bool auto_cells = max_count >= 1024 || (max_count >= lbk::kCellsFrom && nshells <= 2 * nsm);
    const bool cells = p->pair_search == 2 || (p->pair_search == 0 && auto_cells && cells_fit);

    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t nd = (size_t)3 * nshells + (size_t)3 * total + (size_t)3 * nshells;
    const size_t bytes = nd * sizeof(double) + (size_t)nshells * (sizeof(long long) + sizeof(int) + 3 * sizeof(int)) +
                         sizeof(int);
    void *d = nullptr;
    e = cudaMalloc(&d, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(LB_ERR_OOM, "device allocation for the shells failed");
    }
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    double *daxes = static_cast<double *>(d), *dxyz = daxes + 3 * nshells, *dbox = dxyz + 3 * total;
    long long *doff = reinterpret_cast<long long *>(dbox + 3 * nshells);
    int *dcount = reinterpret_cast<int *>(doff + nshells);
    int *dgrid = dcount + nshells;
    int *derr = dgrid + 3 * nshells;             // index checks of checked builds
    std::vector<double> out((size_t)3 * total);
    e = cudaMemcpyAsync(daxes, axes, 3 * nshells * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dxyz, xyz, 3 * total * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(doff, off.data(), nshells * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dcount, counts, nshells * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbox, box.data(), 3 * nshells * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dgrid, grid.data(), 3 * nshells * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        if (p->precision == 64) {
            lbk::ShellArgs<double> a{};
            a.axes = daxes; a.count = dcount; a.offset = doff; a.xyz = dxyz; a.max_count = max_count;
            a.cgrid = dgrid; a.cbox = dbox; a.max_cells = cells ? max_cells : 1; a.err = derr;
            e = lbk::launch_shells<double>(a, *p, nshells, cells, st);
        } else {
            lbk::ShellArgs<float> a{};
            a.axes = daxes; a.count = dcount; a.offset = doff; a.xyz = dxyz; a.max_count = max_count;
            a.cgrid = dgrid; a.cbox = dbox; a.max_cells = cells ? max_cells : 1; a.err = derr;
            e = lbk::launch_shells<float>(a, *p, nshells, cells, st);
        }
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), dxyz, 3 * total * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("lb_relax_shells: ") + cudaGetErrorString(e));
    if (herr) return fail(LB_ERR_STATE, "an index check of the checked build failed (an index outside its array)");
    for (double v : out)
        if (!std::isfinite(v)) return fail(LB_ERR_UNSTABLE, "non-finite bead position: reduce dt or k");
    std::memcpy(xyz, out.data(), out.size() * sizeof(double));
    return LB_OK;
}
