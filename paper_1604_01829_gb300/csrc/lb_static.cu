// Allocation-free variant of the mass/momentum reduction (lb_moments_noalloc).
//
// Some callers cannot call cudaMalloc: a caller whose device memory is
// already reserved by another allocator (a caching allocator that holds the
// free memory), or a caller that must not make the device synchronise in the
// middle of a running simulation (cudaMalloc and cudaFree may synchronise).
// This entry point gives them the reduction with no allocation at all: its
// per-block partial sums live in a file-scope device array of fixed size.
//
// Limits and sharing: one partial per block of LB_NOALLOC_NODES_PER_BLOCK
// nodes, at most LB_NOALLOC_MAX_BLOCKS blocks, so lattices of more than
// LB_NOALLOC_MAX_NODES nodes are rejected. Every call on a device uses the
// same array; each block overwrites its own partial, so nothing needs
// clearing, but calls that overlap on the GPU (other streams, other host
// threads) race on it. The array's device address is looked up with the
// device current on every call made outside stream capture; a captured call
// uses the address of the device's last call outside capture.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerBlock = LB_NOALLOC_NODES_PER_BLOCK;
constexpr int kMaxBlocks = LB_NOALLOC_MAX_BLOCKS;

// The scratch: 4 partial sums per block. Host code must not pass this name to
// a kernel (in host code it is only a stand-in); it passes the address
// obtained from cudaGetSymbolAddress instead.
static __device__ __align__(256) double g_noalloc_partials[4 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_moments_blocks(const T *f, lbk::Geom g, bool odd, double *partials) {
    double s[4] = {0, 0, 0, 0};
    const long long first = (long long)blockIdx.x * kNodesPerBlock;
    const long long last = first + kNodesPerBlock < g.N ? first + kNodesPerBlock : g.N;
    for (long long n = first + threadIdx.x; n < last; n += kThreads) {
        const int x = (int)(n % g.nx);
        const long long r = n / g.nx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        if (lbk::is_wall(g, x, y, z)) continue;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const double v = (double)lbk::load_pre(f, g, x, y, z, n, i, odd);
            s[0] += v;
            if (lbk::cx(i)) s[1] += lbk::cx(i) * v;
            if (lbk::cy(i)) s[2] += lbk::cy(i) * v;
            if (lbk::cz(i)) s[3] += lbk::cz(i) * v;
        }
    }
    __shared__ double red[4][kThreads];
#pragma unroll
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) partials[4LL * blockIdx.x + c] = red[c][0];
}

__global__ void __launch_bounds__(kThreads) k_moments_sum(const double *partials, int nblocks, double mass_shift,
                                                          double *out) {
    __shared__ double red[4][kThreads];
    double s[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
        for (int c = 0; c < 4; ++c) s[c] += partials[4LL * b + c];
#pragma unroll
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0] + mass_shift;
        out[1] = red[1][0];
        out[2] = red[2][0];
        out[3] = red[3][0];
    }
}

struct ErrOut {
    char *buf;
    size_t len;
};

lb_status noalloc_fail(const ErrOut &eo, lb_status s, const std::string &m) {
    if (eo.buf && eo.len > 0) std::snprintf(eo.buf, eo.len, "%s", m.c_str());
    return s;
}

// Device address of the scratch array on the current device. Outside stream
// capture it is looked up on every call (a cheap host query), so an address
// cached before a reset of the device's primary context is never used
// again; while `s` is being captured the address cached by an earlier call
// on this device is used, and a capture with no earlier call is refused.
lb_status scratch_address(const ErrOut &eo, cudaStream_t s, double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(eo, LB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(eo, LB_ERR_ARG, "device ordinal out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    const bool capturing = e != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    if (e != cudaSuccess) (void)cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!capturing) {
        double *ptr = nullptr;
        e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_partials);
        if (e != cudaSuccess || !ptr)
            return noalloc_fail(eo, LB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch[dev] = ptr;
    } else if (!g_scratch[dev]) {
        return noalloc_fail(eo, LB_ERR_STATE,
                            "lb_moments_noalloc: the first call on a device must come before any stream capture");
    }
    *out = g_scratch[dev];
    return LB_OK;
}

}  // namespace

extern "C" lb_status lb_moments_noalloc(const void *d_populations, int precision, int nx, int ny, int nz,
                                        int odd_parity, double rho0, double pore_radius, int pore_axis,
                                        double *d_out, void *cuda_stream, char *err, size_t err_len) {
    const ErrOut eo{err, err_len};
    if (!d_populations || !d_out) return noalloc_fail(eo, LB_ERR_ARG, "null device pointer");
    if (precision != 32 && precision != 64) return noalloc_fail(eo, LB_ERR_ARG, "precision must be 32 or 64");
    if (nx < 2 || ny < 2 || nz < 2) return noalloc_fail(eo, LB_ERR_ARG, "lattice sizes must be >= 2");
    const long long N = (long long)nx * ny * nz;
    if (N > (long long)LB_NOALLOC_MAX_NODES)
        return noalloc_fail(eo, LB_ERR_ARG, "lattice of " + std::to_string(N) + " nodes exceeds the " +
                                            std::to_string((long long)LB_NOALLOC_MAX_NODES) +
                                            "-node limit of lb_moments_noalloc's static scratch");
    if (pore_radius > 0.0 && (pore_axis < 0 || pore_axis > 2))
        return noalloc_fail(eo, LB_ERR_ARG, "pore_axis must be 0, 1 or 2");
    lbk::Geom g{};
    g.nx = nx; g.ny = ny; g.nz = nz; g.N = N;
    g.pore_axis = -1;
    long long nfluid = N;
    if (pore_radius > 0.0) {
        g.pore_axis = pore_axis;
        g.pore_t = (long long)std::ceil(4.0 * (pore_radius * pore_radius));
        const int na = pore_axis == 0 ? ny : nx, nb = pore_axis == 2 ? ny : nz;
        const int nl = pore_axis == 0 ? nx : (pore_axis == 1 ? ny : nz);
        long long c = 0;
        for (int b = 0; b < nb; ++b)
            for (int a = 0; a < na; ++a) {
                const long long da = 2LL * a + 1 - na, db = 2LL * b + 1 - nb;
                if (da * da + db * db < g.pore_t) ++c;
            }
        nfluid = c * nl;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *scratch = nullptr;
    lb_status st = scratch_address(eo, s, &scratch);
    if (st != LB_OK) return st;
    const int nblocks = (int)((N + kNodesPerBlock - 1) / kNodesPerBlock);
    if (precision == 32)
        k_moments_blocks<float><<<nblocks, kThreads, 0, s>>>((const float *)d_populations, g, odd_parity != 0, scratch);
    else
        k_moments_blocks<double><<<nblocks, kThreads, 0, s>>>((const double *)d_populations, g, odd_parity != 0, scratch);
    k_moments_sum<<<1, kThreads, 0, s>>>(scratch, nblocks, precision == 32 ? rho0 * (double)nfluid : 0.0, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(eo, LB_ERR_CUDA, std::string("lb_moments_noalloc launch: ") + cudaGetErrorString(e));
    if (eo.buf && eo.len > 0) eo.buf[0] = '\0';
    return LB_OK;
}
