// Fused collide-and-stream for FP32 deviation storage with TMA-staged loads
// (periodic boxes, nx a multiple of 4).
//
// Same step as k_collide_stream (Sec. 1.1 of Ustach & Faller,
// arXiv:1604.01829: collision towards equilibrium plus streaming along the
// links, in place with the AA pattern), but the loads of one x-row of nodes
// (19 planes x nx values) are fetched by the tensor-memory accelerator with
// bulk copies into a multi-stage shared-memory ring while the CTA computes
// the previous rows. The bytes in flight per SM are then set by the ring
// depth, not by how many warps the register budget admits.
//
// Which row segments a row needs: on an even step the node's own slots, so
// plane i of the row itself; on an odd step the population arriving along
// link i sits in slot opp(i) of the upstream node x - c_i, i.e. in plane
// opp(i) of row (y - c_y, z - c_z), shifted by -c_x along the row. The whole
// upstream row segment is copied and the shift (with periodic wrap in x) is
// applied when reading shared memory. Every slot a row reads belongs to a
// node of that row and is written back by the same thread, so the in-place
// update stays race-free although the reads happen rows ahead.
//
// Bounded waits: one thread per CTA waits on each stage's mbarrier with a
// clock limit (lb_set_wait_limit, default ~2 s); on expiry it records an
// error code for the host, the CTA stops, and before leaving it waits (bounded
// by ~2 s whatever the limit) for its own copies still in flight.
#include "lb_collide.cuh"

namespace lbk {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// global -> shared bulk copy; completion is counted on the mbarrier in bytes
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// wait with a limit in SM clock cycles; false on expiry
constexpr long long kDrainLimit = 4000000000LL;     // ~2 s: copies in flight after an abort
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

constexpr int kThreads = 256;
#ifndef LB_TMA_MINB
#define LB_TMA_MINB 2
#endif

template <int COLL, bool NOISE, bool ODD>
__global__ void __launch_bounds__(kThreads, LB_TMA_MINB)
    k_collide_stream_tma(const FluidArgs a, int stages, long long wait_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int abort_flag;
    const Geom &g = a.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int rows = ny * nz;
    const unsigned N32 = (unsigned)g.N;
    float *A = static_cast<float *>(a.f);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *ring = reinterpret_cast<float *>(smem + 128);
    const uint32_t row_bytes = (uint32_t)nx * 4u;
    const uint32_t stage_bytes = 19u * row_bytes;

    const int G = gridDim.x;
    const int r0 = blockIdx.x;
    const int mine = r0 < rows ? (rows - r0 + G - 1) / G : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int k) {  // thread 0: fetch the row segments of local row k
        const int row = r0 + k * G;
        const int s = k % stages;
        const int y = row % ny, z = row / ny;
        float *dst = ring + (size_t)s * 19 * nx;
        mbar_arrive_expect_tx(&bars[s], stage_bytes);
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float *src;
            if (!ODD || i == 0) {
                src = A + (size_t)i * N32 + (size_t)row * nx;
            } else {
                int ys = y - cy(i), zs = z - cz(i);
                ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
                zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
                src = A + (size_t)opp(i) * N32 + ((size_t)zs * ny + ys) * nx;
            }
            bulk_g2s(dst + (size_t)i * nx, src, row_bytes, &bars[s]);
        }
    };

    const int prefetch = mine < stages ? mine : stages;
    if (threadIdx.x == 0)
        for (int k = 0; k < prefetch; ++k) issue(k);

    const float g0 = __ldg(a.gforce_f), g1 = __ldg(a.gforce_f + 1), g2 = __ldg(a.gforce_f + 2);
    int done = 0;
    for (int k = 0; k < mine; ++k) {
        const int s = k % stages;
        if (threadIdx.x == 0 && !mbar_wait_bounded(&bars[s], (uint32_t)((k / stages) & 1), wait_limit)) {
            abort_flag = 1;
            if (a.err) atomicExch(a.err, 1);
        }
        __syncthreads();
        if (abort_flag) break;
        const float *sb = ring + (size_t)s * 19 * nx;
        const int row = r0 + k * G;
        const int y = row % ny, z = row / ny;
        const int ym = (y == 0 ? ny - 1 : y - 1) * nx, y0 = y * nx, yp = (y == ny - 1 ? 0 : y + 1) * nx;
        const int nxy = nx * ny;
        const int zm = (z == 0 ? nz - 1 : z - 1) * nxy, z0 = z * nxy, zp = (z == nz - 1 ? 0 : z + 1) * nxy;
        for (int x = threadIdx.x; x < nx; x += kThreads) {
            const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
            float f[19];
            if (!ODD) {
#pragma unroll
                for (int i = 0; i < 19; ++i) f[i] = sb[i * nx + x];
            } else {
                f[0] = sb[x];
#pragma unroll
                for (int i = 1; i < 19; ++i) {
                    const int xs = cx(i) > 0 ? xm : (cx(i) < 0 ? xp : x);
                    f[i] = sb[i * nx + xs];
                }
            }
            const unsigned n = (unsigned)(x + y0 + z0);
            float Fx = g0, Fy = g1, Fz = g2;
            if (a.tiles && a.tiles[tile_of(x, y, z, a.ntx, a.nty)]) {
                const float *Fn = static_cast<const float *>(a.Fn);
                Fx += Fn[n];
                Fy += Fn[(size_t)N32 + n];
                Fz += Fn[2 * (size_t)N32 + n];
            }
            uint32_t step = 0;
            if (NOISE) step = (uint32_t)(*a.step_base) + a.step_off;
            collide_fp32<COLL, NOISE>(f, Fx, Fy, Fz, a.pf, a, n, step);
            if (!ODD) {
#pragma unroll
                for (int i = 0; i < 19; ++i) A[(size_t)opp(i) * N32 + n] = f[i];
            } else {
                A[n] = f[0];
                const int X3[3] = {xm, x, xp}, Y3[3] = {ym, y0, yp}, Z3[3] = {zm, z0, zp};
#pragma unroll
                for (int i = 1; i < 19; ++i)
                    A[(size_t)i * N32 + (unsigned)(X3[1 + cx(i)] + Y3[1 + cy(i)] + Z3[1 + cz(i)])] = f[i];
            }
        }
        __syncthreads();   // every thread is done reading stage s
        ++done;
        if (threadIdx.x == 0 && k + stages < mine) issue(k + stages);
    }
    // after an abort, let this CTA's copies still in flight land before leaving
    if (threadIdx.x == 0 && abort_flag) {
        const int issued = mine < done + stages ? mine : done + stages;
        for (int k = done; k < issued; ++k)
            mbar_wait_bounded(&bars[k % stages], (uint32_t)((k / stages) & 1), kDrainLimit);
    }
}

template <int COLL, bool NOISE>
cudaError_t launch_tma_t(const FluidArgs &a, bool odd, int stages, int grid, size_t smem, long long wait_limit,
                         cudaStream_t s) {
    auto kern = odd ? k_collide_stream_tma<COLL, NOISE, true> : k_collide_stream_tma<COLL, NOISE, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kThreads, smem, s>>>(a, stages, wait_limit);
    return cudaGetLastError();
}

}  // namespace

bool tma_collide_supported(const Geom &g, bool fp32) {
    return fp32 && g.pore_axis < 0 && g.nx % 4 == 0 && g.nx <= 1024 && g.N % 4 == 0;
}

cudaError_t launch_collide_stream_tma(const FluidArgs &a, int collision, bool noise, bool odd, int stages_hint,
                                      int ctas_per_sm_hint, long long wait_limit, cudaStream_t s) {
    if (!tma_collide_supported(a.g, true)) return cudaErrorNotSupported;
    const size_t row_stage = 19ull * a.g.nx * 4ull;
    int stages = stages_hint > 0 ? stages_hint : (int)(100000 / row_stage);
    if (stages < 2) stages = 2;
    if (stages > 6) stages = 6;
    const size_t smem = 128 + (size_t)stages * row_stage;
    if (smem > 220 * 1024) return cudaErrorNotSupported;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = ctas_per_sm_hint > 0 ? ctas_per_sm_hint : (int)((224 * 1024) / (smem + 1024));
    const int rows = a.g.ny * a.g.nz;
    int grid = sms * (per_sm > 0 ? per_sm : 1);
    if (grid > rows) grid = rows;
    if (wait_limit <= 0) wait_limit = kDrainLimit;
    if (collision == 0) return launch_tma_t<0, false>(a, odd, stages, grid, smem, wait_limit, s);
    if (noise) return launch_tma_t<1, true>(a, odd, stages, grid, smem, wait_limit, s);
    return launch_tma_t<1, false>(a, odd, stages, grid, smem, wait_limit, s);
}

}  // namespace lbk
