// Trajectory analysis of rigid raspberries on the GPU (Ustach & Faller,
// arXiv:1604.01829, Sec. 2.4-2.7 and the SI sections "Body-frame
// translational displacement" and "Body-frame angular displacement").
//
// Input: per body, nrec recorded centres X_k and orientations q_k (unit
// quaternions, Hamilton convention, lab = R(q) body) at a fixed interval.
// Per body and lag l (in records) the kernels average over all time origins
//   0-2  (X_{t+l} - X_t)_a^2 per lab axis                      Eq. (dt_lab)
//   3-5  (X^b_{t+l} - X^b_t)_a^2 per body axis, with the body-frame trajectory
//        X^b_n = sum_{k<=n} R(q_{k-1})^T (X_k - X_{k-1})       Eqs. (labdisp),
//        (quat), (bodyframedisplacement), (bodyframetrajectory), (dt_body)
//   6    Theta^2, Theta the angle between p(t) and p(t+l), p = R(q) p_ref
//                                                                Eq. (delta_theta)
//   7-9  (Theta_a(t+l) - Theta_a(t))^2, Theta_a the summed body-frame angular
//        displacements about body axis a by the projection method of the SI
//                                     Eqs. (bodyframerotdisplacement),
//                                     (bodyframerottrajectory), (dr_body)
// Readings: the body-frame displacement over an interval uses the
// orientation at its start; the angle of the projected axis is taken with
// atan2, equal to the printed arctangent of the component ratio for
// rotations below 90 degrees per interval; the lab-frame angle is computed
// as atan2(|p x p'|, p . p'), the same angle as the printed arccosine of the
// dot product of the unit vectors without its loss of precision at small
// angles.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_rigid.cuh"

namespace lbk {

namespace {

constexpr int kW = 9;   // work per (body, record): p-hat, body-frame trajectory, body-frame angles

__device__ __forceinline__ double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ void axes_of(const double *q, double ax[3][3]) {
    double R[9];
    quat_to_R(q, R);
    for (int c = 0; c < 3; ++c)            // body axis c in the lab frame: column c of R
        for (int r = 0; r < 3; ++r) ax[c][r] = R[3 * r + c];
}

// one thread per (body, record): unit reference vector, increments of the
// body-frame trajectory and of the body-frame angles over [k-1, k]
__global__ void k_msd_prep(const double *X, const double *q, int nrec, int nb, const double *p_ref, double *work) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nrec * nb) return;
    const int b = (int)(t / nrec), k = (int)(t % nrec);
    const double *qk = q + ((long long)b * nrec + k) * 4;
    double ak[3][3];
    axes_of(qk, ak);
    double *w = work + t * kW;
    const double pn = sqrt(dot3(p_ref, p_ref));
    for (int r = 0; r < 3; ++r) w[r] = (ak[0][r] * p_ref[0] + ak[1][r] * p_ref[1] + ak[2][r] * p_ref[2]) / pn;
    if (k == 0) {
        for (int c = 3; c < kW; ++c) w[c] = 0.0;
        return;
    }
    double ap[3][3];
    axes_of(qk - 4, ap);
    const double *Xk = X + ((long long)b * nrec + k) * 3;
    const double d[3] = {Xk[0] - Xk[-3], Xk[1] - Xk[-2], Xk[2] - Xk[-1]};
    for (int c = 0; c < 3; ++c) w[3 + c] = dot3(ap[c], d);
    // i, j, k of step k against those of step k-1 (projection method)
    w[6] = atan2(dot3(ak[2], ap[1]), dot3(ak[2], ap[2]));
    w[7] = atan2(dot3(ak[0], ap[2]), dot3(ak[0], ap[0]));
    w[8] = atan2(dot3(ak[1], ap[0]), dot3(ak[1], ap[1]));
}

// one thread per (body, column 3..8): running sums over the records, in order
__global__ void k_msd_scan(int nrec, int nb, double *work) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 6) return;
    const int b = t / 6, c = 3 + t % 6;
    double *w = work + (long long)b * nrec * kW + c;
    double s = 0.0;
    for (int k = 0; k < nrec; ++k) {
        s += w[(long long)k * kW];
        w[(long long)k * kW] = s;
    }
}

constexpr int kThreads = 256;

// one block per (lag, body): averages over all time origins
__global__ void __launch_bounds__(kThreads) k_msd_lags(const double *X, int nrec, int nb, int max_lag,
                                                     const double *work, double *out) {
    const int l = blockIdx.x + 1, b = blockIdx.y;
    const int n = nrec - l;
    double acc[LB_MSD_COLS];
    for (int c = 0; c < LB_MSD_COLS; ++c) acc[c] = 0.0;
    const double *Xb = X + (long long)b * nrec * 3;
    const double *wb = work + (long long)b * nrec * kW;
    for (int t = threadIdx.x; t < n; t += kThreads) {
        const double *x0 = Xb + (long long)t * 3, *x1 = Xb + (long long)(t + l) * 3;
        const double *w0 = wb + (long long)t * kW, *w1 = wb + (long long)(t + l) * kW;
        for (int a = 0; a < 3; ++a) {
            const double dx = x1[a] - x0[a];
            acc[a] += dx * dx;
            const double db = w1[3 + a] - w0[3 + a];
            acc[3 + a] += db * db;
            const double dr = w1[6 + a] - w0[6 + a];
            acc[7 + a] += dr * dr;
        }
        const double cr[3] = {w0[1] * w1[2] - w0[2] * w1[1], w0[2] * w1[0] - w0[0] * w1[2],
                              w0[0] * w1[1] - w0[1] * w1[0]};
        const double th = atan2(sqrt(dot3(cr, cr)), dot3(w0, w1));
        acc[6] += th * th;
    }
    __shared__ double red[LB_MSD_COLS][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = 0; c < LB_MSD_COLS; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < LB_MSD_COLS) {
        double v = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[threadIdx.x][w];
        out[((long long)b * max_lag + (l - 1)) * LB_MSD_COLS + threadIdx.x] = v / (double)n;
    }
}

}  // namespace

cudaError_t launch_msd(const double *X, const double *q, int nrec, int nbodies, int max_lag, const double *p_ref,
                       double *work, double *out, cudaStream_t s) {
    const long long nt = (long long)nrec * nbodies;
    k_msd_prep<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(X, q, nrec, nbodies, p_ref, work);
    k_msd_scan<<<(unsigned)((6 * nbodies + 127) / 128), 128, 0, s>>>(nrec, nbodies, work);
    k_msd_lags<<<dim3((unsigned)max_lag, (unsigned)nbodies), kThreads, 0, s>>>(X, nrec, nbodies, max_lag, work, out);
    return cudaGetLastError();
}

// Host side of the trajectory readers: the valid records of body `id` (of
// nb) in the ring, oldest first. Records k = k0 .. step / every exist;
// the ring keeps the last cap of them.
cudaError_t copy_records(const double *ring, int every, int cap, long long k0, long long step, int nb, int id,
                         int max_records, long long *steps, double *X, double *q, int *count, cudaStream_t s) {
    *count = 0;
    if (!ring || every <= 0) return cudaSuccess;
    const long long k_last = step / every;
    long long k_first = k_last - cap + 1;
    if (k_first < k0) k_first = k0;
    long long n = k_last - k_first + 1;
    if (n <= 0) return cudaSuccess;
    if (n > max_records) {                  // the most recent max_records
        k_first = k_last - max_records + 1;
        n = max_records;
    }
    // one strided 2-D copy per contiguous run of slots (at most two)
    std::vector<double> rec((size_t)n * 7);
    long long done = 0;
    while (done < n) {
        const long long slot = (k_first + done - 1) % cap;
        const long long run = std::min<long long>(n - done, cap - slot);
        cudaError_t e = cudaMemcpy2DAsync(rec.data() + done * 7, 7 * sizeof(double),
                                          ring + (slot * nb + id) * 7, (size_t)nb * 7 * sizeof(double),
                                          7 * sizeof(double), (size_t)run, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        done += run;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (long long r = 0; r < n; ++r) {
        if (steps) steps[r] = (k_first + r) * every;
        if (X) std::memcpy(X + 3 * r, &rec[7 * r], 3 * sizeof(double));
        if (q) std::memcpy(q + 4 * r, &rec[7 * r + 3], 4 * sizeof(double));
    }
    *count = (int)n;
    return cudaSuccess;
}

}  // namespace lbk

extern "C" lb_status lb_msd_trajectory(const double *X, const double *q, int nrec, int nbodies, int max_lag,
                                       const double p_ref[3], double *out, void *cuda_stream, char *err,
                                       size_t err_len) {
    auto fail = [&](lb_status st, const std::string &m) {
        if (err && err_len) {
            std::strncpy(err, m.c_str(), err_len - 1);
            err[err_len - 1] = 0;
        }
        return st;
    };
    if (!X || !q || !p_ref || !out) return fail(LB_ERR_ARG, "null pointer");
    if (nbodies < 1 || nrec < 2 || max_lag < 1 || max_lag >= nrec || nbodies > 65535)
        return fail(LB_ERR_ARG, "need nbodies in [1, 65535], nrec >= 2 and 1 <= max_lag < nrec");
    if (!(p_ref[0] * p_ref[0] + p_ref[1] * p_ref[1] + p_ref[2] * p_ref[2] > 0.0))
        return fail(LB_ERR_ARG, "p_ref must be non-zero");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t nX = (size_t)nrec * nbodies * 3, nq = (size_t)nrec * nbodies * 4;
    const size_t nw = (size_t)nrec * nbodies * lbk::kW, no = (size_t)max_lag * nbodies * LB_MSD_COLS;
    double *d = nullptr;
    const size_t total = nX + nq + nw + no + 3;
    cudaError_t e = cudaMalloc((void **)&d, total * sizeof(double));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(LB_ERR_OOM, "device allocation for the trajectory failed");
    }
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    double *dX = d, *dq = dX + nX, *dw = dq + nq, *dout = dw + nw, *dp = dout + no;
    e = cudaMemcpyAsync(dX, X, nX * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dq, q, nq * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, p_ref, 3 * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = lbk::launch_msd(dX, dq, nrec, nbodies, max_lag, dp, dw, dout, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, no * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("lb_msd_trajectory: ") + cudaGetErrorString(e));
    return LB_OK;
}

// --------------------------------------------------------------- pore frame
// Pore-frame analysis (Sec. 2.8 and the SI "Pore-frame coordinate
// determination"): centres relative to the pore axis (x^c, y^c across it, z
// along it); one interval's displacement rotated into the frame of its start
// (x^p radial, y^p azimuthal, z^p axial; cos and sin of theta as x^c / r and
// y^c / r) and summed; the MSD of the sub-trajectories binned by the radial
// coordinate of their first record.
namespace lbk {
namespace {

struct PoreFrame {
    int a1, a2, ax;
    double c1, c2;
};

__device__ __forceinline__ double radial(double xc, double yc) {
    return sqrt(__dadd_rn(__dmul_rn(xc, xc), __dmul_rn(yc, yc)));   // no contraction: bins depend on it
}

// one thread per record: increment over [k-1, k] (zero for k = 0) and r_k
__global__ void k_pore_prep(const double *X, int nrec, PoreFrame pf, double *work) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrec) return;
    const double *x = X + 3ll * k;
    const double xc = x[pf.a1] - pf.c1, yc = x[pf.a2] - pf.c2;
    double *w = work + 4ll * k;
    w[3] = radial(xc, yc);
    if (k == 0) {
        w[0] = w[1] = w[2] = 0.0;
        return;
    }
    const double *xp = x - 3;
    const double xp1 = xp[pf.a1] - pf.c1, yp1 = xp[pf.a2] - pf.c2;
    const double r0 = radial(xp1, yp1);
    const double c = r0 > 0.0 ? xp1 / r0 : 1.0, s = r0 > 0.0 ? yp1 / r0 : 0.0;
    const double dx = xc - xp1, dy = yc - yp1, dz = x[pf.ax] - xp[pf.ax];
    w[0] = c * dx + s * dy;
    w[1] = -s * dx + c * dy;
    w[2] = dz;
}

__global__ void k_pore_scan(int nrec, double *work) {
    const int c = threadIdx.x;
    if (c >= 3) return;
    double acc = 0.0;
    for (int k = 0; k < nrec; ++k) {
        acc += work[4ll * k + c];
        work[4ll * k + c] = acc;
    }
}

// one block per lag: per-bin sums in shared memory
__global__ void k_pore_lags(int nrec, int nbins, double R, int max_lag, const double *work, double *out,
                            long long *counts) {
    extern __shared__ double sm[];
    double *acc = sm;                                            // [nbins][3]
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(sm + 3 * nbins);
    for (int i = threadIdx.x; i < 4 * nbins; i += blockDim.x) sm[i] = 0.0;
    __syncthreads();
    const int l = blockIdx.x + 1;
    for (int t = threadIdx.x; t < nrec - l; t += blockDim.x) {
        const double *w0 = work + 4ll * t, *w1 = work + 4ll * (t + l);
        const double fb = floor(__dmul_rn(w0[3] / R, (double)nbins));
        if (!(fb >= 0.0 && fb < (double)nbins)) continue;
        const int b = (int)fb;
        for (int c = 0; c < 3; ++c) {
            const double d = w1[c] - w0[c];
            atomicAdd(&acc[3 * b + c], d * d);
        }
        atomicAdd(&cnt[b], 1ull);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        const unsigned long long n = cnt[b];
        for (int c = 0; c < 3; ++c)
            out[((long long)b * max_lag + (l - 1)) * 3 + c] = n ? acc[3 * b + c] / (double)n : 0.0;
        counts[(long long)b * max_lag + (l - 1)] = (long long)n;
    }
}

}  // namespace
}  // namespace lbk

extern "C" lb_status lb_pore_msd(const double *X, int nrec, int nx, int ny, int nz, int axis, double R_pore,
                                 int nbins, int max_lag, double *out, long long *counts, void *cuda_stream,
                                 char *err, size_t err_len) {
    auto fail = [&](lb_status st, const std::string &m) {
        if (err && err_len) {
            std::strncpy(err, m.c_str(), err_len - 1);
            err[err_len - 1] = 0;
        }
        return st;
    };
    if (!X || !out || !counts) return fail(LB_ERR_ARG, "null pointer");
    if (nrec < 2 || max_lag < 1 || max_lag >= nrec || nbins < 1 || nbins > 4096 || axis < 0 || axis > 2 ||
        !(R_pore > 0.0) || nx < 1 || ny < 1 || nz < 1)
        return fail(LB_ERR_ARG, "need nrec >= 2, 1 <= max_lag < nrec, 1 <= nbins <= 4096, axis 0-2, R_pore > 0");
    const int n[3] = {nx, ny, nz};
    lbk::PoreFrame pf;
    pf.ax = axis;
    pf.a1 = axis == 0 ? 1 : 0;
    pf.a2 = axis == 2 ? 1 : 2;
    pf.c1 = 0.5 * n[pf.a1];
    pf.c2 = 0.5 * n[pf.a2];
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t nX = 3ull * nrec, nw = 4ull * nrec, no = 3ull * nbins * max_lag, nc = (size_t)nbins * max_lag;
    double *d = nullptr;
    cudaError_t e = cudaMalloc((void **)&d, (nX + nw + no + nc) * sizeof(double));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(LB_ERR_OOM, "device allocation for the trajectory failed");
    }
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    double *dX = d, *dw = dX + nX, *dout = dw + nw;
    long long *dcnt = reinterpret_cast<long long *>(dout + no);
    const size_t smem = 4ull * nbins * sizeof(double);
    e = cudaMemcpyAsync(dX, X, nX * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        lbk::k_pore_prep<<<(nrec + 255) / 256, 256, 0, s>>>(dX, nrec, pf, dw);
        lbk::k_pore_scan<<<1, 32, 0, s>>>(nrec, dw);
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(lbk::k_pore_lags, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            lbk::k_pore_lags<<<max_lag, 256, smem, s>>>(nrec, nbins, R_pore, max_lag, dw, dout, dcnt);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, no * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dcnt, nc * sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(LB_ERR_CUDA, std::string("lb_pore_msd: ") + cudaGetErrorString(e));
    return LB_OK;
}
