// C ABI (include/lb.h) and host runtime: parameter validation, device
// memory, the per-step launch sequence, population and force I/O, kernel
// timing. Every entry point returns an lb_status and never throws.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lb_ctx.h"


namespace {

thread_local std::string g_create_error;

lb_status fail(lb_ctx *h, lb_status s, const std::string &msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return s;
}

lb_status cuda_fail(lb_ctx *h, cudaError_t e, const char *where) {
    return fail(h, LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// steps per captured CUDA graph replayed by long lb_step calls (even)
#ifndef LB_GRAPH_STEPS
#define LB_GRAPH_STEPS 8
#endif
// node count from which long lb_step calls launch eagerly instead of
// replaying graphs
#ifndef LB_EAGER_NODES
#define LB_EAGER_NODES (1LL << 20)
#endif

#define LB_CUDA(h, call)                                                  \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);          \
    } while (0)

template <typename P>
lb_status dev_alloc(lb_ctx *h, P **ptr, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(h, LB_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
    h->dev_bytes += bytes;
    return LB_OK;
}

void compute_gforce(const lb_ctx *h, double g[3]) {
    for (int a = 0; a < 3; ++a) g[a] = h->p.body_force[a];
    if (h->p.compensate_force && h->nfluid > 0)
        for (const Body &b : h->hb)
            if (b.fixed != 1)
                for (int a = 0; a < 3; ++a) g[a] -= b.F_ext[a] / (double)h->nfluid;
}

// The uniform force density in FP64 and FP32, staged in host memory that
// stays valid until the asynchronous copy has run.
lb_status push_gforce(lb_ctx *h) {
    compute_gforce(h, h->g_host);
    for (int a = 0; a < 3; ++a) h->gf_host[a] = (float)h->g_host[a];
    LB_CUDA(h, cudaMemcpyAsync(h->gforce, h->g_host, 3 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    LB_CUDA(h, cudaMemcpyAsync(h->gforce_f, h->gf_host, 3 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

long long count_fluid(const lb_ctx *h) {
    if (h->g.pore_axis < 0) return h->g.N;
    const int ax = h->g.pore_axis;
    const int na = ax == 0 ? h->g.ny : h->g.nx;
    const int nb = ax == 2 ? h->g.ny : h->g.nz;
    const int nl = ax == 0 ? h->g.nx : (ax == 1 ? h->g.ny : h->g.nz);
    long long c = 0;
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < na; ++a) {
            const long long da = 2LL * a + 1 - na, db = 2LL * b + 1 - nb;
            if (da * da + db * db < h->g.pore_t) ++c;
        }
    return c * nl;
}

lb_status upload_bodies(lb_ctx *h) {
    if (h->uploaded) return LB_OK;
    const int nb = (int)h->hb.size();
    const int nbeads = (int)h->hbody_of.size();
    if (nb > 0) {
        lb_status s;
        if ((s = dev_alloc(h, &h->db, sizeof(Body) * nb)) != LB_OK) return s;
        if ((s = dev_alloc(h, &h->ds, sizeof(double) * 3 * (size_t)std::max(nbeads, 1))) != LB_OK) return s;
        if ((s = dev_alloc(h, &h->dsf, sizeof(float) * 3 * (size_t)std::max(nbeads, 1))) != LB_OK) return s;
        if ((s = dev_alloc(h, &h->dbody_of, sizeof(int) * (size_t)std::max(nbeads, 1))) != LB_OK) return s;
        if ((s = dev_alloc(h, &h->dFbead, sizeof(double) * 3 * (size_t)std::max(nbeads, 1))) != LB_OK) return s;
        LB_CUDA(h, cudaMemcpyAsync(h->db, h->hb.data(), sizeof(Body) * nb, cudaMemcpyHostToDevice, h->stream));
        if (nbeads > 0) {
            LB_CUDA(h, cudaMemcpyAsync(h->ds, h->hs.data(), sizeof(double) * 3 * nbeads, cudaMemcpyHostToDevice, h->stream));
            h->hsf.assign(h->hs.begin(), h->hs.end());
            LB_CUDA(h, cudaMemcpyAsync(h->dsf, h->hsf.data(), sizeof(float) * 3 * nbeads, cudaMemcpyHostToDevice, h->stream));
            LB_CUDA(h, cudaMemcpyAsync(h->dbody_of, h->hbody_of.data(), sizeof(int) * nbeads, cudaMemcpyHostToDevice, h->stream));
        }
        LB_CUDA(h, cudaMemsetAsync(h->dFbead, 0, sizeof(double) * 3 * (size_t)std::max(nbeads, 1), h->stream));
        // host-mapped body I/O; without it (allocation refused) the copies below serve
        if (cudaHostAlloc((void **)&h->io_map, sizeof(double) * (12 * (size_t)nb + 1), cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer((void **)&h->io_dmap, h->io_map, 0) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_io, cudaEventDisableTiming) == cudaSuccess) {
            std::memset(h->io_map, 0, sizeof(double) * (12 * (size_t)nb + 1));
            for (int b = 0; b < nb; ++b)
                for (int a = 0; a < 3; ++a) {
                    h->io_map[3 * b + a] = h->hb[b].F_ext[a];
                    h->io_map[3 * (size_t)nb + 3 * b + a] = h->hb[b].T_ext[a];
                }
        } else {
            cudaGetLastError();
            if (h->io_map) cudaFreeHost(h->io_map);
            h->io_map = h->io_dmap = nullptr;
        }
        const size_t fbytes = (h->fp32 ? sizeof(float) : sizeof(double)) * 3 * (size_t)h->g.N;
        const long long ntiles = (long long)h->ntx * h->nty * h->ntz;
        const size_t tbytes = sizeof(int) * (size_t)ntiles;
        h->list_cap = (int)std::min<long long>(ntiles, 8LL * std::max(nbeads, 1));
        for (int k = 0; k < 2; ++k) {
            if ((s = dev_alloc(h, &h->Fbuf[k], fbytes)) != LB_OK) return s;
            if ((s = dev_alloc(h, &h->tiles[k], tbytes)) != LB_OK) return s;
            if ((s = dev_alloc(h, &h->tlist[k], sizeof(int) * (size_t)h->list_cap)) != LB_OK) return s;
            if ((s = dev_alloc(h, &h->tcount[k], sizeof(int))) != LB_OK) return s;
            LB_CUDA(h, cudaMemsetAsync(h->tcount[k], 0, sizeof(int), h->stream));
            LB_CUDA(h, cudaMemsetAsync(h->Fbuf[k], 0, fbytes, h->stream));
            LB_CUDA(h, cudaMemsetAsync(h->tiles[k], 0, tbytes, h->stream));
        }
    }
    lb_status s = push_gforce(h);
    if (s != LB_OK) return s;
    h->uploaded = true;
    return LB_OK;
}

// refresh the host mirror of the bodies from the device
lb_status pull_bodies(lb_ctx *h) {
    if (!h->uploaded || h->hb.empty()) return LB_OK;
    // the host's external forces stay authoritative: the device records take
    // them at the next step's prologue
    std::vector<double> ext(6 * h->hb.size());
    for (size_t b = 0; b < h->hb.size(); ++b)
        for (int a = 0; a < 3; ++a) {
            ext[6 * b + a] = h->hb[b].F_ext[a];
            ext[6 * b + 3 + a] = h->hb[b].T_ext[a];
        }
    LB_CUDA(h, cudaMemcpyAsync(h->hb.data(), h->db, sizeof(Body) * h->hb.size(), cudaMemcpyDeviceToHost, h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    for (size_t b = 0; b < h->hb.size(); ++b)
        for (int a = 0; a < 3; ++a) {
            h->hb[b].F_ext[a] = ext[6 * b + a];
            h->hb[b].T_ext[a] = ext[6 * b + 3 + a];
        }
    return LB_OK;
}

lb_status push_bodies(lb_ctx *h) {
    if (!h->uploaded || h->hb.empty()) return LB_OK;
    LB_CUDA(h, cudaMemcpyAsync(h->db, h->hb.data(), sizeof(Body) * h->hb.size(), cudaMemcpyHostToDevice, h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

// Synchronises the stream (completing the copies the caller queued before)
// and returns LB_ERR_TIMEOUT if a kernel recorded that a bounded wait ran out
// since the last check (the error word is reset, so it is reported once).
// The error word travels in the same synchronisation as the caller's copies.
lb_status check_device_error(lb_ctx *h) {
    LB_CUDA(h, cudaMemcpyAsync(h->err_host, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    const int e = *h->err_host;
    if (e && h->io_map) h->io_map[12 * h->hb.size()] = 0.0;   // reported here, not again from the mapped copy
    if (e & 2) {
        LB_CUDA(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
        return fail(h, LB_ERR_STATE, "an index check of the checked build failed (an index outside its array)");
    }
    if (e) {
        LB_CUDA(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
        return fail(h, LB_ERR_TIMEOUT, "a bounded device wait ran out (TMA copy did not complete in time)");
    }
    return LB_OK;
}

lb_status check_handle(lb_ctx *h) {
    if (!h) return fail(nullptr, LB_ERR_ARG, "null handle");
    return LB_OK;
}

lbk::FluidArgs fluid_args(const lb_ctx *h, int cur, uint32_t step_off) {
    lbk::FluidArgs a{};
    a.g = h->g;
    a.f = h->f;
    a.masks = h->dmask;
    // MRT coefficients with c_k = w_diag / b_k = (1/36) / b_k folded in
    static const double bk[19] = {1.0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9,
                                  1.0 / 9, 2.0 / 3, 2.0 / 3, 2.0 / 3, 2.0 / 9, 2.0 / 9, 2.0 / 9, 2.0, 4.0 / 3,
                                  4.0 / 9};
    auto rate = [&](int k) {
        return k == 4 ? h->p.gamma_bulk : (k <= 9 ? h->p.gamma_shear : (k <= 15 ? h->p.gamma_odd : h->p.gamma_even));
    };
    a.pd.rho0 = h->p.rho0;
    a.pd.omega = 1.0 / h->p.tau;
    for (int k = 4; k <= 9; ++k) {
        const double c = (1.0 / 36.0) / bk[k], g = rate(k);
        a.pd.ke[k - 4] = c * (1.0 - g);
        a.pd.km[k - 4] = c * g;
        a.pd.ks[k - 4] = c * 0.5 * (1.0 + g);
    }
    for (int k = 10; k <= 18; ++k) a.pd.kg[k - 10] = (1.0 / 36.0) / bk[k] * rate(k);
    for (int k = 4; k <= 18; ++k) a.pd.kn[k - 4] = (1.0 / 36.0) / bk[k] * h->sig[k - 4] * 3.4641016151377544;
    a.pf.rho0 = (float)a.pd.rho0;
    a.pf.omega = (float)a.pd.omega;
    for (int k = 0; k < 6; ++k) {
        a.pf.ke[k] = (float)a.pd.ke[k];
        a.pf.km[k] = (float)a.pd.km[k];
        a.pf.ks[k] = (float)a.pd.ks[k];
    }
    for (int k = 0; k < 9; ++k) a.pf.kg[k] = (float)a.pd.kg[k];
    for (int k = 0; k < 15; ++k) a.pf.kn[k] = (float)(a.pd.kn[k] * 2.3283064365386963e-10);
    a.gforce = h->gforce;
    a.gforce_f = h->gforce_f;
    const bool bodies = !h->hb.empty() && !h->hbody_of.empty();
    a.Fn = bodies ? h->Fbuf[cur] : nullptr;
    a.tiles = bodies ? h->tiles[cur] : nullptr;
    a.ntx = h->ntx;
    a.nty = h->nty;
    a.key0 = (uint32_t)h->p.seed;
    a.key1 = (uint32_t)(h->p.seed >> 32);
    a.instance = h->p.instance;
    a.step_base = h->step_dev;
    a.step_off = step_off;
    a.err = h->err_dev;
    const size_t es = h->fp32 ? 4 : 8;
    // in place, or (f_src / f_dst set) from one buffer into another
    char *src = static_cast<char *>(const_cast<void *>(h->f_src ? h->f_src : h->f));
    char *dst = static_cast<char *>(h->f_dst ? h->f_dst : h->f);
    a.f = src;
    for (int i = 0; i < 19; ++i) {
        a.plane[i] = src + (size_t)i * (size_t)h->g.N * es;
        a.out[i] = dst + (size_t)i * (size_t)h->g.N * es;
    }
    return a;
}

// the captured step pair holds launch arguments by value: drop it whenever
// one of them changes
void drop_graph(lb_ctx *h) {
    for (cudaGraphExec_t *g : {&h->gexec, &h->gexec8})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    for (auto &g : h->gexec1)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

lb_status timed_collide(lb_ctx *h, const lbk::FluidArgs &a, bool odd) {
    const bool noise = h->p.collision == 1 && h->p.kT > 0.0;
    if (h->timing) {
        if (h->ev_used + 2 > h->ev.size()) {
            if (h->ev.size() >= 8192) {
                // fold the recorded pairs into the totals to bound the event pool
                LB_CUDA(h, cudaStreamSynchronize(h->stream));
                for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
                    float ms = 0.f;
                    LB_CUDA(h, cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
                    h->timed_ms += ms;
                    h->timed_n += 1;
                }
                h->ev_used = 0;
            } else {
                for (int k = 0; k < 256; ++k) {
                    cudaEvent_t e;
                    LB_CUDA(h, cudaEventCreate(&e));
                    h->ev.push_back(e);
                }
            }
        }
        LB_CUDA(h, cudaEventRecord(h->ev[h->ev_used], h->stream));
    }
    const bool oop = a.out[0] != a.plane[0];
    const bool tma = !oop && h->cs_variant == 2 && lbk::tma_collide_supported(h->g, h->fp32);
    cudaError_t e = oop ? lbk::launch_collide_stream_oop(a, h->fp32, h->p.collision, odd, h->block, h->stream)
                  : tma ? lbk::launch_collide_stream_tma(a, h->p.collision, noise, odd, h->tma_stages, h->tma_ctas,
                                                         h->wait_limit, h->stream)
                        : lbk::launch_collide_stream(a, h->fp32, h->p.collision, noise, odd, h->block, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "collide_stream launch");
    if (h->timing) {
        LB_CUDA(h, cudaEventRecord(h->ev[h->ev_used + 1], h->stream));
        h->ev_used += 2;
    }
    return LB_OK;
}

}  // namespace

namespace lbk {
// host-side hooks used by the adjoint driver (lb_adjoint.cu)
lb_status ctx_upload(lb_ctx *h) { return upload_bodies(h); }
// the device body records take the host's external forces now (the adjoint
// steps with kernels of its own, which do not read the mapped staging), and
// the mapped totals are stale once it has run
lb_status ctx_apply_external(lb_ctx *h) {
    h->out_fresh = false;
    if (!h->io_map || h->hb.empty()) return LB_OK;
    lb_status s = pull_bodies(h);
    if (s != LB_OK) return s;
    return push_bodies(h);
}
lb_status ctx_fail(lb_ctx *h, lb_status s, const std::string &m) { return fail(h, s, m); }
}  // namespace lbk

extern "C" {

const char *lb_status_string(lb_status s) {
    switch (s) {
    case LB_OK: return "ok";
    case LB_ERR_ARG: return "invalid argument";
    case LB_ERR_OOM: return "out of memory";
    case LB_ERR_CUDA: return "CUDA error";
    case LB_ERR_UNSTABLE: return "non-finite mass or momentum";
    case LB_ERR_TIMEOUT: return "device wait timed out";
    case LB_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char *lb_last_error(lb_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int lb_lattice(int *c, double *w, int *opp) {
    for (int i = 0; i < 19; ++i) {
        if (c) { c[3 * i] = lbk::cx(i); c[3 * i + 1] = lbk::cy(i); c[3 * i + 2] = lbk::cz(i); }
        if (w) w[i] = lbk::wq(i);
        if (opp) opp[i] = lbk::opp(i);
    }
    return 19;
}

lb_status lb_create(const lb_params *p, void *cuda_stream, lb_handle *out) {
    if (!p || !out) return fail(nullptr, LB_ERR_ARG, "null argument");
    *out = nullptr;
    if (p->nx < 2 || p->ny < 2 || p->nz < 2) return fail(nullptr, LB_ERR_ARG, "lattice sizes must be >= 2");
    const double N = (double)p->nx * p->ny * p->nz;
    if (N > 2.0e9) return fail(nullptr, LB_ERR_ARG, "lattice too large (node count must fit 31 bits)");
    if (p->precision != 32 && p->precision != 64) return fail(nullptr, LB_ERR_ARG, "precision must be 32 or 64");
    if (p->collision != 0 && p->collision != 1) return fail(nullptr, LB_ERR_ARG, "collision must be 0 (BGK) or 1 (MRT)");
    if (p->collision == 0 && !(p->tau > 0.5)) return fail(nullptr, LB_ERR_ARG, "BGK needs tau > 1/2");
    if (p->collision == 1) {
        const double r[4] = {p->gamma_shear, p->gamma_bulk, p->gamma_odd, p->gamma_even};
        for (double v : r)
            if (!(v > -1.0 && v < 1.0)) return fail(nullptr, LB_ERR_ARG, "MRT rates must lie in (-1, 1)");
    }
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) return fail(nullptr, LB_ERR_ARG, "rho0 must be > 0");
    if (!(p->kT >= 0.0) || !std::isfinite(p->kT)) return fail(nullptr, LB_ERR_ARG, "kT must be >= 0");
    if (p->kT > 0.0 && p->collision == 0)
        return fail(nullptr, LB_ERR_ARG, "thermal noise needs MRT collision (BGK has no separate non-conserved modes)");
    if (!(p->gamma_bead >= 0.0) || !std::isfinite(p->gamma_bead)) return fail(nullptr, LB_ERR_ARG, "gamma_bead must be >= 0");
    if (p->md_substeps < 0 || p->md_substeps > 4) return fail(nullptr, LB_ERR_ARG, "md_substeps must be 0-4 (0 = 1)");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->body_force[a])) return fail(nullptr, LB_ERR_ARG, "body_force must be finite");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, LB_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }

    lb_ctx *h = new (std::nothrow) lb_ctx();
    if (!h) return fail(nullptr, LB_ERR_OOM, "host allocation failed");
    h->p = *p;
    h->p.md_substeps = p->md_substeps > 1 ? p->md_substeps : 1;
    h->fp32 = p->precision == 32;
    h->g.nx = p->nx; h->g.ny = p->ny; h->g.nz = p->nz;
    h->g.N = (long long)p->nx * p->ny * p->nz;
    h->g.pore_axis = -1;
    h->g.pore_t = 0;
    h->g.pore_in = 0;
    h->nfluid = h->g.N;
    h->ntx = (p->nx + 3) / 4; h->nty = (p->ny + 3) / 4; h->ntz = (p->nz + 3) / 4;
    // noise amplitudes per mode (divided by sqrt(rho)): sqrt(3 kT b_k (1 - g_k^2))
    if (p->collision == 1 && p->kT > 0.0) {
        const double b[15] = {2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 2.0 / 3, 2.0 / 3, 2.0 / 3,
                              2.0 / 9, 2.0 / 9, 2.0 / 9, 2.0, 4.0 / 3, 4.0 / 9};
        for (int k = 0; k < 15; ++k) {
            const int mode = k + 4;
            const double gk = mode == 4 ? p->gamma_bulk : (mode <= 9 ? p->gamma_shear : (mode <= 15 ? p->gamma_odd : p->gamma_even));
            h->sig[k] = std::sqrt(3.0 * p->kT * b[k] * (1.0 - gk * gk));
        }
    }
    // block shape: x fastest, 128 threads
    int bx = ((p->nx + 31) / 32) * 32;
    if (bx > 128) bx = 128;
    h->block = dim3(bx, 128 / bx, 1);

    if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
    else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { lb_status s = cuda_fail(nullptr, e, "cudaStreamCreate"); delete h; return s; }
        h->own_stream = true;
    }
    e = cudaMallocHost((void **)&h->err_host, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lb_status s = cuda_fail(nullptr, e, "side stream");
        lb_destroy(h);
        return s;
    }
    const size_t es = h->fp32 ? 4 : 8;
    lb_status s;
    if ((s = dev_alloc(h, &h->f, es * 19 * (size_t)h->g.N)) != LB_OK ||
        (s = dev_alloc(h, &h->gforce, 3 * sizeof(double))) != LB_OK ||
        (s = dev_alloc(h, &h->gforce_f, 3 * sizeof(float))) != LB_OK ||
        (s = dev_alloc(h, &h->step_dev, sizeof(unsigned long long))) != LB_OK ||
        (s = dev_alloc(h, &h->err_dev, sizeof(int))) != LB_OK) {
        g_create_error = h->err;
        lb_destroy(h);
        return s;
    }
    h->red_blocks = 1024;
    if ((s = dev_alloc(h, &h->partials, sizeof(double) * 4 * h->red_blocks)) != LB_OK ||
        (s = dev_alloc(h, &h->out4, sizeof(double) * 4)) != LB_OK) {
        g_create_error = h->err;
        lb_destroy(h);
        return s;
    }
    e = cudaMemsetAsync(h->step_dev, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = lbk::launch_init(h->f, h->fp32, h->g.N, p->rho0, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cuda_fail(nullptr, e, "lb_create init");
        lb_destroy(h);
        return LB_ERR_CUDA;
    }
    *out = h;
    return LB_OK;
}

lb_status lb_destroy(lb_handle h) {
    if (!h) return LB_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    lbk::adj_free(h);
    void *bufs[] = {h->f, h->gforce, h->gforce_f, h->step_dev, h->err_dev, h->Fbuf[0], h->Fbuf[1], h->tiles[0], h->tiles[1],
                    h->tlist[0], h->tlist[1], h->tcount[0], h->tcount[1],
                    h->db, h->ds, h->dsf, h->dbody_of, h->dFbead, h->partials, h->out4, h->rec, h->dmask, h->dwchan};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->err_host) cudaFreeHost(h->err_host);
    if (h->io_map) cudaFreeHost(h->io_map);
    if (h->ev_io) cudaEventDestroy(h->ev_io);
    delete h;
    return LB_OK;
}

lb_status lb_set_pore(lb_handle h, double radius, int axis) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (h->g.chan) return fail(h, LB_ERR_STATE, "a lattice has either a pore or channel walls");
    drop_graph(h);
    if (h->step > 0 || h->uploaded) return fail(h, LB_ERR_STATE, "lb_set_pore must come before the first lb_step");
    if (axis < 0 || axis > 2) return fail(h, LB_ERR_ARG, "axis must be 0, 1 or 2");
    if (!(radius > 0.0) || !std::isfinite(radius)) return fail(h, LB_ERR_ARG, "radius must be > 0");
    // wall iff d^2 >= R^2 with d the node-centre distance; in doubled
    // coordinates 4 d^2 is an integer, so the test is 4 d^2 >= ceil(4 R^2)
    const double t = std::ceil(4.0 * (radius * radius));
    h->g.pore_axis = axis;
    h->g.pore_t = (long long)t;
    h->pore_R = radius;
    h->wall = lbk::WallBeads{};
    const double inner = std::sqrt(t) - 2.0 * std::sqrt(2.0) - 0.01;
    h->g.pore_in = inner > 0 ? (long long)std::floor(inner * inner) : 0;
    h->nfluid = count_fluid(h);
    // wall masks of the positions across the axis, read by the fluid kernel
    if (h->dmask) {
        LB_CUDA(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->dmask);
        h->dmask = nullptr;
    }
    lb_status s = dev_alloc(h, &h->dmask, sizeof(uint32_t) * (size_t)lbk::pore_section_size(h->g));
    if (s != LB_OK) return s;
    LB_CUDA(h, lbk::launch_build_masks(h->g, h->dmask, h->stream));
    // populations of new wall nodes are never read; nothing else changes
    return LB_OK;
}

lb_status lb_set_channel_walls(lb_handle h, const double u_lo[3], const double u_hi[3]) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (h->step > 0 || h->uploaded) return fail(h, LB_ERR_STATE, "lb_set_channel_walls must come before the first lb_step");
    if (h->g.pore_axis >= 0) return fail(h, LB_ERR_STATE, "a lattice has either a pore or channel walls");
    if (!u_lo || !u_hi || u_lo[1] != 0.0 || u_hi[1] != 0.0 || h->g.ny < 2)
        return fail(h, LB_ERR_ARG, "wall velocities must be tangential (y component 0), ny >= 2");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(u_lo[a]) || !std::isfinite(u_hi[a])) return fail(h, LB_ERR_ARG, "non-finite wall velocity");
    drop_graph(h);
    // bounce-back terms 6 w_i rho0 (c_i . u_wall) of both walls, then the velocities
    static const int C[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                 {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                 {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                 {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    double tab[44];
    for (int side = 0; side < 2; ++side) {
        const double *u = side ? u_hi : u_lo;
        for (int i = 0; i < 19; ++i) {
            const double w = i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
            tab[19 * side + i] = 6.0 * w * h->p.rho0 * (C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2]);
        }
        for (int a = 0; a < 3; ++a) tab[38 + 3 * side + a] = u[a];
    }
    lb_status s;
    if (!h->dwchan && (s = dev_alloc(h, &h->dwchan, sizeof(tab))) != LB_OK) return s;
    LB_CUDA(h, cudaMemcpy(h->dwchan, tab, sizeof(tab), cudaMemcpyHostToDevice));
    h->g.chan = 1;
    h->g.wchan = h->dwchan;
    if (h->dmask) {
        cudaFree(h->dmask);
        h->dmask = nullptr;
    }
    if ((s = dev_alloc(h, &h->dmask, sizeof(uint32_t) * (size_t)h->g.ny)) != LB_OK) return s;
    LB_CUDA(h, lbk::launch_build_masks(h->g, h->dmask, h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

lb_status lb_set_pore_beads(lb_handle h, double spacing, double r_pore_bead, double r_bead, double epsilon) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    drop_graph(h);
    if (h->g.pore_axis < 0) return fail(h, LB_ERR_STATE, "lb_set_pore_beads needs a pore (lb_set_pore)");
    if (spacing == 0.0) {
        h->wall = lbk::WallBeads{};
        return LB_OK;
    }
    if (!lbk::make_wall_beads(h->g, h->pore_R, spacing, r_pore_bead, r_bead, epsilon, h->wall))
        return fail(h, LB_ERR_ARG, "spacing > 0, radii >= 0 with a positive sum, epsilon >= 0");
    return LB_OK;
}

lb_status lb_add_raspberry(lb_handle h, const double *beads, int nbeads, const double X[3], const double q[4],
                           double mass, const double inertia[3], const double F_ext[3], const double T_ext[3],
                           int fixed, int *body_id) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (h->uploaded) return fail(h, LB_ERR_STATE, "bodies must be added before the first lb_step");
    if (nbeads < 0 || (nbeads > 0 && !beads) || !X || !q || !inertia)
        return fail(h, LB_ERR_ARG, "bad raspberry arguments");
    if (!(mass > 0.0) || !(inertia[0] > 0 && inertia[1] > 0 && inertia[2] > 0))
        return fail(h, LB_ERR_ARG, "mass and inertia must be positive");
    const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(qn > 0.0) || !std::isfinite(qn)) return fail(h, LB_ERR_ARG, "quaternion must be non-zero");
    for (int k = 0; k < 3 * nbeads; ++k)
        if (!std::isfinite(beads[k])) return fail(h, LB_ERR_ARG, "non-finite bead offset");
    if (!lbk::all_finite(X, 3) || !lbk::all_finite(&mass, 1) || !lbk::all_finite(inertia, 3) ||
        !lbk::all_finite(F_ext, 3) || !lbk::all_finite(T_ext, 3))
        return fail(h, LB_ERR_ARG, "non-finite position, mass, inertia or external force");
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
    if (fixed < 0 || fixed > 2) return fail(h, LB_ERR_ARG, "fixed must be 0, 1 or 2");
    b.fixed = fixed;
    const int id = (int)h->hb.size();
    h->hb.push_back(b);
    for (int k = 0; k < 3 * nbeads; ++k) h->hs.push_back(beads[k]);
    for (int k = 0; k < nbeads; ++k) h->hbody_of.push_back(id);
    h->bead_start.push_back((int)h->hbody_of.size());
    if (body_id) *body_id = id;
    return LB_OK;
}

lb_status lb_set_body_state(lb_handle h, int id, const double X[3], const double V[3], const double q[4],
                            const double w[3]) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (id < 0 || id >= (int)h->hb.size()) return fail(h, LB_ERR_ARG, "bad body id");
    if (!lbk::all_finite(X, 3) || !lbk::all_finite(V, 3) || !lbk::all_finite(q, 4) || !lbk::all_finite(w, 3))
        return fail(h, LB_ERR_ARG, "non-finite body state");
    lb_status s = pull_bodies(h);
    if (s != LB_OK) return s;
    Body &b = h->hb[id];
    for (int a = 0; a < 3; ++a) {
        if (X) b.X[a] = X[a];
        if (V) b.V[a] = V[a];
        if (w) b.w[a] = w[a];
    }
    if (q) {
        const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(qn > 0.0)) return fail(h, LB_ERR_ARG, "quaternion must be non-zero");
        for (int a = 0; a < 4; ++a) b.q[a] = q[a] / qn;
    }
    return push_bodies(h);
}

lb_status lb_set_external_forces(lb_handle h, int nbodies, const double *F_ext, const double *T_ext) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (nbodies < 0 || nbodies > (int)h->hb.size() || (nbodies > 0 && !F_ext))
        return fail(h, LB_ERR_ARG, "bad external force arguments");
    if (!lbk::all_finite(F_ext, 3 * nbodies) || !lbk::all_finite(T_ext, 3 * nbodies))
        return fail(h, LB_ERR_ARG, "non-finite external force or torque");
    for (int b = 0; b < nbodies; ++b)
        for (int a = 0; a < 3; ++a) {
            h->hb[b].F_ext[a] = F_ext[3 * b + a];
            h->hb[b].T_ext[a] = T_ext ? T_ext[3 * b + a] : 0.0;
        }
    if (!h->uploaded || nbodies == 0) return LB_OK;
    if (h->io_map) {
        // into the host-mapped staging the next step's prologue reads; wait
        // until the steps already queued have read the previous values
        LB_CUDA(h, cudaEventSynchronize(h->ev_io));
        const size_t nbt = h->hb.size();
        for (int b = 0; b < nbodies; ++b)
            for (int a = 0; a < 3; ++a) {
                h->io_map[3 * b + a] = F_ext[3 * b + a];
                h->io_map[3 * nbt + 3 * b + a] = T_ext ? T_ext[3 * b + a] : 0.0;
            }
        if (h->p.compensate_force) return push_gforce(h);
        return LB_OK;
    }
    // strided copies straight into the device body records
    LB_CUDA(h, cudaMemcpy2DAsync(&h->db[0].F_ext[0], sizeof(Body), F_ext, 3 * sizeof(double), 3 * sizeof(double),
                                 nbodies, cudaMemcpyHostToDevice, h->stream));
    if (T_ext)
        LB_CUDA(h, cudaMemcpy2DAsync(&h->db[0].T_ext[0], sizeof(Body), T_ext, 3 * sizeof(double), 3 * sizeof(double),
                                     nbodies, cudaMemcpyHostToDevice, h->stream));
    else
        for (int b = 0; b < nbodies; ++b)
            LB_CUDA(h, cudaMemsetAsync(&h->db[b].T_ext[0], 0, 3 * sizeof(double), h->stream));
    if (h->p.compensate_force) return push_gforce(h);
    return LB_OK;
}

namespace {

// The body prologue of step h->step + k (k-th of a group; the device step
// counter is advanced once per group, so kernels read *step_dev + k): the
// previous step's second half kick if finish_prev, this step's kick and
// drift, the clearing of its spread-force tiles. On stream `st`. The first
// step of a group (k = 0) has no fluid kernel of this group beside it, so its
// clearing takes a full-GPU grid.
lb_status launch_step_prologue(lb_ctx *h, int k, bool finish_prev, cudaStream_t st) {
    const int nb = (int)h->hb.size();
    const bool coupled = nb > 0 && !h->hbody_of.empty();
    const int cur = (int)((h->step + k) & 1);
    const int nsub = h->p.md_substeps;
    // with MD substeps the record is taken after the last substep's drift
    const lbk::Recorder rec{nsub == 1 ? h->rec : nullptr, h->rec_every, h->rec_cap, h->step_dev, (uint32_t)k};
    cudaError_t e = lbk::launch_step_pre(h->db, nb, finish_prev, coupled ? h->Fbuf[cur] : nullptr, h->fp32,
                                         coupled ? h->tiles[cur] : nullptr, h->tlist[cur], h->tcount[cur],
                                         h->list_cap, h->g, h->ntx, h->nty, rec, st, 1.0 / nsub, h->io_dmap,
                                         k == 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "step_pre launch");
    // the list of this buffer restarts empty for this step's coupling
    if (coupled) LB_CUDA(h, cudaMemsetAsync(h->tcount[cur], 0, sizeof(int), st));
    return LB_OK;
}

// The coupling of MD substep `sub` of step h->step + k on the main stream.
lb_status launch_step_coupling(lb_ctx *h, int k, int sub) {
    const int nbeads = (int)h->hbody_of.size();
    const long long t = h->step + k;
    const bool odd = (t & 1) != 0;
    const int cur = (int)(t & 1), prev = cur ^ 1;
    lbk::CoupleArgs c{};
    c.g = h->g;
    c.f = h->f_src ? h->f_src : h->f;
    c.fp32 = h->fp32;
    c.odd = odd;
    c.rho0 = h->p.rho0;
    c.rho0_f = (float)h->p.rho0;
    c.gamma = h->p.gamma_bead;
    const double dt = 1.0 / h->p.md_substeps;
    // bead noise of variance 2 kT gamma / dt per substep (Philox call 4 + sub)
    c.noise_amp = h->p.kT > 0.0 ? std::sqrt(2.0 * h->p.kT * h->p.gamma_bead / dt) : 0.0;
    c.dt = dt;
    c.dt_f = (float)dt;
    c.call = 4u + (uint32_t)sub;
    c.gforce = h->gforce;
    c.gforce_f = h->gforce_f;
    c.Fprev = h->Fbuf[prev];
    c.Fcur = h->Fbuf[cur];
    c.tiles_cur = h->tiles[cur];
    c.tlist = h->tlist[cur];
    c.tcount = h->tcount[cur];
    c.ntx = h->ntx;
    c.nty = h->nty;
    c.s = h->ds;
    c.sf = h->dsf;
    c.gamma_f = (float)c.gamma;
    c.noise_amp_f = (float)c.noise_amp;
    c.bead_body = h->dbody_of;
    c.bodies = h->db;
    c.F_bead = h->dFbead;
    c.nbeads = nbeads;
    c.key0 = (uint32_t)h->p.seed;
    c.key1 = (uint32_t)(h->p.seed >> 32);
    c.instance = h->p.instance;
    c.step_base = h->step_dev;
    c.step_off = (uint32_t)k;
    c.err = h->err_dev;
    c.ntiles = (long long)h->ntx * h->nty * h->ntz;
    c.list_cap = h->list_cap;
    c.nbodies = (int)h->hb.size();
    cudaError_t e = lbk::launch_couple(c, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "couple launch");
    e = lbk::launch_wall_beads(h->wall, h->db, h->ds, h->dbody_of, nbeads, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "wall beads launch");
    return LB_OK;
}

// Launches n steps starting at step h->step (without finishing the group).
// With bodies, the prologue of step k runs on the side stream beside the
// fluid kernel of step k-1: it needs the coupling of k-1 (body sums, and it
// clears the force buffer that coupling read as the previous step's) but
// touches nothing that fluid kernel reads (the other force buffer); the
// coupling of step k waits for it.
lb_status launch_steps(lb_ctx *h, int n) {
    const bool bodies = !h->hb.empty();
    lb_status s;
    if (bodies) {
        LB_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
        LB_CUDA(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        if ((s = launch_step_prologue(h, 0, false, h->side)) != LB_OK) return s;
    }
    for (int k = 0; k < n; ++k) {
        const long long t = h->step + k;
        const int cur = (int)(t & 1);
        if (bodies) {
            LB_CUDA(h, cudaEventRecord(h->ev_join, h->side));
            LB_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
            if (!h->hbody_of.empty()) {
                // MD substeps: bodies move by dt = 1/n between the couplings of one LB step
                const int nsub = h->p.md_substeps;
                for (int sub = 0; sub < nsub; ++sub) {
                    if (sub > 0) {
                        const lbk::Recorder rec{sub == nsub - 1 ? h->rec : nullptr, h->rec_every, h->rec_cap,
                                                h->step_dev, (uint32_t)k};
                        cudaError_t e = lbk::launch_substep(h->db, (int)h->hb.size(), 1.0 / nsub, rec, h->stream);
                        if (e != cudaSuccess) return cuda_fail(h, e, "substep launch");
                    }
                    if ((s = launch_step_coupling(h, k, sub)) != LB_OK) return s;
                }
            }
            if (k + 1 < n) {                  // the next prologue may start now
                LB_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
                LB_CUDA(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
                // enqueued before this step's fluid kernel (graph replay at
                // 256^3: 0.4675 against 0.4685 ms enqueued after it; eager
                // launches 0.4635 either way)
                if ((s = launch_step_prologue(h, k + 1, true, h->side)) != LB_OK) return s;
            }
        }
        if ((s = timed_collide(h, fluid_args(h, cur, (uint32_t)k), (t & 1) != 0)) != LB_OK) return s;
    }
    return LB_OK;
}

// end of a group of n steps: the last step's second half kick, counter advance
lb_status finish_group(lb_ctx *h, int n) {
    cudaError_t e = lbk::launch_finish(h->db, (int)h->hb.size(), 1.0 / h->p.md_substeps, h->step_dev, (unsigned)n,
                                       h->stream, h->io_dmap ? h->io_dmap + 6 * h->hb.size() : nullptr, h->err_dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "finish launch");
    return LB_OK;
}

lb_status eager_steps(lb_ctx *h, int n) {
    lb_status s = launch_steps(h, n);
    if (s != LB_OK) return s;
    s = finish_group(h, n);
    h->step += n;
    return s;
}

// Eight steps (n = 8) or an even and an odd step (n = 2) as one CUDA graph,
// replayed from even step counts; one step from the current parity as its
// own graph (n = 1), so a caller stepping one step at a time submits one
// launch per step. Long calls replay the eight-step graph: fewer graph
// launches, and the body kick and counter advance that close each group run
// once per eight steps (measured on GB300 at 256^3 with 64 bodies: 0.4672
// against 0.4695 ms per step with the pair graph).
lb_status ensure_graph(lb_ctx *h, int n = 2) {
    cudaGraphExec_t &slot = n == LB_GRAPH_STEPS ? h->gexec8 : (n == 2 ? h->gexec : h->gexec1[h->step & 1]);
    if (slot) return LB_OK;
    cudaGraph_t graph = nullptr;
    LB_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    lb_status s = launch_steps(h, n);
    if (s == LB_OK) s = finish_group(h, n);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (s != LB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
    e = cudaGraphInstantiate(&slot, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
    return LB_OK;
}

}  // namespace

namespace {
lb_status step_groups(lb_ctx *h, int nsteps);
}

lb_status lb_step(lb_handle h, int nsteps) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    const lb_status s = step_groups(h, nsteps);
    if (s == LB_OK && nsteps > 0 && h->ev_io) {
        // the external forces are read and the totals written by these steps
        LB_CUDA(h, cudaEventRecord(h->ev_io, h->stream));
        h->out_fresh = true;
    }
    return s;
}

namespace {
lb_status step_groups(lb_ctx *h, int nsteps) {
    if (nsteps < 0) return fail(h, LB_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return LB_OK;
    lb_status s = upload_bodies(h);
    if (s != LB_OK) return s;
    // timed kernels and the TMA variant launch step by step; short calls
    // replay single-step graphs
    if (h->timing || h->cs_variant == 2) return eager_steps(h, nsteps);
    // Long calls on a large lattice launch eagerly: there the device step
    // outlasts the host's launches, and the eager step measured faster than
    // the replayed graph (256^3: 0.4633 against 0.4672 ms; 128^3: 0.0769
    // against 0.0823), whatever the graph's length
    if (nsteps >= 4 && h->g.N >= LB_EAGER_NODES) return eager_steps(h, nsteps);
    if (nsteps < 4) {
        for (int k = 0; k < nsteps; ++k) {
            if ((s = ensure_graph(h, 1)) != LB_OK) return s;
            LB_CUDA(h, cudaGraphLaunch(h->gexec1[h->step & 1], h->stream));
            h->step += 1;
        }
        return LB_OK;
    }
    if (h->step & 1) {
        if ((s = eager_steps(h, 1)) != LB_OK) return s;
        --nsteps;
    }
    const int octets = nsteps / LB_GRAPH_STEPS;
    if (octets > 0) {
        if ((s = ensure_graph(h, LB_GRAPH_STEPS)) != LB_OK) return s;
        for (int r = 0; r < octets; ++r) LB_CUDA(h, cudaGraphLaunch(h->gexec8, h->stream));
        h->step += (long long)LB_GRAPH_STEPS * octets;
        nsteps -= LB_GRAPH_STEPS * octets;
    }
    const int pairs = nsteps / 2;
    if (pairs > 0) {
        if ((s = ensure_graph(h)) != LB_OK) return s;
        for (int r = 0; r < pairs; ++r) LB_CUDA(h, cudaGraphLaunch(h->gexec, h->stream));
        h->step += 2LL * pairs;
    }
    if (nsteps & 1) return eager_steps(h, 1);
    return LB_OK;
}
}  // namespace

}  // extern "C"

namespace lbk {
// The first part of step h->step as the adjoint's turn needs it: the body
// prologue (kick, drift, clearing of the step's spread-force tiles) and the
// bead coupling, both on the main stream, without the fluid kernel and the
// group's finishing launch. The handle is left partly stepped; the caller
// restores a whole state before stepping it again.
lb_status ctx_turn(lb_ctx *h, const void *src) {
    h->f_src = src != h->f ? src : nullptr;
    lb_status s = launch_step_prologue(h, 0, false, h->stream);
    if (s == LB_OK && !h->hbody_of.empty()) s = launch_step_coupling(h, 0, 0);
    h->f_src = nullptr;
    return s;
}

// One whole step (deterministic fluid, launched eagerly) that reads the
// populations at src and leaves the next state's at dst (either may be the
// handle's own array; src == dst == f is the ordinary in-place step). The
// handle's other state (bodies, forces, tiles, step count) advances in place.
lb_status ctx_step_oop(lb_ctx *h, const void *src, void *dst) {
    if (src == dst && dst != h->f) return ctx_fail(h, LB_ERR_ARG, "out-of-place step into its own source");
    if (h->p.collision == 1 && h->p.kT > 0.0) return ctx_fail(h, LB_ERR_STATE, "out-of-place steps are deterministic");
    lb_status s = upload_bodies(h);
    if (s != LB_OK) return s;
    h->f_src = src != h->f ? src : nullptr;
    h->f_dst = dst != h->f ? dst : nullptr;
    s = eager_steps(h, 1);
    h->f_src = nullptr;
    h->f_dst = nullptr;
    return s;
}
}  // namespace lbk

extern "C" {

lb_status lb_forces(lb_handle h, int id, double F[3], double T[3], double *per_bead) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (id < 0 || id >= (int)h->hb.size()) return fail(h, LB_ERR_ARG, "bad body id");
    if (!h->uploaded) {
        for (int a = 0; a < 3; ++a) {
            if (F) F[a] = 0.0;
            if (T) T[a] = 0.0;
        }
        if (per_bead)
            std::memset(per_bead, 0, sizeof(double) * 3 * (h->bead_start[id + 1] - h->bead_start[id]));
        return LB_OK;
    }
    if (F) LB_CUDA(h, cudaMemcpyAsync(F, &h->db[id].F_tot[0], 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (T) LB_CUDA(h, cudaMemcpyAsync(T, &h->db[id].T_tot[0], 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    const int b0 = h->bead_start[id], b1 = h->bead_start[id + 1];
    if (per_bead && b1 > b0)
        LB_CUDA(h, cudaMemcpyAsync(per_bead, h->dFbead + 3 * (size_t)b0, sizeof(double) * 3 * (b1 - b0),
                                   cudaMemcpyDeviceToHost, h->stream));
    return check_device_error(h);
}

lb_status lb_step_io(lb_handle h, int nsteps, int nbodies, const double *F_ext, const double *T_ext, double *F,
                     double *T) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    lb_status s = LB_OK;
    if (F_ext) s = lb_set_external_forces(h, nbodies, F_ext, T_ext);
    if (s == LB_OK) s = lb_step(h, nsteps);
    if (s == LB_OK && (F || T)) s = lb_forces_all(h, nbodies, F, T);
    return s;
}

lb_status lb_forces_all(lb_handle h, int nbodies, double *F, double *T) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (nbodies < 0 || nbodies > (int)h->hb.size()) return fail(h, LB_ERR_ARG, "bad body count");
    if (nbodies == 0) return LB_OK;
    if (!h->uploaded) {
        if (F) std::memset(F, 0, sizeof(double) * 3 * nbodies);
        if (T) std::memset(T, 0, sizeof(double) * 3 * nbodies);
        return LB_OK;
    }
    if (h->io_map && h->out_fresh) {
        // the totals and the error word of the last group, written by its
        // finishing launch into host-mapped memory: no copy
        LB_CUDA(h, cudaStreamSynchronize(h->stream));
        const size_t nbt = h->hb.size();
        const double *out = h->io_map + 6 * nbt;
        const int err = (int)out[6 * nbt];
        if (err) {
            h->io_map[12 * nbt] = 0.0;
            LB_CUDA(h, cudaMemsetAsync(h->err_dev, 0, sizeof(int), h->stream));
            if (err & 2) return fail(h, LB_ERR_STATE, "an index check of the checked build failed (an index outside its array)");
            return fail(h, LB_ERR_TIMEOUT, "a bounded device wait ran out (TMA copy did not complete in time)");
        }
        for (int b = 0; b < nbodies; ++b)
            for (int a = 0; a < 3; ++a) {
                if (F) F[3 * b + a] = out[6 * b + a];
                if (T) T[3 * b + a] = out[6 * b + 3 + a];
            }
        return LB_OK;
    }
    if (F) LB_CUDA(h, cudaMemcpy2DAsync(F, 3 * sizeof(double), &h->db[0].F_tot[0], sizeof(Body), 3 * sizeof(double),
                                        nbodies, cudaMemcpyDeviceToHost, h->stream));
    if (T) LB_CUDA(h, cudaMemcpy2DAsync(T, 3 * sizeof(double), &h->db[0].T_tot[0], sizeof(Body), 3 * sizeof(double),
                                        nbodies, cudaMemcpyDeviceToHost, h->stream));
    return check_device_error(h);
}

lb_status lb_get_body(lb_handle h, int id, double X[3], double V[3], double q[4], double w[3]) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (id < 0 || id >= (int)h->hb.size()) return fail(h, LB_ERR_ARG, "bad body id");
    lb_status s = pull_bodies(h);
    if (s != LB_OK) return s;
    const Body &b = h->hb[id];
    for (int a = 0; a < 3; ++a) {
        if (X) X[a] = b.X[a];
        if (V) V[a] = b.V[a];
        if (w) w[a] = b.w[a];
    }
    if (q)
        for (int a = 0; a < 4; ++a) q[a] = b.q[a];
    return LB_OK;
}

lb_status lb_get_populations(lb_handle h, double *host, size_t n) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!host || n != 19 * (size_t)h->g.N) return fail(h, LB_ERR_ARG, "buffer must hold 19*N doubles");
    double *tmp = nullptr;
    lb_status s = dev_alloc(h, &tmp, sizeof(double) * n);
    if (s != LB_OK) return s;
    h->dev_bytes -= sizeof(double) * n;
    cudaError_t e = lbk::launch_gather(h->f, h->fp32, h->g, (h->step & 1) != 0, h->p.rho0, tmp, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_get_populations");
    return LB_OK;
}

lb_status lb_set_populations(lb_handle h, const double *host, size_t n) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!host || n != 19 * (size_t)h->g.N) return fail(h, LB_ERR_ARG, "buffer must hold 19*N doubles");
    double *tmp = nullptr;
    lb_status s = dev_alloc(h, &tmp, sizeof(double) * n);
    if (s != LB_OK) return s;
    h->dev_bytes -= sizeof(double) * n;
    cudaError_t e = cudaMemcpyAsync(tmp, host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = lbk::launch_scatter(h->f, h->fp32, h->g, (h->step & 1) != 0, h->p.rho0, tmp, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_set_populations");
    return LB_OK;
}

lb_status lb_sample_populations(lb_handle h, const long long *nodes, int count, double *out) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (count < 0 || (count > 0 && (!nodes || !out))) return fail(h, LB_ERR_ARG, "bad sample arguments");
    if (count == 0) return LB_OK;
    for (int k = 0; k < count; ++k)
        if (nodes[k] < 0 || nodes[k] >= h->g.N) return fail(h, LB_ERR_ARG, "node index out of range");
    long long *dn = nullptr;
    double *dout = nullptr;
    lb_status s = dev_alloc(h, &dn, sizeof(long long) * count);
    if (s != LB_OK) return s;
    h->dev_bytes -= sizeof(long long) * count;
    s = dev_alloc(h, &dout, sizeof(double) * 19 * count);
    if (s != LB_OK) { cudaFree(dn); return s; }
    h->dev_bytes -= sizeof(double) * 19 * count;
    cudaError_t e = cudaMemcpyAsync(dn, nodes, sizeof(long long) * count, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = lbk::launch_sample(h->f, h->fp32, h->g, (h->step & 1) != 0, h->p.rho0, dn, count, dout, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * 19 * count, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dn);
    cudaFree(dout);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_sample_populations");
    return LB_OK;
}

lb_status lb_get_node_force(lb_handle h, double *host, size_t n) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!host || n != 3 * (size_t)h->g.N) return fail(h, LB_ERR_ARG, "buffer must hold 3*N doubles");
    if (!h->Fbuf[0] || h->step == 0) {
        std::memset(host, 0, sizeof(double) * n);
        return LB_OK;
    }
    const int last = (int)((h->step - 1) & 1);
    if (h->fp32) {
        std::vector<float> tmp(n);
        LB_CUDA(h, cudaMemcpyAsync(tmp.data(), h->Fbuf[last], sizeof(float) * n, cudaMemcpyDeviceToHost, h->stream));
        LB_CUDA(h, cudaStreamSynchronize(h->stream));
        for (size_t k = 0; k < n; ++k) host[k] = tmp[k];
        return LB_OK;
    }
    LB_CUDA(h, cudaMemcpyAsync(host, h->Fbuf[last], sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    return LB_OK;
}

lb_status lb_conservation(lb_handle h, double *mass, double mom[3]) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    double o[4];
    cudaError_t e = lbk::launch_moments(h->f, h->fp32, h->g, (h->step & 1) != 0, h->partials, h->red_blocks,
                                        h->out4, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(o, h->out4, sizeof(o), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_conservation");
    lb_status de = check_device_error(h);
    if (de != LB_OK) return de;
    if (h->fp32) o[0] += h->p.rho0 * (double)h->nfluid;
    if (mass) *mass = o[0];
    if (mom)
        for (int a = 0; a < 3; ++a) mom[a] = o[a + 1];
    for (double v : o)
        if (!std::isfinite(v)) return fail(h, LB_ERR_UNSTABLE, "non-finite mass or momentum");
    return LB_OK;
}

lb_status lb_info(lb_handle h, lb_info_t *info) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!info) return fail(h, LB_ERR_ARG, "null info");
    info->nodes = h->g.N;
    info->fluid_nodes = h->nfluid;
    info->step = h->step;
    info->nbodies = (int)h->hb.size();
    info->nbeads = (int)h->hbody_of.size();
    info->precision = h->fp32 ? 32 : 64;
    info->device_bytes = h->dev_bytes;
    return LB_OK;
}

lb_status lb_set_kernel_variant(lb_handle h, int variant, int stages, int ctas_per_sm) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    drop_graph(h);
    if (variant < 0 || variant > 2 || stages < 0 || stages > 6 || ctas_per_sm < 0 || ctas_per_sm > 8)
        return fail(h, LB_ERR_ARG, "variant 0-2, stages 0-6, ctas_per_sm 0-8");
    if (variant == 2 && !lbk::tma_collide_supported(h->g, h->fp32))
        return fail(h, LB_ERR_ARG, "the TMA-staged kernel needs FP32 storage, no pore and nx % 4 == 0");
    h->cs_variant = variant;
    h->tma_stages = stages;
    h->tma_ctas = ctas_per_sm;
    return LB_OK;
}

// ------------------------------------------------------------- checkpoints
namespace {

struct CkptHeader {
    char magic[8];
    int nx, ny, nz, precision, collision, nbodies, nbeads, pore_axis, chan, list_cap;
    double pore_R;
    unsigned long long seed;
    long long step, ntiles;
    unsigned long long body_bytes, total;
};

// the sections of a checkpoint: device pointer and bytes, in file order
std::vector<std::pair<void *, size_t>> ckpt_sections(lb_ctx *h) {
    std::vector<std::pair<void *, size_t>> v;
    const size_t es = h->fp32 ? 4 : 8;
    v.push_back({h->f, 19 * es * (size_t)h->g.N});
    const int nb = (int)h->hb.size(), nbeads = (int)h->hbody_of.size();
    if (nb > 0) {
        v.push_back({h->db, sizeof(Body) * nb});
        v.push_back({h->dFbead, sizeof(double) * 3 * (size_t)std::max(nbeads, 1)});
        const size_t ntiles = (size_t)h->ntx * h->nty * h->ntz;
        for (int k = 0; k < 2; ++k) {
            v.push_back({h->Fbuf[k], 3 * es * (size_t)h->g.N});
            v.push_back({h->tiles[k], sizeof(int) * ntiles});
            v.push_back({h->tlist[k], sizeof(int) * (size_t)h->list_cap});
            v.push_back({h->tcount[k], sizeof(int)});
        }
        // the external forces staged for the next step
        if (h->io_dmap) v.push_back({h->io_dmap, sizeof(double) * 6 * (size_t)nb});
    }
    return v;
}

CkptHeader ckpt_header(lb_ctx *h) {
    CkptHeader c{};
    std::memcpy(c.magic, "LBCKPT1", 8);
    c.nx = h->g.nx; c.ny = h->g.ny; c.nz = h->g.nz;
    c.precision = h->fp32 ? 32 : 64;
    c.collision = h->p.collision;
    c.nbodies = (int)h->hb.size();
    c.nbeads = (int)h->hbody_of.size();
    c.pore_axis = h->g.pore_axis;
    c.chan = h->g.chan;
    c.list_cap = h->list_cap;
    c.pore_R = h->pore_R;
    c.seed = h->p.seed;
    c.step = h->step;
    c.ntiles = (long long)h->ntx * h->nty * h->ntz;
    c.body_bytes = sizeof(Body);
    size_t total = sizeof(CkptHeader);
    for (auto &s : ckpt_sections(h)) total += s.second;
    c.total = total;
    return c;
}

}  // namespace

lb_status lb_checkpoint_size(lb_handle h, size_t *bytes) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!bytes) return fail(h, LB_ERR_ARG, "null argument");
    lb_status s = upload_bodies(h);
    if (s != LB_OK) return s;
    *bytes = (size_t)ckpt_header(h).total;
    return LB_OK;
}

lb_status lb_checkpoint_save(lb_handle h, void *host, size_t bytes) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!host) return fail(h, LB_ERR_ARG, "null buffer");
    lb_status s = upload_bodies(h);
    if (s != LB_OK) return s;
    const CkptHeader c = ckpt_header(h);
    if (bytes < c.total) return fail(h, LB_ERR_ARG, "buffer smaller than lb_checkpoint_size");
    char *p = static_cast<char *>(host);
    std::memcpy(p, &c, sizeof(c));
    p += sizeof(c);
    for (auto &sec : ckpt_sections(h)) {
        LB_CUDA(h, cudaMemcpyAsync(p, sec.first, sec.second, cudaMemcpyDeviceToHost, h->stream));
        p += sec.second;
    }
    return check_device_error(h);
}

lb_status lb_checkpoint_load(lb_handle h, const void *host, size_t bytes) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!host || bytes < sizeof(CkptHeader)) return fail(h, LB_ERR_ARG, "buffer too small for a checkpoint");
    CkptHeader c;
    std::memcpy(&c, host, sizeof(c));
    if (std::memcmp(c.magic, "LBCKPT1", 8) != 0) return fail(h, LB_ERR_ARG, "not a checkpoint of this library");
    lb_status s = upload_bodies(h);
    if (s != LB_OK) return s;
    const CkptHeader mine = ckpt_header(h);
    if (c.nx != mine.nx || c.ny != mine.ny || c.nz != mine.nz || c.precision != mine.precision ||
        c.collision != mine.collision || c.nbodies != mine.nbodies || c.nbeads != mine.nbeads ||
        c.pore_axis != mine.pore_axis || c.chan != mine.chan || c.list_cap != mine.list_cap ||
        c.pore_R != mine.pore_R || c.seed != mine.seed || c.ntiles != mine.ntiles ||
        c.body_bytes != mine.body_bytes || c.total != mine.total)
        return fail(h, LB_ERR_STATE, "the checkpoint was taken from a lattice with other parameters or bodies");
    if (bytes < c.total) return fail(h, LB_ERR_ARG, "buffer shorter than the checkpoint");
    drop_graph(h);
    const char *p = static_cast<const char *>(host) + sizeof(c);
    for (auto &sec : ckpt_sections(h)) {
        LB_CUDA(h, cudaMemcpyAsync(sec.first, p, sec.second, cudaMemcpyHostToDevice, h->stream));
        p += sec.second;
    }
    const unsigned long long st = (unsigned long long)c.step;
    LB_CUDA(h, cudaMemcpyAsync(h->step_dev, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    h->step = c.step;
    h->out_fresh = false;                 // the loaded totals are read by copy until the next step
    if (h->io_map) {                      // the loaded external forces become the host's
        const size_t nb = h->hb.size();
        for (size_t b = 0; b < nb; ++b)
            for (int a = 0; a < 3; ++a) {
                h->hb[b].F_ext[a] = h->io_map[3 * b + a];
                h->hb[b].T_ext[a] = h->io_map[3 * nb + 3 * b + a];
            }
        return push_gforce(h);
    }
    return LB_OK;
}

lb_status lb_set_wait_limit(lb_handle h, long long cycles) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (cycles < 0) return fail(h, LB_ERR_ARG, "cycles must be >= 0 (0: the default of ~2 s)");
    h->wait_limit = cycles;
    return LB_OK;
}

lb_status lb_record_bodies(lb_handle h, int every, int capacity) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    drop_graph(h);
    if (every < 0 || (every > 0 && capacity < 1)) return fail(h, LB_ERR_ARG, "every >= 0 and capacity >= 1");
    if (every > 0 && h->hb.empty()) return fail(h, LB_ERR_ARG, "no bodies to record");
    if (h->rec) {
        LB_CUDA(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->rec);
        h->dev_bytes -= sizeof(double) * 7 * (size_t)h->rec_cap * h->hb.size();
        h->rec = nullptr;
    }
    h->rec_every = h->rec_cap = 0;
    if (every == 0) return LB_OK;
    lb_status s = upload_bodies(h);        // the body set is fixed from here on
    if (s != LB_OK) return s;
    if ((s = dev_alloc(h, &h->rec, sizeof(double) * 7 * (size_t)capacity * h->hb.size())) != LB_OK) return s;
    h->rec_every = every;
    h->rec_cap = capacity;
    h->rec_k0 = h->step / every + 1;
    return LB_OK;
}

lb_status lb_get_trajectory(lb_handle h, int body, int max_records, long long *steps, double *X, double *q,
                            int *count) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    if (!count || max_records < 0) return fail(h, LB_ERR_ARG, "count must not be NULL, max_records >= 0");
    if (body < 0 || body >= (int)h->hb.size()) return fail(h, LB_ERR_ARG, "bad body id");
    cudaError_t e = lbk::copy_records(h->rec, h->rec_every, h->rec_cap, h->rec_k0, h->step, (int)h->hb.size(), body,
                                      max_records, steps, X, q, count, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_get_trajectory");
    return LB_OK;
}

lb_status lb_set_timing(lb_handle h, int on) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    h->timing = on != 0;
    return LB_OK;
}

lb_status lb_kernel_time(lb_handle h, double *total_ms, long long *launches) {
    if (check_handle(h) != LB_OK) return LB_ERR_ARG;
    LB_CUDA(h, cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float ms = 0.f;
        LB_CUDA(h, cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
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
