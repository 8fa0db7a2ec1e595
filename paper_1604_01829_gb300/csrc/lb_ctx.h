// Host state of one lattice handle, shared by the C-ABI runtime (lb_api.cu)
// and the adjoint driver (lb_adjoint.cu). Not part of the public ABI.
#pragma once

#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_internal.h"

using lbk::Body;

struct AdjWork;   // the adjoint's device workspace (lb_adjoint.cu), kept between calls

struct lb_ctx {
    lb_params p{};
    lbk::Geom g{};
    bool fp32 = false;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;            // body prologue of step t beside the fluid kernel of t-1
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool own_stream = false;
    void *f = nullptr;
    // an out-of-place step (adjoint): the populations it reads (coupling and
    // fluid kernel) and where the fluid kernel stores them; null = f
    const void *f_src = nullptr;
    void *f_dst = nullptr;
    double *gforce = nullptr;               // device (3)
    float *gforce_f = nullptr;              // device (3), FP32 copy
    unsigned long long *step_dev = nullptr; // device step counter
    int *err_dev = nullptr;                 // device error word of bounded waits
    int *err_host = nullptr;                // pinned host copy of it (read in the caller's synchronisation)
    uint32_t *dmask = nullptr;              // pore wall masks across the axis (launch_build_masks)
    double pore_R = 0.0;                    // pore radius (lb_set_pore)
    double *dwchan = nullptr;               // channel walls: Geom::wchan
    lbk::WallBeads wall{};                  // pore-wall beads (lb_set_pore_beads)
    int cs_variant = 0;                     // collide kernel: 0 auto (plain), 1 plain, 2 TMA-staged
    int tma_stages = 0, tma_ctas = 0;       // 0 = library default
    long long wait_limit = 0;               // bounded device waits, SM clock cycles (0: ~2 s)
    long long step = 0;                     // host mirror
    long long nfluid = 0;
    double sig[15] = {};
    // bead force fields (double buffered) and their 4x4x4 tile flags
    void *Fbuf[2] = {nullptr, nullptr};     // [3][N] each, storage precision
    int *tiles[2] = {nullptr, nullptr};      // 4x4x4 tile flags of each force buffer
    int *tlist[2] = {nullptr, nullptr};      // flagged tiles of each buffer
    int *tcount[2] = {nullptr, nullptr};     // entries of tlist
    int list_cap = 0;
    int ntx = 0, nty = 0, ntz = 0;
    // bodies
    std::vector<Body> hb;
    std::vector<double> hs;
    std::vector<float> hsf;                  // bead offsets in FP32 (kept for the async upload)
    std::vector<int> hbody_of;
    std::vector<int> bead_start{0};
    Body *db = nullptr;
    double *ds = nullptr;
    float *dsf = nullptr;
    int *dbody_of = nullptr;
    double *dFbead = nullptr;
    // per-step body I/O in host-mapped pinned memory (Grace-Blackwell: the
    // GPU reads and writes it over the coherent chip-to-chip link, no copy):
    // [0, 6 nb) external forces then torques ([3 nb] each, host-written, read
    // by each step's prologue), [6 nb, 12 nb) force and torque totals per body
    // and [12 nb] the error word (written at the end of each group of steps)
    double *io_map = nullptr;          // host address
    double *io_dmap = nullptr;         // device address of the same memory
    cudaEvent_t ev_io = nullptr;       // after the last group that reads the external forces
    bool out_fresh = false;            // the totals there are those of the current state
    bool uploaded = false;
    // reductions
    double *partials = nullptr;
    double *out4 = nullptr;
    int red_blocks = 0;
    // trajectory recorder: ring [rec_cap][nbodies][7] (X, q), one record
    // every rec_every steps; records k >= rec_k0 (k = step / rec_every)
    double *rec = nullptr;
    int rec_every = 0, rec_cap = 0;
    long long rec_k0 = 0;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;   // pairs
    cudaGraphExec_t gexec = nullptr;   // an even and an odd step (lb_step)
    cudaGraphExec_t gexec8 = nullptr;  // eight steps from an even count (long lb_step calls)
    cudaGraphExec_t gexec1[2] = {nullptr, nullptr};   // one step from an even / odd count
    size_t ev_used = 0;
    double timed_ms = 0.0;
    long long timed_n = 0;
    dim3 block{128, 1, 1};
    size_t dev_bytes = 0;
    AdjWork *adjw = nullptr;
    double g_host[3] = {};
    float gf_host[3] = {};
    std::string err;
};


namespace lbk {
lb_status ctx_upload(lb_ctx *h);
lb_status ctx_apply_external(lb_ctx *h);
lb_status ctx_fail(lb_ctx *h, lb_status s, const std::string &m);
// the prologue and coupling of the next step, reading the populations at src
lb_status ctx_turn(lb_ctx *h, const void *src);
lb_status ctx_step_oop(lb_ctx *h, const void *src, void *dst);
void adj_free(lb_ctx *h);
}  // namespace lbk
