// Internal launch interface between the C-ABI runtime (lb_api.cu) and the
// kernels (lb_fluid.cu, lb_bodies.cu). Not part of the public ABI.
#pragma once

#include <cmath>
#include <cuda_runtime.h>
#include <cstdint>

#include "lb_device.cuh"

namespace lbk {

// Collision parameters in the compute precision of the kernel (the FP32
// kernel gets them pre-rounded on the host, so it converts nothing).
template <typename R>
struct CollParams {
    R rho0;
    R omega;                     // BGK 1/tau
    // MRT, per mode k with c_k = w_diag / b_k folded in (modes 4-9):
    R ke[6];                     // c_k (1 - g_k): weight of the equilibrium moment
    R km[6];                     // c_k g_k: weight of the pre-collision moment
    R ks[6];                     // c_k (1 + g_k)/2: weight of the Guo source moment
    R kg[9];                     // ghost modes 10-18: c_k g_k
    R kn[15];                    // noise modes 4-18: c_k sqrt(3 kT b_k (1 - g_k^2)) sqrt(12) / sqrt(rho),
                                 //   applied to a centred uniform variate in (-1/2, 1/2) (FP32: times 2^-32)
};

// Everything the fused collide-and-stream kernel reads besides populations.
struct FluidArgs {
    Geom g;
    void *f;                     // populations: double[19][N] (FP64) or float[19][N] deviations
    CollParams<double> pd;
    CollParams<float> pf;
    const double *gforce;        // device: uniform force density (3)
    const float *gforce_f;       // device: the same, rounded to FP32
    const void *Fn;              // device: spread bead force [3][N] in the storage precision, or nullptr
    const int *tiles;            // device: 4x4x4 tile flags of Fn or nullptr
    int ntx, nty;
    uint32_t key0, key1, instance;
    const unsigned long long *step_base;  // device step counter of the first step of this launch group
    uint32_t step_off;
    int *err;                    // device error word (a bounded wait ran out), may be null
    void *plane[19];             // base of each population plane (f + i N), uniform per launch
    const uint32_t *masks;       // pore: per position across the axis, bit 31 wall node, bit i the
                                 // upstream node of link i is a wall (launch_build_masks)
    void *out[19];               // out-of-place step (launch_collide_stream_oop): where each plane's
                                 // populations are stored; the loads read f / plane
};

// Rigid bodies (FP64, array of structs; few bodies, one thread each).
struct Body {
    double X[3], V[3], q[4], w[3];   // centre, velocity, orientation (w,x,y,z), body-frame omega
    double F_last[3], T_last[3];     // last step: lab-frame force, body-frame torque
    double F_ext[3], T_ext[3];       // lab frame
    double F_tot[3], T_tot[3];       // last step: lab-frame totals (beads + external)
    double acc[6];                   // bead force / torque accumulators of the running step
    double R[9];                     // rotation of the running step (row-major, lab = R body)
    double wl[3];                    // lab-frame omega of the running step
    double mass, I[3];
    double inv_mass, inv_I[3];       // reciprocals, so the step divides nothing
    // the running step's state in FP32 for the FP32 coupling: rotation,
    // velocity, lab omega, and X - 1/2 split into floor (Xi) and fraction (Xf)
    float Rf[9], Vf[3], wlf[3], Xf[3];
    int Xi[3];
    int fixed;
    int inst;                        // instance of a batch (0 for a single lattice)
};

// Repulsive pore-wall beads (Sec. 2.3): beads on the cylinder of radius Rc
// (pore radius + pore-bead radius) around the pore axis, ntheta around and
// nrow along it, WCA with sigma^2 = sigma2 and epsilon = eps up to
// rcut2 = 2^(1/3) sigma^2, acting on colloid beads only. wt, wz: half
// widths of the window of wall beads around a bead's nearest one that can
// lie within the cutoff (host-computed; the whole ring or row when large).
struct WallBeads {
    int on, axis, ntheta, nrow, wt, wz;
    double cu, cv;               // axis position across it (box centre)
    double Rc, L, sigma2, rcut2, eps;
};

// wall-bead parameters from the user's (host; lb_fluid.cu); false if invalid
bool make_wall_beads(const Geom &g, double pore_R, double spacing, double r_pore_bead, double r_bead, double eps,
                     WallBeads &w);

struct CoupleArgs {
    Geom g;
    const void *f;               // populations (pre-collision of this step)
    bool fp32;                   // deviation storage
    bool odd;                    // parity of the step count
    double rho0;
    double gamma;
    double noise_amp;            // sqrt(2 kT gamma), 0 = off
    const double *gforce;        // uniform force density (3)
    const void *Fprev;           // [3][N] spread force of the previous step (storage precision)
    void *Fcur;                  // [3][N] spread force of this step (zero on entry)
    const float *gforce_f;       // uniform force density rounded to FP32
    int *tiles_cur;              // flags of Fcur
    int *tlist;                  // flagged tiles of Fcur, in the order they were flagged
    int *tcount;                 // entries of tlist
    int tile_base;               // added to tile indices recorded in tlist (batch pools)
    int ntx, nty;
    const double *s;             // body-frame bead offsets [3*nbeads]
    const float *sf;             // the same in FP32 (FP32 coupling)
    float gamma_f, noise_amp_f;  // gamma and noise_amp in FP32
    float rho0_f;                // rho0 in FP32
    const int *bead_body;        // body index of each bead
    Body *bodies;
    double *F_bead;              // out: bead forces [3*nbeads]
    int nbeads;
    uint32_t key0, key1, instance;
    const unsigned long long *step_base;
    uint32_t step_off;
    // extents for the index checks of checked builds (LB_CHECKS); err may be null
    int *err;
    long long ntiles;
    int list_cap, nbodies;
    // MD substeps: the fluid receives -w dt F_b of this substep (dt = 1 without
    // substeps); Philox call word of the bead noise, 4 + substep
    double dt;
    float dt_f;
    uint32_t call;
};

// launchers (return the launch error)
cudaError_t launch_init(void *f, bool fp32, long long N, double rho0, cudaStream_t s);
cudaError_t launch_collide_stream(const FluidArgs &a, bool fp32, int collision, bool noise, bool odd,
                                  dim3 block, cudaStream_t s);
// the same step out of place (deterministic fluid): loads from f / plane,
// stores into out, in the AA layout of the next step; every slot of a fluid
// node is written, the slots of wall nodes are not
cudaError_t launch_collide_stream_oop(const FluidArgs &a, bool fp32, int collision, bool odd, dim3 block,
                                      cudaStream_t s);
// TMA-staged variant (FP32 storage, periodic, nx % 4 == 0); cudaErrorNotSupported otherwise
bool tma_collide_supported(const Geom &g, bool fp32);
// positions across the pore axis: nx*ny (axis z), nx*nz (axis y), ny*nz (axis x)
long long pore_section_size(const Geom &g);
// wall masks of a pore geometry into out[pore_section_size(g)]
cudaError_t launch_build_masks(const Geom &g, uint32_t *out, cudaStream_t s);
// wait_limit: SM clock cycles a stage's wait may take before the launch gives up
// (error word set); <= 0 selects ~2 s
cudaError_t launch_collide_stream_tma(const FluidArgs &a, int collision, bool noise, bool odd, int stages_hint,
                                      int ctas_per_sm_hint, long long wait_limit, cudaStream_t s);
cudaError_t launch_gather(const void *f, bool fp32, const Geom &g, bool odd, double rho0, double *out,
                          cudaStream_t s);
cudaError_t launch_scatter(void *f, bool fp32, const Geom &g, bool odd, double rho0, const double *in,
                           cudaStream_t s);
cudaError_t launch_sample(const void *f, bool fp32, const Geom &g, bool odd, double rho0,
                          const long long *nodes, int count, double *out, cudaStream_t s);
cudaError_t launch_moments(const void *f, bool fp32, const Geom &g, bool odd, double *partials,
                           int nblocks, double *out4, cudaStream_t s);

// Trajectory recorder: after the drift of step t, if (t + 1) % every == 0,
// the step prologue writes every body's centre and orientation (7 doubles,
// X then q) into record slot ((t + 1) / every - 1) % cap of `ring`
// ([cap][nbodies][7]). ring == nullptr: off.
struct Recorder {
    double *ring;
    int every, cap;
    const unsigned long long *step_base;
    uint32_t step_off;
};

// dt: the MD (sub)step, 1 without substeps
cudaError_t launch_step_pre(Body *b, int nbodies, bool finish_prev, void *F, bool fp32, int *tiles, const int *tlist,
                            const int *tcount, int list_cap, const Geom &g, int ntx, int nty, const Recorder &rec,
                            cudaStream_t s, double dt = 1.0, const double *ext = nullptr, bool alone = false);

// The valid records of body `id` in a recorder ring, oldest first (host
// arrays; lb_traj.cu).
cudaError_t copy_records(const double *ring, int every, int cap, long long k0, long long step, int nb, int id,
                         int max_records, long long *steps, double *X, double *q, int *count, cudaStream_t s);

// MSD analysis of recorded trajectories (lb_traj.cu); all pointers device
cudaError_t launch_msd(const double *X, const double *q, int nrec, int nbodies, int max_lag, const double *p_ref,
                       double *work, double *out, cudaStream_t s);
cudaError_t launch_couple(const CoupleArgs &a, cudaStream_t s);
// end of a group of steps: second half kick of every body and the step
// counter advance, in one launch (nbodies may be 0)
cudaError_t launch_finish(Body *b, int nbodies, double dt, unsigned long long *step, unsigned int by, cudaStream_t s,
                          double *out = nullptr, const int *err = nullptr);
// between MD substeps: second half kick, next first half kick and drift (dt each)
cudaError_t launch_substep(Body *b, int nbodies, double dt, const Recorder &rec, cudaStream_t s);
// force and torque of the pore-wall beads on every bead (after the coupling)
cudaError_t launch_wall_beads(const WallBeads &w, Body *b, const double *s, const int *bead_body, int nbeads,
                              cudaStream_t st);

// host-side argument check: all n values finite (a null pointer passes)
inline bool all_finite(const double *v, int n) {
    if (!v) return true;
    for (int k = 0; k < n; ++k)
        if (!std::isfinite(v[k])) return false;
    return true;
}

}  // namespace lbk
