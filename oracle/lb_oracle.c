/*
 * FP64 CPU oracle for the lattice Boltzmann + raspberry-coupling step.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library. It shares no code,
 * header, table or constant generator with the CUDA library: every table
 * here is built from its own definition.
 *
 * It is written to be read against Ustach & Faller, "The Raspberry model for
 * protein-like particles" (arXiv:1604.01829):
 *   - Sec. 1.1: LB as streaming along discrete velocity links plus a
 *     collision that relaxes towards a Maxwell-Boltzmann equilibrium, either
 *     on one time scale (BGK) or mode by mode (multiple relaxation times);
 *     optional thermal noise ("stochastic or deterministic"); boundary nodes
 *     reflect the populations that stream into them (bounce-back).
 *   - Sec. 1.1, Eq. (latticeboltzmannfriction): bead force
 *     F = -xi_bead (v - u(r,t)) + f_s, u interpolated between the nearest
 *     grid points, f_s obeying fluctuation-dissipation.
 *   - Sec. 1.2 and Sec. 2.3: the raspberry is a rigid body; beads are virtual
 *     sites of the centre-of-mass particle; bead forces and torques act on
 *     it; translation by velocity Verlet, rotation by a quaternion.
 *   - Sec. 2.3: pore boundary nodes sit half a grid spacing outside the wall.
 * Points the paper leaves open are taken as follows (each reading is also
 * listed with the design notes):
 *   D3Q19 lattice; second-order equilibrium; Guo forcing with
 *   u = (j + F/2)/rho; orthogonal moment basis (Dunweg-Schiller-Ladd
 *   polynomials), m* = m_eq + g_k (m - m_eq) + (1+g_k)/2 S_k; fluctuating
 *   modes with amplitude sqrt(3 rho kT b_k (1-g_k^2)); Philox4x32-10
 *   uniform variates of unit variance (16-bit for the fluid modes, 32-bit
 *   for the beads); trilinear interpolation between the
 *   8 nodes surrounding a bead and the transposed spread of -F; node centres
 *   at integer+1/2; a node is a wall node when its centre lies at distance
 *   >= R from the pore axis.
 *
 * Deliberately plain: two population arrays and push streaming, the MRT
 * collision as explicit 19x19 matrix products with the inverse found by
 * Gauss-Jordan elimination, nested loops over beads and corners.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19

/* ---------------------------------------------------------------- lattice */

/* D3Q19 velocities: rest, 6 axis links, 12 face diagonals, each diagonal
 * followed by its opposite (Sec. 1.1 "discrete velocity links"). */
static const int CV[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double WQ[NQ];
static int OPP[NQ];
static double MM[NQ][NQ];   /* moment matrix M[k][i] = e_k(c_i)          */
static double MINV[NQ][NQ]; /* its inverse by Gauss-Jordan elimination   */
static double BK[NQ];       /* b_k = sum_i w_i e_k(c_i)^2                */
static int tables_ready = 0;

/* Moment polynomials e_k(c) of the orthogonal D3Q19 basis. */
static double basis_poly(int k, const int c[3])
{
    double x = c[0], y = c[1], z = c[2];
    double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return z * x;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
    }
    return 0.0;
}

/* Plain Gauss-Jordan inversion with partial pivoting; returns 0 on success. */
static int invert(int n, const double *a, double *inv)
{
    double *m = (double *)malloc(sizeof(double) * n * 2 * n);
    if (!m) return -1;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            m[r * 2 * n + c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(m[r * 2 * n + col]) > fabs(m[piv * 2 * n + col])) piv = r;
        if (fabs(m[piv * 2 * n + col]) < 1e-14) { free(m); return -1; }
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = m[col * 2 * n + c];
                m[col * 2 * n + c] = m[piv * 2 * n + c];
                m[piv * 2 * n + c] = t;
            }
        double d = m[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) m[col * 2 * n + c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fct = m[r * 2 * n + col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) m[r * 2 * n + c] -= fct * m[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = m[r * 2 * n + n + c];
    free(m);
    return 0;
}

static void init_tables(void)
{
    if (tables_ready) return;
    for (int i = 0; i < NQ; ++i) {
        int c2 = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
        WQ[i] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int j = 0; j < NQ; ++j)
            if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2])
                OPP[i] = j;
    }
    for (int k = 0; k < NQ; ++k) {
        BK[k] = 0.0;
        for (int i = 0; i < NQ; ++i) {
            MM[k][i] = basis_poly(k, CV[i]);
            BK[k] += WQ[i] * MM[k][i] * MM[k][i];
        }
    }
    invert(NQ, &MM[0][0], &MINV[0][0]);
    tables_ready = 1;
}

/* ----------------------------------------------------------------- Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
 * 32x32->64 multiplications with the round key bumped by the Weyl
 * constants between rounds. */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform variate of zero mean and unit variance from 32 random bits:
 * u = (x + 1/2) 2^-32 in (0,1), xi = sqrt(12) (u - 1/2). */
static double unit_uniform(uint32_t x)
{
    double u = ((double)x + 0.5) * (1.0 / 4294967296.0);
    return sqrt(12.0) * (u - 0.5);
}

/* The same from 16 random bits (the fluid noise): u = (h + 1/2) 2^-16. */
static double unit_uniform16(uint32_t h)
{
    double u = ((double)h + 0.5) * (1.0 / 65536.0);
    return sqrt(12.0) * (u - 0.5);
}

/* ------------------------------------------------------------- parameters */

typedef struct {
    int nx, ny, nz;
    int collision;          /* 0 BGK, 1 MRT */
    double tau;             /* BGK relaxation time */
    double gamma_shear, gamma_bulk, gamma_odd, gamma_even; /* MRT: m* - m_eq = g (m - m_eq) */
    double rho0;
    double kT;              /* thermal energy (MRT only) */
    double gamma_bead;      /* xi_bead of Eq. (latticeboltzmannfriction) */
    uint64_t seed;
    uint32_t instance;      /* third Philox counter word */
    double body_force[3];   /* uniform force density on the fluid */
    int compensate_force;   /* add -sum(F_ext)/N_fluid to the fluid */
    /* repulsive pore-wall beads (Sec. 2.3): beads on the cylinder of radius
       wall_R + wall_rp around the pore axis, wall_spacing apart around and
       along it, WCA with sigma = wall_rr + wall_rp, epsilon = wall_eps,
       acting on every colloid bead; their force goes to the body only */
    int wall_beads;
    int wall_axis;
    double wall_R, wall_spacing, wall_rp, wall_rr, wall_eps;
    /* moving walls normal to y (Sec. 2.3, the Stokes-flow set-up): the
       planes y = -1/2 and y = ny - 1/2 bound the fluid, moving with the
       tangential velocities uw_lo and uw_hi; the box is not periodic in y */
    int ywalls;
    double uw_lo[3], uw_hi[3];
    /* MD substeps per LB step (Sec. 2.3: the MD time step is half the LB
       step, so the paper's value is 2; 0 or 1 = one). Each substep moves the
       bodies by dt = 1/n and couples the beads to the fluid of this LB step;
       the fluid receives each substep's bead forces with weight dt. */
    int md_substeps;
} orc_params;

typedef struct {
    int nbodies;
    const int *bead_start;  /* nbodies + 1 offsets into the bead arrays */
    const double *s;        /* body-frame bead offsets, 3 per bead */
    double *X, *V, *q, *w;  /* per body: COM (3), velocity (3), quaternion w,x,y,z (4), body-frame omega (3) */
    double *F_last;         /* per body: lab-frame total force of the previous step (3) */
    double *T_last;         /* per body: body-frame total torque of the previous step (3) */
    const double *mass;     /* per body (1) */
    const double *inertia;  /* per body, principal moments (3) */
    const double *F_ext;    /* per body, lab frame (3) */
    const double *T_ext;    /* per body, lab frame (3) */
    const int *fixed;       /* per body: 1 = kinematics held, not integrated;
                               2 = translation integrated, orientation held (omega = 0) */
    double *F_bead;         /* out: lab-frame force on each bead (3 per bead) */
    double *F_tot, *T_tot;  /* out: per body, lab-frame total force and torque (3, 3) */
} orc_bodies;

static size_t nidx(const orc_params *p, int x, int y, int z)
{
    return (size_t)x + (size_t)p->nx * ((size_t)y + (size_t)p->ny * (size_t)z);
}

static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* Second-order equilibrium (Sec. 1.1 "Maxwell-Boltzmann" relaxation target). */
static void equilibrium(double rho, const double u[3], double feq[NQ])
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < NQ; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = WQ[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Guo source term s_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F */
static void guo_source(const double u[3], const double F[3], double s[NQ])
{
    for (int i = 0; i < NQ; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        double t = 0.0;
        for (int a = 0; a < 3; ++a) t += (3.0 * (CV[i][a] - u[a]) + 9.0 * cu * CV[i][a]) * F[a];
        s[i] = WQ[i] * t;
    }
}

static double mode_rate(const orc_params *p, int k)
{
    if (k < 4) return 0.0;              /* conserved: rate is irrelevant */
    if (k == 4) return p->gamma_bulk;
    if (k <= 9) return p->gamma_shear;
    if (k <= 15) return p->gamma_odd;
    return p->gamma_even;
}

/* Collision of one node (Sec. 1.1). f: pre-collision populations, F: force
 * density on the node, fout: post-collision populations. */
static void collide_node(const orc_params *p, const double f[NQ], const double F[3],
                         uint32_t node_id, uint32_t step, double fout[NQ])
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NQ; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += CV[i][a] * f[i];
    }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
    double feq[NQ], s[NQ];
    equilibrium(rho, u, feq);
    guo_source(u, F, s);

    if (p->collision == 0) {
        /* BGK: relax every population on the single time scale tau. */
        for (int i = 0; i < NQ; ++i)
            fout[i] = f[i] - (f[i] - feq[i]) / p->tau + (1.0 - 0.5 / p->tau) * s[i];
        return;
    }

    /* MRT: m = M f, relax each mode towards M f_eq with its own rate. */
    double m[NQ], meq[NQ], S[NQ], ms[NQ];
    for (int k = 0; k < NQ; ++k) {
        m[k] = meq[k] = S[k] = 0.0;
        for (int i = 0; i < NQ; ++i) {
            m[k] += MM[k][i] * f[i];
            meq[k] += MM[k][i] * feq[i];
            S[k] += MM[k][i] * s[i];
        }
    }
    for (int k = 0; k < NQ; ++k) {
        double g = mode_rate(p, k);
        ms[k] = meq[k] + g * (m[k] - meq[k]) + 0.5 * (1.0 + g) * S[k];
    }
    if (p->kT > 0.0) {
        /* Fluctuating modes: the 15 non-conserved moments get noise of
         * variance mu b_k (1 - g_k^2), mu = 3 rho kT, so that their
         * stationary variance is mu b_k. The variates are 16-bit: two
         * Philox calls give 8 words = 16 half-words; mode k takes half-word
         * j = k - 4, the high half of word j/2 for even j, the low half for
         * odd j. */
        uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
        uint32_t r[8];
        for (int call = 0; call < 2; ++call) {
            uint32_t ctr[4] = {node_id, step, p->instance, (uint32_t)call};
            philox4x32_10(ctr, key, &r[4 * call]);
        }
        double mu = 3.0 * rho * p->kT;
        for (int k = 4; k < NQ; ++k) {
            double g = mode_rate(p, k);
            int j = k - 4;
            uint32_t h = (j % 2 == 0) ? (r[j / 2] >> 16) : (r[j / 2] & 0xFFFFu);
            ms[k] += sqrt(mu * BK[k] * (1.0 - g * g)) * unit_uniform16(h);
        }
    }
    for (int i = 0; i < NQ; ++i) {
        fout[i] = 0.0;
        for (int k = 0; k < NQ; ++k) fout[i] += MINV[i][k] * ms[k];
    }
}

/* Hamilton rotation matrix of the unit quaternion q = (w, x, y, z):
 * lab vector = R body vector. */
static void rotation(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - z * w);
    R[0][2] = 2.0 * (x * z + y * w);
    R[1][0] = 2.0 * (x * y + z * w);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - x * w);
    R[2][0] = 2.0 * (x * z - y * w);
    R[2][1] = 2.0 * (y * z + x * w);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static void quat_mul(const double a[4], const double b[4], double o[4])
{
    double r[4];
    r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    memcpy(o, r, sizeof r);
}

static void cross(const double a[3], const double b[3], double o[3])
{
    double r[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    memcpy(o, r, sizeof r);
}

/* Half kicks of the body-frame angular velocity by Euler's equations,
 * I dw/dt = T - w x (I w), over dt/2. The kick before the drift is explicit
 * in w; the kick after it is implicit (fixed-point iteration), so that the
 * pair of half kicks around each step boundary is the trapezoidal rule and
 * the rotation integrator is second order and time-symmetric, the property
 * of the velocity-Verlet rotation schemes cited in Sec. 2.3. */
static void euler_half_kick(double w[3], const double I[3], const double T[3], double dt)
{
    double Iw[3] = {I[0] * w[0], I[1] * w[1], I[2] * w[2]}, wxIw[3];
    cross(w, Iw, wxIw);
    for (int a = 0; a < 3; ++a) w[a] += 0.5 * dt * (T[a] - wxIw[a]) / I[a];
}

#define IMPLICIT_KICK_ITERS 6

static void euler_half_kick_implicit(double w[3], const double I[3], const double T[3], double dt)
{
    double w0[3] = {w[0], w[1], w[2]};
    for (int it = 0; it < IMPLICIT_KICK_ITERS; ++it) {
        double Iw[3] = {I[0] * w[0], I[1] * w[1], I[2] * w[2]}, wxIw[3];
        cross(w, Iw, wxIw);
        for (int a = 0; a < 3; ++a) w[a] = w0[a] + 0.5 * dt * (T[a] - wxIw[a]) / I[a];
    }
}

/* ------------------------------------------------------- pore-wall beads */

#define ORC_PI 3.14159265358979323846

/* Ring and row counts of the wall-bead lattice and the pore-bead position
 * (j around, k along the axis). The axis passes through the box centre; the
 * beads sit at (k + 1/2) L / n_rows along it. */
static void wall_lattice(const orc_params *p, int *nth, int *nrow)
{
    int n[3] = {p->nx, p->ny, p->nz};
    double Rc = p->wall_R + p->wall_rp;
    *nth = (int)lround(2.0 * ORC_PI * Rc / p->wall_spacing);
    if (*nth < 3) *nth = 3;
    *nrow = (int)lround(n[p->wall_axis] / p->wall_spacing);
    if (*nrow < 1) *nrow = 1;
}

/* WCA force on a colloid bead at r (lab frame) from every wall bead, with
 * the minimum image along the periodic axis:
 *   U(d) = 4 eps ((sigma/d)^12 - (sigma/d)^6) + eps for d < 2^(1/6) sigma,
 *   F = -dU/dd along d = r - r_wall: 24 eps (2 (sigma/d)^12 - (sigma/d)^6) d / d^2. */
static void wall_bead_force(const orc_params *p, const double r[3], double F[3])
{
    F[0] = F[1] = F[2] = 0.0;
    if (!p->wall_beads) return;
    int n[3] = {p->nx, p->ny, p->nz};
    int ax = p->wall_axis, a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
    int nth, nrow;
    wall_lattice(p, &nth, &nrow);
    double Rc = p->wall_R + p->wall_rp, L = n[ax];
    double sigma = p->wall_rr + p->wall_rp;
    double rcut2 = pow(2.0, 1.0 / 3.0) * sigma * sigma;
    for (int k = 0; k < nrow; ++k)
        for (int j = 0; j < nth; ++j) {
            double pw[3];
            double th = 2.0 * ORC_PI * j / nth;
            pw[a1] = 0.5 * n[a1] + Rc * cos(th);
            pw[a2] = 0.5 * n[a2] + Rc * sin(th);
            pw[ax] = (k + 0.5) * L / nrow;
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = r[a] - pw[a];
            d[ax] -= L * floor(d[ax] / L + 0.5);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rcut2) continue;
            double sr2 = sigma * sigma / r2, sr6 = sr2 * sr2 * sr2;
            double fm = 24.0 * p->wall_eps * (2.0 * sr6 * sr6 - sr6) / r2;
            for (int a = 0; a < 3; ++a) F[a] += fm * d[a];
        }
}

/* Exposed for tests: the wall force on one bead, and the potential. */
void orc_wall_bead_force(const orc_params *p, const double r[3], double F[3]) { wall_bead_force(p, r, F); }

double orc_wall_bead_energy(const orc_params *p, const double r[3])
{
    if (!p->wall_beads) return 0.0;
    int n[3] = {p->nx, p->ny, p->nz};
    int ax = p->wall_axis, a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
    int nth, nrow;
    wall_lattice(p, &nth, &nrow);
    double Rc = p->wall_R + p->wall_rp, L = n[ax];
    double sigma = p->wall_rr + p->wall_rp;
    double rcut2 = pow(2.0, 1.0 / 3.0) * sigma * sigma;
    double U = 0.0;
    for (int k = 0; k < nrow; ++k)
        for (int j = 0; j < nth; ++j) {
            double pw[3];
            double th = 2.0 * ORC_PI * j / nth;
            pw[a1] = 0.5 * n[a1] + Rc * cos(th);
            pw[a2] = 0.5 * n[a2] + Rc * sin(th);
            pw[ax] = (k + 0.5) * L / nrow;
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = r[a] - pw[a];
            d[ax] -= L * floor(d[ax] / L + 0.5);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rcut2) continue;
            double sr2 = sigma * sigma / r2, sr6 = sr2 * sr2 * sr2;
            U += 4.0 * p->wall_eps * (sr6 * sr6 - sr6) + p->wall_eps;
        }
    return U;
}

/* ------------------------------------------------------------- public API */

int orc_init_tables(void) { init_tables(); return 0; }

void orc_lattice(int *c, double *w, int *opp)
{
    init_tables();
    for (int i = 0; i < NQ; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = CV[i][a];
        w[i] = WQ[i];
        opp[i] = OPP[i];
    }
}

void orc_mrt_tables(double *M, double *Minv, double *b)
{
    init_tables();
    for (int k = 0; k < NQ; ++k) {
        b[k] = BK[k];
        for (int i = 0; i < NQ; ++i) {
            M[k * NQ + i] = MM[k][i];
            Minv[k * NQ + i] = MINV[k][i];
        }
    }
}

void orc_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    philox4x32_10(ctr, key, out);
}

double orc_unit_uniform(uint32_t x) { return unit_uniform(x); }
double orc_unit_uniform16(uint32_t h) { return unit_uniform16(h & 0xFFFFu); }

void orc_equilibrium(double rho, const double *u, double *feq)
{
    init_tables();
    equilibrium(rho, u, feq);
}

void orc_collide_node(const orc_params *p, const double *f, const double *F,
                      uint32_t node_id, uint32_t step, double *fout)
{
    init_tables();
    collide_node(p, f, F, node_id, step, fout);
}

void orc_rotation(const double *q, double *R9)
{
    double R[3][3];
    rotation(q, R);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R9[3 * a + b] = R[a][b];
}

void orc_quat_mul(const double *a, const double *b, double *o) { quat_mul(a, b, o); }

/* Cylindrical pore (Sec. 2.3): the axis runs along `axis` through the box
 * centre; a node whose centre (integer + 1/2) lies at distance >= R from the
 * axis is a wall (boundary) node, so that along a lattice direction the first
 * wall node sits half a grid spacing outside a wall of radius R. */
void orc_pore_mask(int nx, int ny, int nz, double R, int axis, unsigned char *mask)
{
    int n[3] = {nx, ny, nz};
    int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
    double c1 = 0.5 * n[a1], c2 = 0.5 * n[a2];
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int r[3] = {x, y, z};
                double d1 = r[a1] + 0.5 - c1, d2 = r[a2] + 0.5 - c2;
                mask[(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)] =
                    (d1 * d1 + d2 * d2 >= R * R) ? 1 : 0;
            }
}

/* Populations at rest: f_i = w_i rho0 on every node. f is [19][N]. */
void orc_init(const orc_params *p, double *f)
{
    init_tables();
    size_t N = (size_t)p->nx * p->ny * p->nz;
    for (int i = 0; i < NQ; ++i)
        for (size_t n = 0; n < N; ++n) f[(size_t)i * N + n] = WQ[i] * p->rho0;
}

/* Mass and momentum of the fluid nodes: out = {sum f, sum c_x f, sum c_y f,
 * sum c_z f}. Neumaier-compensated sums over the nodes, so that the
 * conservation checks see the step's own round-off and not the reduction's. */
static void kadd(double *s, double *c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else *c += (v - t) + *s;
    *s = t;
}

void orc_moments_sum(const orc_params *p, const double *f, const unsigned char *mask, double *out)
{
    init_tables();
    size_t N = (size_t)p->nx * p->ny * p->nz;
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (size_t n = 0; n < N; ++n) {
        if (mask && mask[n]) continue;
        for (int i = 0; i < NQ; ++i) {
            double v = f[(size_t)i * N + n];
            kadd(&s[0], &c[0], v);
            for (int a = 0; a < 3; ++a)
                if (CV[i][a]) kadd(&s[a + 1], &c[a + 1], CV[i][a] * v);
        }
    }
    for (int a = 0; a < 4; ++a) out[a] = s[a] + c[a];
}

/* Node density and velocity u = (j + F/2)/rho for every node (F may be NULL). */
void orc_node_velocity(const orc_params *p, const double *f, const double *F, double *rho, double *u)
{
    init_tables();
    size_t N = (size_t)p->nx * p->ny * p->nz;
    for (size_t n = 0; n < N; ++n) {
        double r = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < NQ; ++i) {
            double v = f[(size_t)i * N + n];
            r += v;
            for (int a = 0; a < 3; ++a) j[a] += CV[i][a] * v;
        }
        rho[n] = r;
        for (int a = 0; a < 3; ++a)
            u[3 * n + a] = (j[a] + (F ? 0.5 * (p->body_force[a] + F[(size_t)a * N + n]) : 0.0)) / r;
    }
}

/*
 * One full step. f: [19][N] pre-collision populations (updated in place to
 * the next pre-collision populations). mask: N bytes, 1 = wall node (NULL =
 * none). Fnode: [3][N] bead force density spread onto the nodes by the
 * previous step (read for the bead velocity interpolation, then replaced by
 * this step's). b: bodies (NULL or nbodies == 0 for a plain fluid step).
 * step: the step index, second Philox counter word.
 *
 * Order within the step:
 *  1. bodies: first half kick with last step's force/torque, drift
 *     (velocity Verlet for the COM; quaternion rotated by the half-step
 *     body-frame angular velocity), Sec. 2.3;
 *  2. virtual sites r_b = X + R(q) s_b, v_b = V + omega x (r_b - X), Sec. 1.2;
 *  3. bead coupling, Eq. (latticeboltzmannfriction): trilinear u at r_b from
 *     the 8 surrounding nodes, F_b = -gamma (v_b - u) + f_s, -w_j F_b spread
 *     onto the same nodes, F and T summed onto the body (Sec. 2.3);
 *  4. collision of every fluid node with the force g + spread force;
 *  5. push streaming; a population streaming into a wall node returns to
 *     its origin in the opposite direction (halfway bounce-back, Sec. 1.1);
 *  6. bodies: second half kick with this step's force and torque.
 * Returns 0, or -1 on bad input.
 */
/* First half kick with the previous (sub)step's force and torque, then the
 * drift over dt: V += dt F/(2M), X += dt V, explicit Euler half kick of the
 * body-frame omega, q <- q (x) exp(omega dt / 2). */
static void bodies_kick_drift(orc_bodies *b, double dt)
{
    for (int bi = 0; bi < b->nbodies; ++bi) {
        if (b->fixed[bi] == 1) continue;
        double M = b->mass[bi];
        double *X = &b->X[3 * bi], *V = &b->V[3 * bi], *q = &b->q[4 * bi], *w = &b->w[3 * bi];
        for (int a = 0; a < 3; ++a) {
            V[a] += 0.5 * dt * b->F_last[3 * bi + a] / M;
            X[a] += dt * V[a];
        }
        if (b->fixed[bi] == 2) {           /* orientation held */
            for (int a = 0; a < 3; ++a) w[a] = 0.0;
            continue;
        }
        euler_half_kick(w, &b->inertia[3 * bi], &b->T_last[3 * bi], dt);
        double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (wn > 0.0) {
            double h = 0.5 * wn * dt;
            double dq[4] = {cos(h), sin(h) * w[0] / wn, sin(h) * w[1] / wn, sin(h) * w[2] / wn};
            quat_mul(q, dq, q);
        }
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        for (int a = 0; a < 4; ++a) q[a] /= qn;
    }
}

/* Virtual sites and friction coupling of one (sub)step: every bead's drag
 * against the fluid velocity interpolated from the populations f of this
 * LB step (with the previous step's node force Fnode), bead noise of
 * variance 2 kT gamma / dt (Philox call 4 + substep), -w dt F_b added to
 * Fnew, and the bodies' totals F_tot, T_tot. */
static void couple_bodies(const orc_params *p, const double *f, const unsigned char *mask, const double *Fnode,
                          const double g[3], double *Fnew, orc_bodies *b, uint32_t step32, int substep, double dt)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const size_t N = (size_t)nx * ny * nz;
    for (int bi = 0; bi < b->nbodies; ++bi) {
        double R[3][3];
        rotation(&b->q[4 * bi], R);
        const double *X = &b->X[3 * bi], *V = &b->V[3 * bi], *wb = &b->w[3 * bi];
        double wl[3];
        for (int a = 0; a < 3; ++a) wl[a] = R[a][0] * wb[0] + R[a][1] * wb[1] + R[a][2] * wb[2];
        double Ft[3] = {0, 0, 0}, Tt[3] = {0, 0, 0};
        for (int k = b->bead_start[bi]; k < b->bead_start[bi + 1]; ++k) {
            const double *s = &b->s[3 * k];
            double rel[3], r[3], v[3], wxr[3];
            for (int a = 0; a < 3; ++a) rel[a] = R[a][0] * s[0] + R[a][1] * s[1] + R[a][2] * s[2];
            for (int a = 0; a < 3; ++a) r[a] = X[a] + rel[a];
            cross(wl, rel, wxr);
            for (int a = 0; a < 3; ++a) v[a] = V[a] + wxr[a];

            /* the 8 nodes around r; node centres at integer + 1/2 */
            int base[3];
            double frac[3];
            for (int a = 0; a < 3; ++a) {
                double t = r[a] - 0.5;
                double fl = floor(t);
                base[a] = (int)fl;
                frac[a] = t - fl;
            }
            double ub[3] = {0, 0, 0};
            size_t node[8];
            double wgt[8];
            int fluid[8];
            for (int cidx = 0; cidx < 8; ++cidx) {
                int o[3] = {cidx & 1, (cidx >> 1) & 1, (cidx >> 2) & 1};
                double wt = 1.0;
                for (int a = 0; a < 3; ++a) wt *= o[a] ? frac[a] : 1.0 - frac[a];
                int yraw = base[1] + o[1];
                wgt[cidx] = wt;
                if (p->ywalls && (yraw < 0 || yraw >= ny)) {
                    /* a node beyond a moving wall carries the wall's velocity */
                    const double *uw = yraw < 0 ? p->uw_lo : p->uw_hi;
                    for (int a = 0; a < 3; ++a) ub[a] += wt * uw[a];
                    fluid[cidx] = 0;
                    node[cidx] = 0;
                    continue;
                }
                int xx = wrap(base[0] + o[0], nx), yy = wrap(yraw, ny), zz = wrap(base[2] + o[2], nz);
                size_t n = nidx(p, xx, yy, zz);
                node[cidx] = n;
                fluid[cidx] = !(mask && mask[n]);
                if (!fluid[cidx]) continue; /* wall nodes carry u = 0 */
                double rho = 0.0, j[3] = {0, 0, 0};
                for (int i = 0; i < NQ; ++i) {
                    double fv = f[(size_t)i * N + n];
                    rho += fv;
                    for (int a = 0; a < 3; ++a) j[a] += CV[i][a] * fv;
                }
                for (int a = 0; a < 3; ++a)
                    ub[a] += wt * (j[a] + 0.5 * (g[a] + Fnode[(size_t)a * N + n])) / rho;
            }
            double Fb[3];
            double fs[3] = {0, 0, 0};
            if (p->kT > 0.0 && p->gamma_bead > 0.0) {
                uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
                uint32_t ctr[4] = {(uint32_t)k, step32, p->instance, 4u + (uint32_t)substep};
                uint32_t rr[4];
                philox4x32_10(ctr, key, rr);
                double amp = sqrt(2.0 * p->kT * p->gamma_bead / dt);
                for (int a = 0; a < 3; ++a) fs[a] = amp * unit_uniform(rr[a]);
            }
            for (int a = 0; a < 3; ++a) Fb[a] = -p->gamma_bead * (v[a] - ub[a]) + fs[a];
            for (int cidx = 0; cidx < 8; ++cidx) {
                if (!fluid[cidx]) continue; /* momentum into a wall node is taken by the wall */
                for (int a = 0; a < 3; ++a) Fnew[(size_t)a * N + node[cidx]] -= dt * wgt[cidx] * Fb[a];
            }
            double tq[3];
            cross(rel, Fb, tq);
            for (int a = 0; a < 3; ++a) {
                b->F_bead[3 * k + a] = Fb[a];
                Ft[a] += Fb[a];
                Tt[a] += tq[a];
            }
            /* pore-wall beads act on the bead, not on the fluid */
            double Fw[3];
            wall_bead_force(p, r, Fw);
            cross(rel, Fw, tq);
            for (int a = 0; a < 3; ++a) {
                Ft[a] += Fw[a];
                Tt[a] += tq[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            b->F_tot[3 * bi + a] = Ft[a] + b->F_ext[3 * bi + a];
            b->T_tot[3 * bi + a] = Tt[a] + b->T_ext[3 * bi + a];
        }
    }
}

/* Second half kick over dt with this (sub)step's totals, which become the
 * next first half kick's force and (body-frame) torque. */
static void bodies_kick2(orc_bodies *b, double dt)
{
    for (int bi = 0; bi < b->nbodies; ++bi) {
        double R[3][3];
        rotation(&b->q[4 * bi], R);
        double Tb[3];
        const double *Tl = &b->T_tot[3 * bi];
        for (int a = 0; a < 3; ++a) Tb[a] = R[0][a] * Tl[0] + R[1][a] * Tl[1] + R[2][a] * Tl[2];
        for (int a = 0; a < 3; ++a) {
            b->F_last[3 * bi + a] = b->F_tot[3 * bi + a];
            b->T_last[3 * bi + a] = Tb[a];
        }
        if (b->fixed[bi] == 1) continue;
        for (int a = 0; a < 3; ++a) b->V[3 * bi + a] += 0.5 * dt * b->F_tot[3 * bi + a] / b->mass[bi];
        if (b->fixed[bi] == 2) continue;
        euler_half_kick_implicit(&b->w[3 * bi], &b->inertia[3 * bi], Tb, dt);
    }
}

int orc_step(const orc_params *p, double *f, const unsigned char *mask, double *Fnode,
             orc_bodies *b, int64_t step)
{
    init_tables();
    if (p->collision == 0 && p->kT > 0.0) return -1;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const size_t N = (size_t)nx * ny * nz;
    const uint32_t step32 = (uint32_t)step;
    const int nbodies = b ? b->nbodies : 0;
    const int nsub = p->md_substeps > 1 ? p->md_substeps : 1;
    const double dt = 1.0 / nsub;

    size_t nfluid = 0;
    for (size_t n = 0; n < N; ++n) nfluid += (mask && mask[n]) ? 0 : 1;

    /* uniform force density on the fluid */
    double g[3];
    for (int a = 0; a < 3; ++a) g[a] = p->body_force[a];
    if (p->compensate_force && nfluid > 0)
        for (int bi = 0; bi < nbodies; ++bi)
            if (b->fixed[bi] != 1)
                for (int a = 0; a < 3; ++a) g[a] -= b->F_ext[3 * bi + a] / (double)nfluid;

    double *Fnew = (double *)calloc(3 * N, sizeof(double));
    double *fpost = (double *)malloc(sizeof(double) * NQ * N);
    if (!Fnew || !fpost) { free(Fnew); free(fpost); return -1; }

    /* 1.-3. the MD substeps: first half kick and drift, virtual sites and
       coupling, and (between substeps) the second half kick */
    if (nbodies > 0)
        for (int sub = 0; sub < nsub; ++sub) {
            bodies_kick_drift(b, dt);
            couple_bodies(p, f, mask, Fnode, g, Fnew, b, step32, sub, dt);
            if (sub + 1 < nsub) bodies_kick2(b, dt);
        }

    /* 4. collision */
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t n = nidx(p, x, y, z);
                if (mask && mask[n]) {
                    for (int i = 0; i < NQ; ++i) fpost[(size_t)i * N + n] = f[(size_t)i * N + n];
                    continue;
                }
                double fl[NQ], fo[NQ], F[3];
                for (int i = 0; i < NQ; ++i) fl[i] = f[(size_t)i * N + n];
                for (int a = 0; a < 3; ++a) F[a] = g[a] + Fnew[(size_t)a * N + n];
                collide_node(p, fl, F, (uint32_t)n, step32, fo);
                for (int i = 0; i < NQ; ++i) fpost[(size_t)i * N + n] = fo[i];
            }

    /* 5. push streaming with halfway bounce-back; wall nodes keep their values */
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t n = nidx(p, x, y, z);
                if (mask && mask[n]) continue;
                for (int i = 0; i < NQ; ++i) {
                    int ty = y + CV[i][1];
                    if (p->ywalls && (ty < 0 || ty >= ny)) {
                        /* halfway bounce-back on a moving wall: the population
                           returns reversed and takes the wall's momentum,
                           f_opp(i) = f*_i - 6 w_i rho0 (c_i . u_wall) */
                        const double *uw = ty < 0 ? p->uw_lo : p->uw_hi;
                        double cu = CV[i][0] * uw[0] + CV[i][1] * uw[1] + CV[i][2] * uw[2];
                        f[(size_t)OPP[i] * N + n] = fpost[(size_t)i * N + n] - 6.0 * WQ[i] * p->rho0 * cu;
                        continue;
                    }
                    size_t to = nidx(p, wrap(x + CV[i][0], nx), wrap(ty, ny), wrap(z + CV[i][2], nz));
                    if (mask && mask[to])
                        f[(size_t)OPP[i] * N + n] = fpost[(size_t)i * N + n];
                    else
                        f[(size_t)i * N + to] = fpost[(size_t)i * N + n];
                }
            }

    /* 6. second half kick of the last substep */
    if (nbodies > 0) bodies_kick2(b, dt);

    memcpy(Fnode, Fnew, sizeof(double) * 3 * N);
    free(Fnew);
    free(fpost);
    return 0;
}

/* ------------------------------------------------------------------ adjoint */

/* Reverse of one node's collision: given lam_out = dJ/df* (19), returns
 * dJ/df (19) and dJ/dF (3) of f* = collide(f, F) for the deterministic
 * collision (kT = 0), by the chain rule through rho, j, u = (j + F/2)/rho,
 * f_eq(rho, u) and the Guo source s(u, F) in population space. */
static void collide_node_adjoint(const orc_params *p, const double f[NQ], const double F[3],
                                 const double lam_out[NQ], double lam_f[NQ], double lam_F[3])
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NQ; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += CV[i][a] * f[i];
    }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
    double lam_feq[NQ], lam_s[NQ];
    for (int i = 0; i < NQ; ++i) lam_f[i] = 0.0;
    if (p->collision == 0) {
        const double om = 1.0 / p->tau;
        for (int i = 0; i < NQ; ++i) {
            lam_f[i] = (1.0 - om) * lam_out[i];
            lam_feq[i] = om * lam_out[i];
            lam_s[i] = (1.0 - 0.5 * om) * lam_out[i];
        }
    } else {
        double lam_ms[NQ];
        for (int k = 0; k < NQ; ++k) {
            lam_ms[k] = 0.0;
            for (int i = 0; i < NQ; ++i) lam_ms[k] += MINV[i][k] * lam_out[i];
        }
        for (int i = 0; i < NQ; ++i) {
            lam_feq[i] = lam_s[i] = 0.0;
            for (int k = 0; k < NQ; ++k) {
                double g = mode_rate(p, k);
                lam_f[i] += MM[k][i] * g * lam_ms[k];
                lam_feq[i] += MM[k][i] * (1.0 - g) * lam_ms[k];
                lam_s[i] += MM[k][i] * 0.5 * (1.0 + g) * lam_ms[k];
            }
        }
    }
    /* through f_eq(rho, u) and s(u, F) */
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double lam_rho = 0.0, lam_u[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) lam_F[a] = 0.0;
    for (int i = 0; i < NQ; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        double cF = CV[i][0] * F[0] + CV[i][1] * F[1] + CV[i][2] * F[2];
        lam_rho += lam_feq[i] * WQ[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        for (int a = 0; a < 3; ++a) {
            lam_u[a] += lam_feq[i] * WQ[i] * rho * (3.0 * CV[i][a] + 9.0 * cu * CV[i][a] - 3.0 * u[a]);
            lam_u[a] += lam_s[i] * WQ[i] * (-3.0 * F[a] + 9.0 * CV[i][a] * cF);
            lam_F[a] += lam_s[i] * WQ[i] * (3.0 * (CV[i][a] - u[a]) + 9.0 * cu * CV[i][a]);
        }
    }
    /* u = (j + F/2) / rho */
    double lam_j[3];
    for (int a = 0; a < 3; ++a) {
        lam_j[a] = lam_u[a] / rho;
        lam_F[a] += 0.5 * lam_u[a] / rho;
        lam_rho -= lam_u[a] * u[a] / rho;
    }
    for (int i = 0; i < NQ; ++i)
        lam_f[i] += lam_rho + CV[i][0] * lam_j[0] + CV[i][1] * lam_j[1] + CV[i][2] * lam_j[2];
}

void orc_collide_node_adjoint(const orc_params *p, const double *f, const double *F, const double *lam_out,
                              double *lam_f, double *lam_F)
{
    init_tables();
    collide_node_adjoint(p, f, F, lam_out, lam_f, lam_F);
}

/* Gradient of J = (1/W) sum over the last W steps of V_axis of body jb
 * (its velocity after each step) with respect to the bead friction gamma and
 * to every body-frame bead offset, by reverse-mode differentiation of
 * orc_step over nsteps steps starting from the given state (which the call
 * advances, exactly as orc_step would). Deterministic steps only (kT = 0);
 * every body must be fixed (1) or translation-only (2). All intermediate
 * states are stored (small cases only). Returns 0, -1 (memory), -2 (bad
 * input). dJ_ds: 3 per bead of all bodies (may be NULL). */
int orc_adjoint_drag(const orc_params *p, double *f, const unsigned char *mask, double *Fnode,
                     orc_bodies *b, int64_t step0, int nsteps, int window, int jb, int axis,
                     double *J, double *dJ_dgamma, double *dJ_ds)
{
    init_tables();
    if (p->kT > 0.0 || nsteps < 1 || window < 1 || window > nsteps || !b || jb < 0 || jb >= b->nbodies ||
        axis < 0 || axis > 2 || p->ywalls || p->wall_beads || p->md_substeps > 1)
        return -2;      /* the reverse pass covers pores and periodic boxes, without walls or wall beads */
    if (b->nbodies > 64) return -2;
    for (int bi = 0; bi < b->nbodies; ++bi)
        if (b->fixed[bi] != 1 && b->fixed[bi] != 2) return -2;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const size_t N = (size_t)nx * ny * nz;
    const int nb = b->nbodies, nbeads = b->bead_start[nb];
    double *fs = (double *)malloc(sizeof(double) * NQ * N * (size_t)nsteps);
    double *Fs = (double *)malloc(sizeof(double) * 3 * N * (size_t)nsteps);
    double *Bs = (double *)malloc(sizeof(double) * 9 * nb * (size_t)nsteps); /* X, V, F_last */
    double *lf = (double *)calloc(NQ * N, sizeof(double)), *lf2 = (double *)calloc(NQ * N, sizeof(double));
    double *lFp = (double *)calloc(3 * N, sizeof(double)), *lFp2 = (double *)calloc(3 * N, sizeof(double));
    double *lFn = (double *)calloc(3 * N, sizeof(double));
    double *Fnew = (double *)calloc(3 * N, sizeof(double));
    double *lb_ = (double *)calloc(9 * nb, sizeof(double));   /* lam X, V, F_last per body */
    double *Fb = (double *)malloc(sizeof(double) * 3 * (nbeads > 0 ? nbeads : 1));
    if (!fs || !Fs || !Bs || !lf || !lf2 || !lFp || !lFp2 || !lFn || !Fnew || !lb_ || !Fb) {
        free(fs); free(Fs); free(Bs); free(lf); free(lf2); free(lFp); free(lFp2); free(lFn); free(Fnew); free(lb_); free(Fb);
        return -1;
    }
    /* forward, storing the state before every step */
    double Jsum = 0.0;
    for (int n = 0; n < nsteps; ++n) {
        memcpy(fs + (size_t)n * NQ * N, f, sizeof(double) * NQ * N);
        memcpy(Fs + (size_t)n * 3 * N, Fnode, sizeof(double) * 3 * N);
        for (int bi = 0; bi < nb; ++bi)
            for (int a = 0; a < 3; ++a) {
                Bs[((size_t)n * nb + bi) * 9 + a] = b->X[3 * bi + a];
                Bs[((size_t)n * nb + bi) * 9 + 3 + a] = b->V[3 * bi + a];
                Bs[((size_t)n * nb + bi) * 9 + 6 + a] = b->F_last[3 * bi + a];
            }
        orc_step(p, f, mask, Fnode, b, step0 + n);
        if (n >= nsteps - window) Jsum += b->V[3 * jb + axis];
    }
    *J = Jsum / window;

    /* uniform force density as orc_step forms it */
    size_t nfluid = 0;
    for (size_t n = 0; n < N; ++n) nfluid += (mask && mask[n]) ? 0 : 1;
    double g[3];
    for (int a = 0; a < 3; ++a) g[a] = p->body_force[a];
    if (p->compensate_force && nfluid > 0)
        for (int bi = 0; bi < nb; ++bi)
            if (b->fixed[bi] != 1)
                for (int a = 0; a < 3; ++a) g[a] -= b->F_ext[3 * bi + a] / (double)nfluid;

    double lgam = 0.0;
    if (dJ_ds) memset(dJ_ds, 0, sizeof(double) * 3 * nbeads);
    for (int n = nsteps - 1; n >= 0; --n) {
        const double *fn = fs + (size_t)n * NQ * N;
        const double *Fp = Fs + (size_t)n * 3 * N;
        if (n >= nsteps - window) lb_[9 * jb + 3 + axis] += 1.0 / window;

        /* recompute the step's coupling quantities */
        double Ftot[64][3];
        double Xp[64][3], Vp[64][3], Rm[64][3][3], wl[64][3];
        memset(Fnew, 0, sizeof(double) * 3 * N);
        for (int bi = 0; bi < nb; ++bi) {
            const double *Bn = Bs + ((size_t)n * nb + bi) * 9;
            for (int a = 0; a < 3; ++a) {
                if (b->fixed[bi] == 2) {
                    Vp[bi][a] = Bn[3 + a] + 0.5 * Bn[6 + a] / b->mass[bi];
                    Xp[bi][a] = Bn[a] + Vp[bi][a];
                } else {
                    Vp[bi][a] = Bn[3 + a];
                    Xp[bi][a] = Bn[a];
                }
                Ftot[bi][a] = b->F_ext[3 * bi + a];
            }
            rotation(&b->q[4 * bi], Rm[bi]);
            const double *wb = &b->w[3 * bi];
            for (int a = 0; a < 3; ++a) wl[bi][a] = Rm[bi][a][0] * wb[0] + Rm[bi][a][1] * wb[1] + Rm[bi][a][2] * wb[2];
        }
        for (int bi = 0; bi < nb; ++bi)
            for (int k = b->bead_start[bi]; k < b->bead_start[bi + 1]; ++k) {
                const double *s = &b->s[3 * k];
                double rel[3], r[3], v[3], wxr[3];
                for (int a = 0; a < 3; ++a) rel[a] = Rm[bi][a][0] * s[0] + Rm[bi][a][1] * s[1] + Rm[bi][a][2] * s[2];
                for (int a = 0; a < 3; ++a) r[a] = Xp[bi][a] + rel[a];
                cross(wl[bi], rel, wxr);
                for (int a = 0; a < 3; ++a) v[a] = Vp[bi][a] + wxr[a];
                int base[3];
                double fr[3];
                for (int a = 0; a < 3; ++a) {
                    double t = r[a] - 0.5, fl = floor(t);
                    base[a] = (int)fl;
                    fr[a] = t - fl;
                }
                double ub[3] = {0, 0, 0};
                for (int c = 0; c < 8; ++c) {
                    int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                    double wt = 1.0;
                    for (int a = 0; a < 3; ++a) wt *= o[a] ? fr[a] : 1.0 - fr[a];
                    size_t nn = nidx(p, wrap(base[0] + o[0], nx), wrap(base[1] + o[1], ny), wrap(base[2] + o[2], nz));
                    if (mask && mask[nn]) continue;
                    double rho = 0.0, jj[3] = {0, 0, 0};
                    for (int i = 0; i < NQ; ++i) {
                        double fv = fn[(size_t)i * N + nn];
                        rho += fv;
                        for (int a = 0; a < 3; ++a) jj[a] += CV[i][a] * fv;
                    }
                    for (int a = 0; a < 3; ++a) ub[a] += wt * (jj[a] + 0.5 * (g[a] + Fp[(size_t)a * N + nn])) / rho;
                }
                for (int a = 0; a < 3; ++a) {
                    Fb[3 * k + a] = -p->gamma_bead * (v[a] - ub[a]);
                    Ftot[bi][a] += Fb[3 * k + a];
                }
                for (int c = 0; c < 8; ++c) {
                    int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                    double wt = 1.0;
                    for (int a = 0; a < 3; ++a) wt *= o[a] ? fr[a] : 1.0 - fr[a];
                    size_t nn = nidx(p, wrap(base[0] + o[0], nx), wrap(base[1] + o[1], ny), wrap(base[2] + o[2], nz));
                    if (mask && mask[nn]) continue;
                    for (int a = 0; a < 3; ++a) Fnew[(size_t)a * N + nn] -= wt * Fb[3 * k + a];
                }
            }

        /* kick2 reversed: V_{n+1} = V' + F_tot/(2M) (translation-only bodies), F_last_{n+1} = F_tot */
        double lVp[64][3], lXp[64][3], lFt[64][3];
        for (int bi = 0; bi < nb; ++bi)
            for (int a = 0; a < 3; ++a) {
                lXp[bi][a] = lb_[9 * bi + a];
                lFt[bi][a] = lb_[9 * bi + 6 + a];
                lVp[bi][a] = 0.0;
                if (b->fixed[bi] == 2) {
                    lVp[bi][a] = lb_[9 * bi + 3 + a];
                    lFt[bi][a] += lb_[9 * bi + 3 + a] / (2.0 * b->mass[bi]);
                }
            }
        /* F_prev_{n+1} = F_new */
        for (size_t q = 0; q < 3 * N; ++q) lFn[q] = lFp[q];
        /* streaming reversed: adjoint of the post-collision population */
        memset(lf2, 0, sizeof(double) * NQ * N);
        memset(lFp2, 0, sizeof(double) * 3 * N);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    size_t nn = nidx(p, x, y, z);
                    if (mask && mask[nn]) continue;
                    double lpost[NQ], fl[NQ], F[3], lfn[NQ], lF[3];
                    for (int i = 0; i < NQ; ++i) {
                        size_t to = nidx(p, wrap(x + CV[i][0], nx), wrap(y + CV[i][1], ny), wrap(z + CV[i][2], nz));
                        lpost[i] = (mask && mask[to]) ? lf[(size_t)OPP[i] * N + nn] : lf[(size_t)i * N + to];
                        fl[i] = fn[(size_t)i * N + nn];
                    }
                    for (int a = 0; a < 3; ++a) F[a] = g[a] + Fnew[(size_t)a * N + nn];
                    collide_node_adjoint(p, fl, F, lpost, lfn, lF);
                    for (int i = 0; i < NQ; ++i) lf2[(size_t)i * N + nn] = lfn[i];
                    for (int a = 0; a < 3; ++a) lFn[(size_t)a * N + nn] += lF[a];
                }
        /* coupling reversed */
        for (int bi = 0; bi < nb; ++bi)
            for (int k = b->bead_start[bi]; k < b->bead_start[bi + 1]; ++k) {
                const double *s = &b->s[3 * k];
                double rel[3], r[3], v[3], wxr[3];
                for (int a = 0; a < 3; ++a) rel[a] = Rm[bi][a][0] * s[0] + Rm[bi][a][1] * s[1] + Rm[bi][a][2] * s[2];
                for (int a = 0; a < 3; ++a) r[a] = Xp[bi][a] + rel[a];
                cross(wl[bi], rel, wxr);
                for (int a = 0; a < 3; ++a) v[a] = Vp[bi][a] + wxr[a];
                int base[3];
                double fr[3];
                for (int a = 0; a < 3; ++a) {
                    double t = r[a] - 0.5, fl = floor(t);
                    base[a] = (int)fl;
                    fr[a] = t - fl;
                }
                double uj[8][3], rhoj[8], wts[8];
                size_t nns[8];
                int fl8[8];
                double ub[3] = {0, 0, 0};
                for (int c = 0; c < 8; ++c) {
                    int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                    double wt = 1.0;
                    for (int a = 0; a < 3; ++a) wt *= o[a] ? fr[a] : 1.0 - fr[a];
                    size_t nn = nidx(p, wrap(base[0] + o[0], nx), wrap(base[1] + o[1], ny), wrap(base[2] + o[2], nz));
                    wts[c] = wt;
                    nns[c] = nn;
                    fl8[c] = !(mask && mask[nn]);
                    rhoj[c] = 1.0;
                    for (int a = 0; a < 3; ++a) uj[c][a] = 0.0;
                    if (!fl8[c]) continue;
                    double rho = 0.0, jj[3] = {0, 0, 0};
                    for (int i = 0; i < NQ; ++i) {
                        double fv = fn[(size_t)i * N + nn];
                        rho += fv;
                        for (int a = 0; a < 3; ++a) jj[a] += CV[i][a] * fv;
                    }
                    rhoj[c] = rho;
                    for (int a = 0; a < 3; ++a) {
                        uj[c][a] = (jj[a] + 0.5 * (g[a] + Fp[(size_t)a * N + nn])) / rho;
                        ub[a] += wt * uj[c][a];
                    }
                }
                /* lam F_b: from the body total and from the spread */
                double lFbk[3], lw[8];
                for (int a = 0; a < 3; ++a) lFbk[a] = lFt[bi][a];
                for (int c = 0; c < 8; ++c) {
                    lw[c] = 0.0;
                    if (!fl8[c]) continue;
                    for (int a = 0; a < 3; ++a) {
                        lFbk[a] -= wts[c] * lFn[(size_t)a * N + nns[c]];
                        lw[c] -= Fb[3 * k + a] * lFn[(size_t)a * N + nns[c]];
                    }
                }
                /* F_b = -gamma (v - u_b) */
                double lv[3], lub[3];
                for (int a = 0; a < 3; ++a) {
                    lgam += -(v[a] - ub[a]) * lFbk[a];
                    lv[a] = -p->gamma_bead * lFbk[a];
                    lub[a] = p->gamma_bead * lFbk[a];
                }
                /* u_b = sum_c w_c u_c; u_c = (j_c + (g + Fprev_c)/2) / rho_c */
                for (int c = 0; c < 8; ++c) {
                    if (!fl8[c]) continue;
                    double luj[3], lrho = 0.0, lj[3];
                    for (int a = 0; a < 3; ++a) {
                        lw[c] += uj[c][a] * lub[a];
                        luj[a] = wts[c] * lub[a];
                        lj[a] = luj[a] / rhoj[c];
                        lrho -= luj[a] * uj[c][a] / rhoj[c];
                        lFp2[(size_t)a * N + nns[c]] += 0.5 * luj[a] / rhoj[c];
                    }
                    for (int i = 0; i < NQ; ++i)
                        lf2[(size_t)i * N + nns[c]] += lrho + CV[i][0] * lj[0] + CV[i][1] * lj[1] + CV[i][2] * lj[2];
                }
                /* weights w_c = prod_a (o_a ? fr_a : 1 - fr_a), d fr_a / d r_a = 1 */
                double lr[3] = {0, 0, 0};
                for (int c = 0; c < 8; ++c) {
                    int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
                    for (int a = 0; a < 3; ++a) {
                        double d = o[a] ? 1.0 : -1.0;
                        for (int a2 = 0; a2 < 3; ++a2)
                            if (a2 != a) d *= o[a2] ? fr[a2] : 1.0 - fr[a2];
                        lr[a] += lw[c] * d;
                    }
                }
                /* r = X' + R s, v = V' + w x (R s) */
                double lrel[3], lxw[3];
                cross(lv, wl[bi], lxw);   /* (lam_v x w) is the adjoint of w x rel */
                for (int a = 0; a < 3; ++a) {
                    lXp[bi][a] += lr[a];
                    lVp[bi][a] += lv[a];
                    lrel[a] = lr[a] + lxw[a];
                }
                if (dJ_ds)
                    for (int a = 0; a < 3; ++a)
                        dJ_ds[3 * k + a] += Rm[bi][0][a] * lrel[0] + Rm[bi][1][a] * lrel[1] + Rm[bi][2][a] * lrel[2];
            }
        /* kick-drift reversed: V' = V + F_last/(2M), X' = X + V' (translation-only bodies) */
        for (int bi = 0; bi < nb; ++bi)
            for (int a = 0; a < 3; ++a) {
                if (b->fixed[bi] == 2) {
                    double lvt = lVp[bi][a] + lXp[bi][a];
                    lb_[9 * bi + a] = lXp[bi][a];
                    lb_[9 * bi + 3 + a] = lvt;
                    lb_[9 * bi + 6 + a] = lvt / (2.0 * b->mass[bi]);
                } else {
                    lb_[9 * bi + a] = lb_[9 * bi + 3 + a] = lb_[9 * bi + 6 + a] = 0.0;
                }
            }
        double *t = lf; lf = lf2; lf2 = t;
        t = lFp; lFp = lFp2; lFp2 = t;
    }
    *dJ_dgamma = lgam;
    free(fs); free(Fs); free(Bs); free(lf); free(lf2); free(lFp); free(lFp2); free(lFn); free(Fnew); free(lb_); free(Fb);
    return 0;
}
