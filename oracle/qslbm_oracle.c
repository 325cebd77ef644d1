/*
 * qslbm oracle: a plain, slow FP64 CPU restatement of the single-step simplified
 * lattice Boltzmann method for quasi-static MHD pipe flow (Tavares, Magacho,
 * Moriconi, Loureiro, arXiv 2211.09370).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only through seeded parameters.
 *
 * Every function follows the paper's equations in the paper's order, one node at
 * a time, with no blocking, fusion or algebraic rearrangement beyond what the
 * equations themselves state.  Arithmetic is IEEE binary64, round to nearest,
 * built with -ffp-contract=off.  OpenMP splits only loops whose iterations are
 * independent (one output node per iteration), so results do not depend on the
 * thread count.  Reductions run sequentially.
 *
 * Equations (section and equation of the paper):
 *   Sec. III.A  Eq. "Equilibrium distribution simple fluids"      f_i^eq
 *   Sec. III.E  Eq. "single-step algorithm complete"               rho update
 *   Sec. V.A    Eq. "FGS forcing term algorithm"                   F_i (GZS)
 *   Sec. V.A    Eq. "Single-step algorithm with lattice discrete effect"
 *   Sec. V.A    Lorentz force J x B with isotropic finite differences
 *   Sec. V.B    Eq. "Kernel functions for Lagrange interpolation I"
 *   Sec. V.C    explicit IB: d_i = sum_j A_ij, A = D D^T
 *   Sec. V.D    explicit IB for the magnetic field
 *   Sec. V.E    Eq. "IBM correted for velocity field"  (lambda scaling)
 *   Sec. V.F    Eq. "IB corrected for magnetic field"  (lambda_mag scaling)
 *   Sec. V.G    Eq. "Single step algoritm for magnetic field" (tau_m = 1 sweep),
 *               c = 6 eta (c_s^2 = c^2/3), N_mag = ceil(1/dt)
 *   Sec. IV     Eq. "Energy balance equations", Eq. "variable force"
 *   Sec. V.H    Eq. "Error l2 decay" (QS residual)
 *   Sec. III.D  Eq. "single-step algorithm for MHD de rosis": the magnetic
 *               update for any tau_m (mag_scheme = 1: one update per flow step,
 *               the induction equation advanced in time, not quasi-static)
 *   Sec. VII    rescaled time step dt/gamma (Eq. "adaptative time step delta t",
 *               "adaptative time step lattice velocities", "rescaled relaxation
 *               time"): second-order f^eq terms and the g^eq flux over gamma,
 *               tau = nu/(gamma c_s^2) + 1/2, the GZS terms with gamma
 *   Sec. V.H    "Strategies for very high values of resistivity": the sweep
 *               with the extra coefficient alpha (Eq. "magnetic field
 *               quasi-static acelerated"); alpha = 1 is the plain sweep
 *   Sec. III.A  Table I: the D3Q27 flow lattice (flow_q = 27)
 *   Sec. V.G    Eqs. "densities MAC", "momentum Mac": the macroscopic flow
 *               scheme for tau >= 1 (flow_scheme = 1, R18)
 *
 * Readings where the paper is silent or garbled:
 *   R1 f^eq(x - c_i) in the density update carries the index i.
 *   R2 In the velocity update with the discrete-effect correction every term is
 *      a momentum and the sum is divided by rho(t+1) once.
 *   R3 The field lattice is D2Q5 (w0 = 1/3, w = 1/6, c_m^2 = 1/3) or D3Q7
 *      (w0 = 1/4, w = 1/8, c_m^2 = 1/4); c = 2 eta / c_m^2, which is the paper's
 *      c = 6 eta when c_m^2 = 1/3.  N_mag = ceil(c), capped.
 *   R4 The sweep evolves the induced field b (B = B^ext + b); the flux uses the
 *      full B.  B^ext is held by outside sources and is not relaxed.  The curl of
 *      B^ext is not part of J.
 *   R5 IB on b after every sweep; IB on u once per flow step.  Wall values are
 *      zero (no slip, insulating).  All markers interpolate the same predictor
 *      field before any spreads.
 *   R6 Kernel pieces are taken on half-open intervals (-3/2,-1/2], (-1/2,1/2],
 *      (1/2,3/2], zero elsewhere, so exactly three nodes per axis carry weight.
 *   R7 lambda = nu/nu_ref, lambda_m = eta/eta_ref.  eta_ref = c_m^2/2 (the
 *      sweep's own relaxation time one, so lambda_m = c >= 1) unless given.
 *      nu_ref = nu (lambda = 1, which turns the Sec. V.E scaling into the plain
 *      explicit corrector of Sec. V.C) unless given: with nu_ref = c_s^2/2 the
 *      scaling has a pole at d = 1/(1 - lambda) that the pipes' marker rings
 *      cross (d up to 1.35) and the flow diverges.
 *   R8 Parameter mapping with L = pipe radius (channel half width):
 *      nu = U0 R/Re, eta = U0 R/Rm, B0 = Ha sqrt(eta nu)/R, F0 = 4 nu U0/R^2
 *      (pipe) or 2 nu U0/R^2 (channel); automatic U0 = min(0.05, Re c_s^2/(2R),
 *      Re R/(2 Ha^2)).
 *   R13 Accelerated sweep: the printed rest equilibrium "(1 - w_1) B + alpha B"
 *      would not keep a uniform field fixed under B <- (1/alpha) sum_i g_i.  It
 *      is read as (w_1 - 1 + alpha) b (w_1 the rest weight), which keeps it
 *      fixed and gives the plain sweep at alpha = 1; the moving equilibria are
 *      unchanged.  Per node this is b + (sweep(b) - b)/alpha.
 *   R14 Time-resolved magnetic update (mag_scheme = 1): the field lattice runs
 *      at the flow's speed (c = 1, dx = dt = 1), so eta = c_m^2 (tau_m - 1/2),
 *      tau_m = eta/c_m^2 + 1/2, the flux coefficient is e_beta / c_m^2, and the
 *      update runs once per flow step, followed by the IB on b, with
 *      eta_ref = eta (lambda_m = 1) unless given, as for nu_ref in R7.
 *   R15 Rescaled time step (gamma): a step advances physical time by 1/gamma.
 *      Per step the forces (body and Lorentz, physical rates) add F/gamma to
 *      rho u, the body-force modulation runs on t/gamma, and the magnetic
 *      algorithm uses the per-step resistivity eta/gamma (sweeps: c = 2 eta /
 *      (gamma c_m^2); time-resolved: tau_m = eta/(gamma c_m^2) + 1/2) with the
 *      flux over gamma, so that the quasi-static fixed point does not depend
 *      on gamma.  lambda and lambda_m use nu/gamma and eta/gamma.
 *   R17 3-D flow lattice: D3Q19 unless flow_q = 27, which selects the paper's own
 *      D3Q27 (Sec. III.A, Table I: rest 8/27, six axis 2/27, twelve edge 1/54,
 *      eight corner 1/216; c_s^2 = 1/3).  Every sum over the flow lattice (the
 *      equilibria of the density and momentum updates, the GZS terms and their
 *      correction, the isotropic differences of the Lorentz force, the
 *      diagnostics' Laplacian) runs over the chosen lattice.
 *   R18 Macroscopic flow scheme for tau >= 1 (flow_scheme = 1; Sec. V.G
 *      "Stability improvements for high values of viscosity and resistivity",
 *      Eqs. "densities MAC", "momentum Mac"): tau = 1 at particle speed
 *      c = 6 nu (dx = 1, dt = 1/c).  In the rescaled-time-step form of R15 this
 *      is gamma = 6 nu, which makes tau = nu/(gamma c_s^2) + 1/2 = 1; rho is
 *      sum_i f_i^eq(x - c_i) and rho u is sum_i c_i f_i^eq(x - c_i), the
 *      single-step momentum update at tau = 1.  The paper gives no forcing for
 *      this scheme: the single-step GZS terms and correction at tau = 1 are
 *      used, with the force per step over gamma as in R15, and the magnetic
 *      algorithm runs with the same time step.  It needs 6 nu >= 1 (tau >= 1
 *      in the single-step scheme at gamma = 1), and the automatic U0 then
 *      drops its tau <= 1 bound.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CHANNEL 0
#define ORC_PIPE 1
#define ORC_NONE 2 /* periodic box without walls: used to pin the sweep */

#define ORC_B0_UNIFORM 0
#define ORC_B0_TANH 1
#define ORC_B0_FIELD 2 /* B0 times a caller-given in-plane field [3][ny][nx] */

/* Node loops of smaller domains run on one thread: the fork and join of a
 * parallel region would cost more than the loop (results are the same either
 * way, since every iteration writes its own node). */
#define ORC_OMP_MIN_NODES 512

typedef struct orc_params {
    int dim, nx, ny, nz, geometry;
    double diameter, cx, cy, marker_spacing;
    double Re, Ha, Rm, U0;
    int b0_kind;
    double b0_dir[3], ramp_center, ramp_width;
    double force_amp, force_period;
    int n_mag, n_mag_cap;
    double nu_ref, eta_ref;
    uint64_t seed;
    double perturb;
    int strict_qs;
    double alpha; /* accelerated sweep (Sec. V.H); 0 means 1, the plain sweep */
    int mag_scheme; /* 0: quasi-static sweeps (tau_m = 1); 1: one update per step (R14) */
    double gamma;   /* time-step rescaling (Sec. VII); 0 means 1 */
    const double* b0_field; /* ORC_B0_FIELD: [3][ny][nx], copied at creation */
    int flow_q;     /* 3-D flow lattice: 19 (also 0) or 27 (R17) */
    int flow_scheme; /* 0: single-step; 1: macroscopic scheme for tau >= 1 (R18) */
} orc_params;

typedef struct orc_derived {
    double R, U0, nu, tau, eta, B0, F0, c_mag, lambda, lambda_m, cs2, cm2;
    int n_mag, n_markers;
    double tau_m; /* relaxation time of the magnetic update: 1, or R14 */
    double gamma; /* time-step rescaling in use (R15; 6 nu for R18) */
} orc_derived;

typedef struct lattice {
    int q;
    int c[27][3];
    double w[27];
} lattice;

typedef struct orc {
    orc_params p;
    orc_derived d;
    lattice flow, field;
    long n;
    double *rho, *u[3], *b[3];
    double *rho_new, *u_new[3], *b_new[3];
    double *F[3];
    double *usnap[3];
    long t, tsnap;
    double mass0;
    double ig; /* 1/gamma */
    double* b0f; /* ORC_B0_FIELD: [3][ny][nx] */
    int nm;
    double *X, *Y, *Z, *dj, *sj, *smj;
} orc;

/* ------------------------------------------------------------------ lattices */

static void set_lattice(lattice* L, int q, const int (*c)[3], const double* w) {
    L->q = q;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) L->c[i][a] = c[i][a];
        L->w[i] = w[i];
    }
}

static void make_lattices(orc* o) {
    if (o->p.dim == 2) {
        static const int c9[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                     {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        static const double w9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                     1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        static const int c5[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}};
        static const double w5[5] = {1.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
        set_lattice(&o->flow, 9, c9, w9);
        set_lattice(&o->field, 5, c5, w5);
    } else {
        static const int c19[19][3] = {
            {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
            {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
            {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        double w19[19];
        w19[0] = 1.0 / 3;
        for (int i = 1; i <= 6; ++i) w19[i] = 1.0 / 18;
        for (int i = 7; i < 19; ++i) w19[i] = 1.0 / 36;
        static const int c7[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                     {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        static const double w7[7] = {1.0 / 4, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8};
        if (o->p.flow_q == 27) {
            /* Table I: the D3Q19 set plus the eight corners (+-1, +-1, +-1) */
            int c27[27][3];
            double w27[27];
            for (int i = 0; i < 19; ++i)
                for (int a = 0; a < 3; ++a) c27[i][a] = c19[i][a];
            int i = 19;
            for (int sz = 1; sz >= -1; sz -= 2)
                for (int sy = 1; sy >= -1; sy -= 2)
                    for (int sx = 1; sx >= -1; sx -= 2) {
                        c27[i][0] = sx;
                        c27[i][1] = sy;
                        c27[i][2] = sz;
                        ++i;
                    }
            w27[0] = 8.0 / 27;
            for (i = 1; i <= 6; ++i) w27[i] = 2.0 / 27;
            for (i = 7; i < 19; ++i) w27[i] = 1.0 / 54;
            for (i = 19; i < 27; ++i) w27[i] = 1.0 / 216;
            set_lattice(&o->flow, 27, c27, w27);
        } else {
            set_lattice(&o->flow, 19, c19, w19);
        }
        set_lattice(&o->field, 7, c7, w7);
    }
}

/* ------------------------------------------------------------------- helpers */

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

static long node(const orc* o, int x, int y, int z) {
    x = wrap(x, o->p.nx);
    y = wrap(y, o->p.ny);
    z = wrap(z, o->p.nz);
    return ((long)z * o->p.ny + y) * o->p.nx + x;
}

static void coords(const orc* o, long k, int* x, int* y, int* z) {
    *x = (int)(k % o->p.nx);
    *y = (int)((k / o->p.nx) % o->p.ny);
    *z = (int)(k / ((long)o->p.nx * o->p.ny));
}

/* splitmix64 (Steele, Lea, Flood, OOPSLA 2014): one increment of the Weyl state
 * by the golden-ratio constant followed by the published 64-bit finaliser. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Applied field B^ext at node (x, y, z): uniform B0 * dir, or the ramp
 * B0 * 0.5 (1 + tanh((z - zc)/w)) * dir along the pipe axis (Sec. VI). */
static void bext(const orc* o, int x, int y, int z, double B[3]) {
    if (o->p.b0_kind == ORC_B0_FIELD) { /* a z-invariant field, e.g. of magnets (Sec. VI) */
        long P = (long)o->p.nx * o->p.ny, q = (long)y * o->p.nx + x;
        for (int a = 0; a < 3; ++a) B[a] = o->d.B0 * o->b0f[a * P + q];
        return;
    }
    double amp = o->d.B0;
    if (o->p.b0_kind == ORC_B0_TANH) amp = o->d.B0 * 0.5 * (1.0 + tanh(((double)z - o->p.ramp_center) / o->p.ramp_width));
    for (int a = 0; a < 3; ++a) B[a] = amp * o->p.b0_dir[a];
}

/* ------------------------------------------------------- parameter mapping */

/* N_mag = ceil(c) (Sec. V.G, Eq. "Number of iterations magnetic field"), with
 * c = 1/dt for dx = 1.  A value that is an integer up to a relative 1e-12 of
 * rounding counts as that integer. */
static int ceil_tol(double v) {
    double r = nearbyint(v);
    if (fabs(v - r) <= 1e-12 * fabs(v)) return (int)r;
    return (int)ceil(v);
}

int orc_derive(const orc_params* p, orc_derived* d) {
    memset(d, 0, sizeof(*d));
    d->cs2 = 1.0 / 3.0;
    d->cm2 = (p->dim == 2) ? 1.0 / 3.0 : 1.0 / 4.0;
    if (p->dim == 3 && !(p->flow_q == 0 || p->flow_q == 19 || p->flow_q == 27)) return -1;
    if (p->dim == 2 && !(p->flow_q == 0 || p->flow_q == 9)) return -1;
    double R = 0.5 * p->diameter;
    if (!(R > 0)) return -1;
    d->R = R;
    if (p->flow_scheme != 0 && p->flow_scheme != 1) return -1;
    double U0 = p->U0;
    if (!(U0 > 0)) {
        U0 = 0.05;
        double tau_cap = p->Re * d->cs2 / (2.0 * R);
        if (tau_cap < U0 && p->flow_scheme == 0) U0 = tau_cap; /* R18: no tau bound */
        if (p->Ha > 0) {
            double lor_cap = p->Re * R / (2.0 * p->Ha * p->Ha);
            if (lor_cap < U0) U0 = lor_cap;
        }
    }
    d->U0 = U0;
    d->nu = U0 * R / p->Re;                 /* Re = U0 L / nu  (Sec. II)        */
    double g = p->gamma > 0 ? p->gamma : 1.0;
    if (p->flow_scheme == 1) { /* R18: c = 6 nu, tau = 1 */
        if (g != 1.0 || !(6.0 * d->nu >= 1.0 - 1e-12)) return -1;
        g = 6.0 * d->nu;
    }
    d->gamma = g;
    d->tau = d->nu / (g * d->cs2) + 0.5;    /* nu = gamma c_s^2 (tau - 1/2)    */
    if (p->flow_scheme == 1) d->tau = 1.0;  /* R18: the scheme is tau = 1      */
    d->eta = U0 * R / p->Rm;                /* Rm = U0 L / eta                  */
    d->B0 = p->Ha * sqrt(d->eta * d->nu) / R; /* Ha = B0 L / sqrt(eta nu)       */
    if (p->geometry == ORC_CHANNEL)
        d->F0 = 2.0 * d->nu * U0 / (R * R);
    else
        d->F0 = 4.0 * d->nu * U0 / (R * R);
    /* eta = c_s^2 (tau_m - 1/2) dt with tau_m = 1, c_s^2 = c^2 c_m^2, dx = c dt = 1
     * gives eta = c c_m^2 / 2, so c = 2 eta / c_m^2 and N_mag = ceil(c).          */
    d->c_mag = 2.0 * d->eta / (g * d->cm2);
    d->tau_m = 1.0;
    int n = p->n_mag > 0 ? p->n_mag : ceil_tol(d->c_mag);
    if (p->n_mag <= 0 && p->n_mag_cap > 0 && n > p->n_mag_cap) n = p->n_mag_cap;
    if (n < 1) n = 1;
    if (p->mag_scheme == 1) { /* R14 */
        d->c_mag = 1.0;
        d->tau_m = d->eta / (g * d->cm2) + 0.5;
        n = 1;
    }
    d->n_mag = n;
    double nu_ref = p->nu_ref > 0 ? p->nu_ref : d->nu / g;
    /* eta_ref: c_m^2/2 for the tau_m = 1 sweeps (lambda_m = c); eta/gamma for
     * the time-resolved update (lambda_m = 1, R14: below one the scaling's pole
     * 1/(1 - lambda_m) falls inside the rings' range of d) */
    double eta_ref = p->eta_ref > 0 ? p->eta_ref : (p->mag_scheme == 1 ? d->eta / g : 0.5 * d->cm2);
    d->lambda = d->nu / g / nu_ref;
    d->lambda_m = d->eta / g / eta_ref;
    return 0;
}

/* ----------------------------------------------------------- IB interpolation */

/* One-dimensional factor of the Lagrange interpolation kernel, Sec. V.B
 * Eq. "Kernel functions for Lagrange interpolation I", on half-open pieces. */
double orc_kernel1d(double r) {
    if (r > -1.5 && r <= -0.5) return 0.5 * (r + 1.0) * (r + 2.0);
    if (r > -0.5 && r <= 0.5) return 1.0 - r * r;
    if (r > 0.5 && r <= 1.5) return 0.5 * (r - 1.0) * (r - 2.0);
    return 0.0;
}

/* D(x_k - X_j) = D_x D_y D_z; in two dimensions D_x D_y. */
static double kernel(const orc* o, double rx, double ry, double rz) {
    double v = orc_kernel1d(rx) * orc_kernel1d(ry);
    if (o->p.dim == 3) v *= orc_kernel1d(rz);
    return v;
}

/* Iterate the support S(j) = { k : |x_k - X_j| <= 2 per axis } of marker j and
 * call fn(k, D) for each node; D is zero outside the kernel's pieces. */
typedef void (*support_fn)(orc* o, long k, double D, void* ctx);

static void for_support(orc* o, int j, support_fn fn, void* ctx) {
    double X = o->X[j], Y = o->Y[j], Z = o->Z[j];
    int x0 = (int)ceil(X - 2.0), x1 = (int)floor(X + 2.0);
    int y0 = (int)ceil(Y - 2.0), y1 = (int)floor(Y + 2.0);
    int z0 = 0, z1 = 0;
    if (o->p.dim == 3) {
        z0 = (int)ceil(Z - 2.0);
        z1 = (int)floor(Z + 2.0);
    }
    for (int kz = z0; kz <= z1; ++kz)
        for (int ky = y0; ky <= y1; ++ky)
            for (int kx = x0; kx <= x1; ++kx) {
                double D = kernel(o, (double)kx - X, (double)ky - Y, (double)kz - Z);
                if (D != 0.0) fn(o, node(o, kx, ky, kz), D, ctx);
            }
}

typedef struct {
    double* W;
} ctx_w;
static void add_to_w(orc* o, long k, double D, void* c) {
    (void)o;
    ((ctx_w*)c)->W[k] += D;
}

typedef struct {
    const double* W;
    double acc;
} ctx_d;
static void acc_d(orc* o, long k, double D, void* c) {
    (void)o;
    ctx_d* q = (ctx_d*)c;
    q->acc += D * q->W[k];
}

typedef struct {
    double* f[3];
    double acc[3];
    double delta[3];
} ctx_field;
static void gather_field(orc* o, long k, double D, void* c) {
    (void)o;
    ctx_field* q = (ctx_field*)c;
    for (int a = 0; a < 3; ++a) q->acc[a] += D * q->f[a][k];
}
static void spread_field(orc* o, long k, double D, void* c) {
    (void)o;
    ctx_field* q = (ctx_field*)c;
    for (int a = 0; a < 3; ++a) q->f[a][k] += D * q->delta[a];
}

/* Wall markers (Sec. V.B and Fig. 3(b)): a channel has one marker per node
 * spacing on each wall line; a pipe has rings of round(pi D / spacing) markers
 * at every integer z, centred on (cx, cy). */
static void make_markers(orc* o) {
    const orc_params* p = &o->p;
    o->nm = 0;
    if (p->geometry == ORC_NONE) return;
    if (p->geometry == ORC_CHANNEL) {
        int per = (int)llround(p->nx / p->marker_spacing);
        o->nm = 2 * per * (p->dim == 3 ? p->nz : 1);
        o->X = malloc(sizeof(double) * o->nm);
        o->Y = malloc(sizeof(double) * o->nm);
        o->Z = malloc(sizeof(double) * o->nm);
        int m = 0;
        int nzr = p->dim == 3 ? p->nz : 1;
        for (int z = 0; z < nzr; ++z)
            for (int w = 0; w < 2; ++w)
                for (int i = 0; i < per; ++i) {
                    o->X[m] = i * p->marker_spacing;
                    o->Y[m] = (w == 0) ? p->cy - o->d.R : p->cy + o->d.R;
                    o->Z[m] = z;
                    ++m;
                }
        return;
    }
    int nth = (int)llround(M_PI * p->diameter / p->marker_spacing);
    o->nm = nth * p->nz;
    o->X = malloc(sizeof(double) * o->nm);
    o->Y = malloc(sizeof(double) * o->nm);
    o->Z = malloc(sizeof(double) * o->nm);
    int m = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int i = 0; i < nth; ++i) {
            double th = 2.0 * M_PI * (double)i / (double)nth;
            o->X[m] = p->cx + o->d.R * cos(th);
            o->Y[m] = p->cy + o->d.R * sin(th);
            o->Z[m] = z;
            ++m;
        }
}

/* d_i = sum_j A_ij with A_ij = sum_k D(x_k - X_i) D(x_k - X_j) (Sec. V.C),
 * evaluated as sum_k D(x_k - X_i) W(x_k), W = sum_j D(x_k - X_j).  Then the
 * scalings of Sec. V.E and V.F: s = lambda / (d (1 + d (lambda - 1))). */
static void ib_setup(orc* o) {
    if (o->nm == 0) return;
    double* W = calloc(o->n, sizeof(double));
    ctx_w cw = {W};
    for (int j = 0; j < o->nm; ++j) for_support(o, j, add_to_w, &cw);
    o->dj = malloc(sizeof(double) * o->nm);
    o->sj = malloc(sizeof(double) * o->nm);
    o->smj = malloc(sizeof(double) * o->nm);
    for (int j = 0; j < o->nm; ++j) {
        ctx_d cd = {W, 0.0};
        for_support(o, j, acc_d, &cd);
        double d = cd.acc, l = o->d.lambda, lm = o->d.lambda_m;
        o->dj[j] = d;
        o->sj[j] = l / (d * (1.0 + d * (l - 1.0)));
        o->smj[j] = lm / (d * (1.0 + d * (lm - 1.0)));
    }
    free(W);
}

/* Explicit IB corrector (Sec. V.C-V.F): every marker first interpolates the
 * predictor field, delta_j = s_j (U_b - D f*) with U_b = 0, and only then are
 * the corrections spread, f = f* + D^T delta. */
static void ib_apply(orc* o, double* f[3], const double* s) {
    if (o->nm == 0) return;
    double* delta = malloc(sizeof(double) * 3 * o->nm);
    for (int j = 0; j < o->nm; ++j) {
        ctx_field q;
        for (int a = 0; a < 3; ++a) {
            q.f[a] = f[a];
            q.acc[a] = 0.0;
        }
        for_support(o, j, gather_field, &q);
        for (int a = 0; a < 3; ++a) delta[3 * j + a] = s[j] * (0.0 - q.acc[a]);
    }
    for (int j = 0; j < o->nm; ++j) {
        ctx_field q;
        for (int a = 0; a < 3; ++a) {
            q.f[a] = f[a];
            q.delta[a] = delta[3 * j + a];
        }
        for_support(o, j, spread_field, &q);
    }
    free(delta);
}

/* ---------------------------------------------------------- magnetic sweep */

/* g^eq_{i,alpha} at node y (Sec. III.E Eq. "Equilibrium distribution for
 * magnetic field I-III"): w_i [ b_alpha + sum_beta (c_{i beta}/c_s^2)
 * (u_beta B_alpha - u_alpha B_beta) ], with c_i = c e_i and c_s^2 = c^2 c_m^2,
 * so that c_{i beta}/c_s^2 = e_{i beta} / (c c_m^2).  B = B^ext + b in the flux
 * (B^ext only when strict_qs is set). */
static double geq(const orc* o, int i, int a, long y) {
    int x0, y0, z0;
    coords(o, y, &x0, &y0, &z0);
    double Be[3], B[3], u[3];
    bext(o, x0, y0, z0, Be);
    for (int c = 0; c < 3; ++c) {
        B[c] = o->p.strict_qs ? Be[c] : Be[c] + o->b[c][y];
        u[c] = o->u[c][y];
    }
    double flux = 0.0;
    for (int be = 0; be < 3; ++be) {
        int e = o->field.c[i][be];
        if (e == 0) continue;
        flux += (double)e / (o->d.c_mag * o->d.cm2) * (u[be] * B[a] - u[a] * B[be]) * o->ig;
    }
    if (i == 0) /* rest direction: (w_0 - 1 + alpha) b (reading R13) */
        return (o->p.alpha - 1.0 + o->field.w[0]) * o->b[a][y];
    return o->field.w[i] * (o->b[a][y] + flux);
}

/* One sweep of the tau_m = 1 scheme (Sec. V.G, Eq. "Single step algoritm for
 * magnetic field"): b_alpha(x) <- sum_i g^eq_{i alpha}(x - e_i); with the
 * accelerated equilibria of Sec. V.H the sum is multiplied by 1/alpha.  With
 * mag_scheme = 1 the update of Sec. III.D for any tau_m:
 * b_alpha(x) <- sum_i { g_i(x - e_i) + (tau_m - 1) [g_i(x + e_i) - 2 g_i(x) + g_i(x - e_i)] }. */
static void sweep(orc* o) {
    long n = o->n;
    const double inv_alpha = 1.0 / o->p.alpha;
    const double tm = o->d.tau_m;
    const int full = o->p.mag_scheme == 1;
#pragma omp parallel for schedule(static) if (n >= ORC_OMP_MIN_NODES)
    for (long k = 0; k < n; ++k) {
        int x, y, z;
        coords(o, k, &x, &y, &z);
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int i = 0; i < o->field.q; ++i) {
                long ym = node(o, x - o->field.c[i][0], y - o->field.c[i][1], z - o->field.c[i][2]);
                if (!full) {
                    s += geq(o, i, a, ym);
                } else {
                    long yp = node(o, x + o->field.c[i][0], y + o->field.c[i][1], z + o->field.c[i][2]);
                    double gm = geq(o, i, a, ym), gp = geq(o, i, a, yp), g0 = geq(o, i, a, k);
                    s += gm + (tm - 1.0) * (gp - 2.0 * g0 + gm);
                }
            }
            o->b_new[a][k] = s * inv_alpha;
        }
    }
    for (int a = 0; a < 3; ++a) {
        double* t = o->b[a];
        o->b[a] = o->b_new[a];
        o->b_new[a] = t;
    }
}

/* N magnetic sub-iterations with u frozen, IB on b after each one. */
void orc_mag_sweeps(orc* o, int nsweeps) {
    for (int s = 0; s < nsweeps; ++s) {
        sweep(o);
        ib_apply(o, o->b, o->smj);
    }
}

/* --------------------------------------------------------------- flow step */

/* Eq. "Equilibrium distribution simple fluids" at node y. */
static double feq(const orc* o, int i, long y) {
    const double cs2 = o->d.cs2;
    double cu = 0.0, uu = 0.0;
    for (int a = 0; a < 3; ++a) {
        cu += o->flow.c[i][a] * o->u[a][y];
        uu += o->u[a][y] * o->u[a][y];
    }
    return o->flow.w[i] * o->rho[y] *
           (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) * o->ig - uu / (2.0 * cs2) * o->ig);
}

/* Isotropic first derivative on the flow lattice: d_beta phi(x) ~
 * (1/c_s^2) sum_i w_i c_{i beta} phi(x + c_i). */
static double d_iso(const orc* o, const double* phi, int x, int y, int z, int be) {
    double s = 0.0;
    for (int i = 0; i < o->flow.q; ++i) {
        int cb = o->flow.c[i][be];
        if (cb == 0) continue;
        s += o->flow.w[i] * cb * phi[node(o, x + o->flow.c[i][0], y + o->flow.c[i][1], z + o->flow.c[i][2])];
    }
    return s / o->d.cs2;
}

/* Body force along the pipe axis (z in 3-D, x in the 2-D channel), Eq.
 * "variable force" with a sine modulation: F0 (1 + amp sin(2 pi t / T)). */
static double body_force(const orc* o, long t) {
    double f = o->d.F0;
    if (o->p.force_amp != 0.0 && o->p.force_period > 0.0)
        f *= 1.0 + o->p.force_amp * sin(2.0 * M_PI * ((double)t * o->ig) / o->p.force_period);
    return f;
}
static int axis(const orc* o) { return o->p.dim == 3 ? 2 : 0; }

/* J = curl b by isotropic differences, F = F_body + J x (B^ext + b) (Sec. V.A). */
static void current_at(const orc* o, int x, int y, int z, double J[3]) {
    double dbz_dy = d_iso(o, o->b[2], x, y, z, 1), dby_dz = d_iso(o, o->b[1], x, y, z, 2);
    double dbx_dz = d_iso(o, o->b[0], x, y, z, 2), dbz_dx = d_iso(o, o->b[2], x, y, z, 0);
    double dby_dx = d_iso(o, o->b[1], x, y, z, 0), dbx_dy = d_iso(o, o->b[0], x, y, z, 1);
    J[0] = dbz_dy - dby_dz;
    J[1] = dbx_dz - dbz_dx;
    J[2] = dby_dx - dbx_dy;
}

static void compute_force(orc* o) {
    long n = o->n;
    double fb = body_force(o, o->t);
    int ax = axis(o);
#pragma omp parallel for schedule(static) if (n >= ORC_OMP_MIN_NODES)
    for (long k = 0; k < n; ++k) {
        int x, y, z;
        coords(o, k, &x, &y, &z);
        double J[3], Be[3], B[3];
        current_at(o, x, y, z, J);
        bext(o, x, y, z, Be);
        for (int a = 0; a < 3; ++a) B[a] = Be[a] + o->b[a][k];
        double L[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2], J[0] * B[1] - J[1] * B[0]};
        for (int a = 0; a < 3; ++a) o->F[a][k] = L[a] + (a == ax ? fb : 0.0);
    }
}

/* GZS forcing term (Sec. V.A, Eq. "FGS forcing term algorithm") for direction
 * i at node y: (1 - 1/(2 tau)) w_i [ (c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4 ] . F */
static double gzs(const orc* o, int i, long y) {
    const double cs2 = o->d.cs2;
    double cu = 0.0, cF = 0.0, uF = 0.0, ciF = 0.0;
    for (int a = 0; a < 3; ++a) {
        double c = o->flow.c[i][a];
        cu += c * o->u[a][y];
        cF += c * o->F[a][y];
        uF += o->u[a][y] * o->F[a][y];
    }
    ciF = cF;
    /* rescaled (Sec. VII): [(c_i - u/gamma)/(gamma c_s^2) + (c_i . u) c_i/(gamma^2 c_s^4)] . F */
    const double ig = o->ig, ig2 = o->ig * o->ig;
    return (1.0 - 1.0 / (2.0 * o->d.tau)) * o->flow.w[i] *
           ((ciF * ig - uF * ig2) / cs2 + cu * cF * ig2 / (cs2 * cs2));
}

/* Same forcing term for caller-given u and F (used to pin its moments). */
void orc_gzs_terms(int dim, int flow_q, double tau, double gamma, const double* u, const double* F, double* Fi,
                   int* q_out, int* c_out) {
    orc tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.p.dim = dim;
    tmp.p.flow_q = flow_q;
    make_lattices(&tmp);
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < tmp.flow.q; ++i) {
        double cu = 0.0, cF = 0.0, uF = 0.0;
        for (int a = 0; a < 3; ++a) {
            double c = tmp.flow.c[i][a];
            cu += c * u[a];
            cF += c * F[a];
            uF += u[a] * F[a];
            c_out[3 * i + a] = tmp.flow.c[i][a];
        }
        const double ig = 1.0 / gamma, ig2 = ig * ig;
        Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * tmp.flow.w[i] * ((cF * ig - uF * ig2) / cs2 + cu * cF * ig2 / (cs2 * cs2));
    }
    *q_out = tmp.flow.q;
}

/* The flow lattice of (dim, flow_q): q velocities c[3 q] and weights w[q]
 * (Sec. III.A; Table I for flow_q = 27).  Returns q. */
int orc_flow_lattice(int dim, int flow_q, int* c_out, double* w_out) {
    orc tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.p.dim = dim;
    tmp.p.flow_q = flow_q;
    make_lattices(&tmp);
    for (int i = 0; i < tmp.flow.q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = tmp.flow.c[i][a];
        w_out[i] = tmp.flow.w[i];
    }
    return tmp.flow.q;
}

/* Single-step flow update with the discrete-effect correction (Sec. III.E Eq.
 * "single-step algorithm complete" for rho; Sec. V.A Eq. "Single-step algorithm
 * with lattice discrete effect" for rho u), then u* = (rho u)* / rho*. */
static void flow_update(orc* o) {
    long n = o->n;
    const double tau = o->d.tau;
#pragma omp parallel for schedule(static) if (n >= ORC_OMP_MIN_NODES)
    for (long k = 0; k < n; ++k) {
        int x, y, z;
        coords(o, k, &x, &y, &z);
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < o->flow.q; ++i) {
            const int* c = o->flow.c[i];
            long km = node(o, x - c[0], y - c[1], z - c[2]);
            long kp = node(o, x + c[0], y + c[1], z + c[2]);
            double fm = feq(o, i, km), f0 = feq(o, i, k), fp = feq(o, i, kp);
            if (o->p.flow_scheme == 1)
                rho += fm; /* R18: Eq. "densities MAC" */
            else
                rho += 1.5 * fm - f0 + 0.5 * fp;
            double mom = fm + (tau - 1.0) * (fp - 2.0 * f0 + fm);
            double corr = -0.5 * tau * (gzs(o, i, kp) - gzs(o, i, km));
            for (int a = 0; a < 3; ++a) m[a] += c[a] * mom + c[a] * corr;
        }
        for (int a = 0; a < 3; ++a) m[a] += o->F[a][k] * o->ig; /* F dt, dt = 1/gamma (R15) */
        o->rho_new[k] = rho;
        for (int a = 0; a < 3; ++a) o->u_new[a][k] = m[a] / rho;
    }
    double* t = o->rho;
    o->rho = o->rho_new;
    o->rho_new = t;
    for (int a = 0; a < 3; ++a) {
        t = o->u[a];
        o->u[a] = o->u_new[a];
        o->u_new[a] = t;
    }
}

/* One flow step (order of Sec. V.G: the magnetic algorithm is iterated N_mag
 * times before every velocity update). */
static void one_step(orc* o) {
    orc_mag_sweeps(o, o->d.n_mag);
    compute_force(o);
    flow_update(o);
    ib_apply(o, o->u, o->sj);
    o->t += 1;
}

void orc_step(orc* o, long nsteps) {
    for (long s = 0; s < nsteps; ++s) one_step(o);
}

/* Test hook: one flow update (density, momentum with the GZS correction,
 * plus F) with the force field F [3 n] given by the caller instead of the
 * Lorentz and body forces, and without the IB on u; t does not advance. */
void orc_flow_update_with_force(orc* o, const double* F) {
    for (int a = 0; a < 3; ++a) memcpy(o->F[a], F + (long)a * o->n, (size_t)o->n * sizeof(double));
    flow_update(o);
}

/* Test hook: the force field F [3 n] the next flow update would add for the
 * current state and time (body force plus the Lorentz force J x (B^ext + b)
 * with J = curl b by isotropic differences, Sec. V.A). */
void orc_force(orc* o, double* F) {
    compute_force(o);
    for (int a = 0; a < 3; ++a) memcpy(F + (long)a * o->n, o->F[a], (size_t)o->n * sizeof(double));
}

/* -------------------------------------------------------------- lifecycle */

static int in_fluid(const orc* o, int x, int y, double margin) {
    if (o->p.geometry == ORC_NONE) return 1;
    if (o->p.geometry == ORC_CHANNEL) return fabs((double)y - o->p.cy) <= o->d.R - margin;
    double dx = x - o->p.cx, dy = y - o->p.cy;
    return sqrt(dx * dx + dy * dy) <= o->d.R - margin;
}

orc* orc_create(const orc_params* p) {
    orc* o = calloc(1, sizeof(orc));
    o->p = *p;
    if (o->p.dim == 2) o->p.nz = 1;
    if (o->p.alpha == 0.0) o->p.alpha = 1.0;
    if (!(o->p.gamma > 0.0)) o->p.gamma = 1.0;
    if (orc_derive(&o->p, &o->d) != 0) {
        free(o);
        return NULL;
    }
    o->p.gamma = o->d.gamma; /* R18 sets it from nu */
    o->ig = 1.0 / o->p.gamma;
    make_lattices(o);
    if (o->p.b0_kind == ORC_B0_FIELD) {
        long P = (long)o->p.nx * o->p.ny;
        o->b0f = malloc(3 * P * sizeof(double));
        if (!o->b0f || !o->p.b0_field) {
            free(o->b0f);
            free(o);
            return NULL;
        }
        memcpy(o->b0f, o->p.b0_field, 3 * P * sizeof(double));
        o->p.b0_field = NULL;
    }
    o->n = (long)o->p.nx * o->p.ny * o->p.nz;
    long n = o->n;
    o->rho = calloc(n, sizeof(double));
    o->rho_new = calloc(n, sizeof(double));
    for (int a = 0; a < 3; ++a) {
        o->u[a] = calloc(n, sizeof(double));
        o->b[a] = calloc(n, sizeof(double));
        o->u_new[a] = calloc(n, sizeof(double));
        o->b_new[a] = calloc(n, sizeof(double));
        o->F[a] = calloc(n, sizeof(double));
        o->usnap[a] = calloc(n, sizeof(double));
    }
    /* rho = 1, b = 0, u = seeded perturbation inside the wall: splitmix64 of
     * seed xor (3 k + component), top 53 bits mapped to [-1, 1), times
     * perturb * U0.  In two dimensions only the in-plane components are set. */
    int ncomp = o->p.dim == 3 ? 3 : 2;
    for (long k = 0; k < n; ++k) {
        o->rho[k] = 1.0;
        int x, y, z;
        coords(o, k, &x, &y, &z);
        if (o->p.perturb != 0.0 && in_fluid(o, x, y, 0.0)) {
            for (int a = 0; a < ncomp; ++a) {
                uint64_t r = orc_splitmix64(o->p.seed ^ (uint64_t)(3 * k + a));
                double v = (double)(r >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
                o->u[a][k] = o->p.perturb * o->d.U0 * v;
            }
        }
    }
    make_markers(o);
    o->d.n_markers = o->nm;
    ib_setup(o);
    o->mass0 = 0.0;
    for (long k = 0; k < n; ++k) o->mass0 += o->rho[k];
    for (int a = 0; a < 3; ++a) memcpy(o->usnap[a], o->u[a], sizeof(double) * n);
    o->tsnap = 0;
    return o;
}

void orc_destroy(orc* o) {
    if (!o) return;
    free(o->b0f);
    free(o->rho);
    free(o->rho_new);
    for (int a = 0; a < 3; ++a) {
        free(o->u[a]);
        free(o->b[a]);
        free(o->u_new[a]);
        free(o->b_new[a]);
        free(o->F[a]);
        free(o->usnap[a]);
    }
    free(o->X);
    free(o->Y);
    free(o->Z);
    free(o->dj);
    free(o->sj);
    free(o->smj);
    free(o);
}

void orc_get_derived(const orc* o, orc_derived* d) { *d = o->d; }
long orc_nodes(const orc* o) { return o->n; }
long orc_time(const orc* o) { return o->t; }

/* Fields as [component][z][y][x]; rho has one component, u and b three. */
void orc_get_state(const orc* o, double* rho, double* u, double* b) {
    long n = o->n;
    if (rho) memcpy(rho, o->rho, sizeof(double) * n);
    for (int a = 0; a < 3; ++a) {
        if (u) memcpy(u + a * n, o->u[a], sizeof(double) * n);
        if (b) memcpy(b + a * n, o->b[a], sizeof(double) * n);
    }
}

void orc_set_state(orc* o, const double* rho, const double* u, const double* b, long t) {
    long n = o->n;
    if (rho) memcpy(o->rho, rho, sizeof(double) * n);
    for (int a = 0; a < 3; ++a) {
        if (u) memcpy(o->u[a], u + a * n, sizeof(double) * n);
        if (b) memcpy(o->b[a], b + a * n, sizeof(double) * n);
    }
    o->t = t;
}

int orc_markers(const orc* o, double* X, double* Y, double* Z, double* d, double* s, double* sm) {
    for (int j = 0; j < o->nm; ++j) {
        if (X) X[j] = o->X[j];
        if (Y) Y[j] = o->Y[j];
        if (Z) Z[j] = o->Z[j];
        if (d) d[j] = o->dj[j];
        if (s) s[j] = o->sj[j];
        if (sm) sm[j] = o->smj[j];
    }
    return o->nm;
}

/* Apply the explicit IB corrector to a caller field f[3][n] with the velocity
 * (magnetic = 0) or magnetic (magnetic = 1) scaling. */
void orc_ib_apply_field(orc* o, double* f, int magnetic) {
    double* ff[3] = {f, f + o->n, f + 2 * o->n};
    ib_apply(o, ff, magnetic ? o->smj : o->sj);
}

/* --------------------------------------------------------------- diagnostics */

/* out[0..10]: mass, mass_drift, E_k, E_m, pump, visc, joule, qs_residual,
 * steady_residual, nan_flag, time.  Averages <.> over nodes at least two lattice
 * units inside the wall (Sec. IV: a cylinder of radius smaller than the pipe's).
 * Energy terms are the local forms of Eq. "Energy balance equations":
 *   pump  = <F_body . u>,  visc = -nu <u . lap u>,  joule = -<u . (J x B)>,
 * with isotropic flow-lattice differences (lap phi = (2/c_s^2) sum_i w_i
 * (phi(x + c_i) - phi(x))).  The QS residual of Eq. "Error l2 decay" is the RMS
 * over the same region of eta lap_m b - div_m(u B - B u), with the field
 * lattice's own second difference and central first difference (the operators
 * whose solution the sweep converges to).  The steady residual is
 * |u - u_snap|_2 / ((t - t_snap) |u|_2) over the same region against the state
 * at the previous call, which then becomes the new snapshot (nodes outside the
 * wall are not part of the pipe flow and would converge on their own, slower
 * time scale). */
void orc_observables(orc* o, double* out) {
    long n = o->n;
    double mass = 0.0, ek = 0.0, em = 0.0, pump = 0.0, visc = 0.0, joule = 0.0, qs = 0.0;
    double du2 = 0.0, u2 = 0.0;
    long cnt = 0;
    int nan = 0;
    double fb = body_force(o, o->t);
    int ax = axis(o);
    for (long k = 0; k < n; ++k) {
        mass += o->rho[k];
        if (!isfinite(o->rho[k])) nan = 1;
        for (int a = 0; a < 3; ++a)
            if (!isfinite(o->u[a][k]) || !isfinite(o->b[a][k])) nan = 1;
    }
    for (long k = 0; k < n; ++k) {
        int x, y, z;
        coords(o, k, &x, &y, &z);
        if (!in_fluid(o, x, y, 2.0)) continue;
        ++cnt;
        for (int a = 0; a < 3; ++a) {
            double dd = o->u[a][k] - o->usnap[a][k];
            du2 += dd * dd;
            u2 += o->u[a][k] * o->u[a][k];
        }
        double Be[3], B[3], J[3];
        bext(o, x, y, z, Be);
        for (int a = 0; a < 3; ++a) B[a] = Be[a] + o->b[a][k];
        double uu = 0.0, BB = 0.0;
        for (int a = 0; a < 3; ++a) {
            uu += o->u[a][k] * o->u[a][k];
            BB += B[a] * B[a];
        }
        ek += 0.5 * o->rho[k] * uu;
        em += 0.5 * BB;
        pump += fb * o->u[ax][k];
        double ulap = 0.0;
        for (int a = 0; a < 3; ++a) {
            double lap = 0.0;
            for (int i = 0; i < o->flow.q; ++i) {
                const int* c = o->flow.c[i];
                lap += o->flow.w[i] * (o->u[a][node(o, x + c[0], y + c[1], z + c[2])] - o->u[a][k]);
            }
            lap *= 2.0 / o->d.cs2;
            ulap += o->u[a][k] * lap;
        }
        visc += -o->d.nu * ulap;
        current_at(o, x, y, z, J);
        double L[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2], J[0] * B[1] - J[1] * B[0]};
        joule += -(o->u[0][k] * L[0] + o->u[1][k] * L[1] + o->u[2][k] * L[2]);
        for (int a = 0; a < 3; ++a) {
            double lapb = 0.0, div = 0.0;
            for (int be = 0; be < (o->p.dim == 3 ? 3 : 2); ++be) {
                int e[3] = {0, 0, 0};
                e[be] = 1;
                long kp = node(o, x + e[0], y + e[1], z + e[2]);
                long km = node(o, x - e[0], y - e[1], z - e[2]);
                lapb += o->b[a][kp] + o->b[a][km] - 2.0 * o->b[a][k];
                double Bp[3], Bm[3], Bep[3], Bem[3];
                int xp, yp, zp, xm, ym, zm;
                coords(o, kp, &xp, &yp, &zp);
                coords(o, km, &xm, &ym, &zm);
                bext(o, xp, yp, zp, Bep);
                bext(o, xm, ym, zm, Bem);
                for (int c = 0; c < 3; ++c) {
                    Bp[c] = o->p.strict_qs ? Bep[c] : Bep[c] + o->b[c][kp];
                    Bm[c] = o->p.strict_qs ? Bem[c] : Bem[c] + o->b[c][km];
                }
                double phip = o->u[be][kp] * Bp[a] - o->u[a][kp] * Bp[be];
                double phim = o->u[be][km] * Bm[a] - o->u[a][km] * Bm[be];
                div += 0.5 * (phip - phim);
            }
            double r = o->d.eta * lapb - div;
            qs += r * r;
        }
    }
    double inv = cnt > 0 ? 1.0 / (double)cnt : 0.0;
    out[0] = mass;
    out[1] = (mass - o->mass0) / o->mass0;
    out[2] = ek * inv;
    out[3] = em * inv;
    out[4] = pump * inv;
    out[5] = visc * inv;
    out[6] = joule * inv;
    out[7] = sqrt(qs * inv);
    long dt = o->t - o->tsnap;
    out[8] = (dt > 0 && u2 > 0) ? sqrt(du2) / ((double)dt * sqrt(u2)) : 0.0;
    out[9] = nan;
    out[10] = (double)o->t;
    for (int a = 0; a < 3; ++a) memcpy(o->usnap[a], o->u[a], sizeof(double) * n);
    o->tsnap = o->t;
}
