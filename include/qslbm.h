/*
 * qslbm: C ABI of a GB300 (sm_103a) implementation of the single-step
 * simplified lattice Boltzmann method for quasi-static MHD pipe flow
 * (H.S. Tavares, B. Magacho, L. Moriconi, J. Loureiro, arXiv 2211.09370).
 *
 * One flow step t -> t+1 runs, in the paper's order:
 *   1. N_mag sweeps of the tau_m = 1 magnetic scheme (Sec. V.G, Eq. "Single step
 *      algoritm for magnetic field") on the induced field b, with u frozen; each
 *      sweep is followed by the explicit immersed-boundary corrector for b
 *      (Sec. V.D, scaled as in Sec. V.F, Eq. "IB corrected for magnetic field").
 *   2. The Lorentz force J x B with J = curl b by isotropic differences and the
 *      body force (Sec. V.A, Eq. "variable force").
 *   3. The single-step flow update with GZS forcing and the discrete-effect
 *      correction (Sec. III.E Eq. "single-step algorithm complete" for rho,
 *      Sec. V.A Eq. "Single-step algorithm with lattice discrete effect").
 *   4. The explicit immersed-boundary corrector for u (Sec. V.C, scaled as in
 *      Sec. V.E, Eq. "IBM correted for velocity field").
 *
 * Conventions for every entry point:
 *   - Return value 0 (QSLBM_OK) or a negative QSLBM_E* code; no exception or
 *     signal crosses the ABI.  qslbm_strerror() names a code.
 *   - Host pointers are caller-owned and are read or written before the call
 *     returns.  Field arrays are binary64, layout [component][z][y][x] with x
 *     fastest (rho has one component, u and b three).
 *   - The library owns all device memory of a handle: it is allocated by
 *     qslbm_create and released by qslbm_destroy.
 *   - Work is queued on the CUDA stream given in the parameters (NULL = the
 *     legacy default stream).  qslbm_step and qslbm_mag_sweeps return once the
 *     work is queued; errors raised by device work surface at the next call
 *     that synchronises (qslbm_observables, qslbm_get_state, qslbm_sync,
 *     qslbm_destroy).
 *   - A handle is not thread-safe; distinct handles may be used from distinct
 *     threads.
 *   - The device must be an sm_103 GPU; nothing falls back to the CPU.
 */
#ifndef QSLBM_H
#define QSLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define QSLBM_OK 0
#define QSLBM_EINVAL -1    /* invalid parameter or argument                    */
#define QSLBM_ENOMEM -2    /* device or host allocation failed                 */
#define QSLBM_ECUDA -3     /* a CUDA call failed (message: qslbm_last_error)   */
#define QSLBM_EUNSTABLE -4 /* non-finite field value detected                  */
#define QSLBM_ETIMEOUT -5  /* step cap reached before the stop tolerance, or a bounded device wait gave up */
#define QSLBM_EBUDGET -6   /* request does not fit the device-memory budget    */
#define QSLBM_ENOTFOUND -7 /* unknown request id                               */
#define QSLBM_EARCH -8     /* device is not sm_103                             */

#define QSLBM_CHANNEL 0  /* two flat walls y = cy -/+ D/2, markers on x        */
#define QSLBM_PIPE 1     /* circular pipe of diameter D along z (x in 2-D)    */
#define QSLBM_PERIODIC 2 /* periodic box without walls                        */

#define QSLBM_B0_UNIFORM 0 /* B^ext = B0 * b0_dir                              */
#define QSLBM_B0_TANH 1    /* B^ext = B0 * 0.5 (1 + tanh((z - zc)/w)) * b0_dir  */
#define QSLBM_B0_FIELD 2   /* B^ext = B0 * b0_field(x, y): a z-invariant in-plane
                              field, e.g. of magnets around the pipe (Sec. VI)   */

#define QSLBM_FP32 0
#define QSLBM_FP64 1

/* Magnetic sub-iteration kernels.  PLANES: one launch per sweep, one CTA per
 * z plane (sweep and IB fused).  RESIDENT: one cooperative launch per step
 * keeps every plane in shared memory (needs nz co-resident CTAs and a plane of
 * at most 8192 nodes; create fails with QSLBM_EINVAL if the domain does not
 * fit).  SPLIT: per sweep a node-parallel sweep launch and a per-plane IB
 * launch.  FUSED: per sweep one launch in which each CTA sweeps a band of
 * rows of a z chunk, plane by plane, and applies the IB on b to it in shared
 * memory (the band's rows are staged by the tensor memory accelerator with
 * three halo rows on each side); FP32, 3-D, nx a multiple of 4 up to 256, the
 * same wall ring on every plane; create fails with QSLBM_EINVAL otherwise.
 * AUTO picks RESIDENT when it fits; else, when FUSED applies, it times FUSED
 * and SPLIT on the handle's fields at creation (without changing them) and
 * keeps FUSED only when it is at least 2 % faster (the two give bitwise equal
 * results); else SPLIT. */
/* Initial velocity: rest (plus the seeded noise), or the Ha = 0 profile
 * U0 (1 - r^2/R^2) along the axis inside the wall (plus the noise). */
#define QSLBM_INIT_REST 0
#define QSLBM_INIT_POISEUILLE 1

#define QSLBM_SWEEP_AUTO 0
#define QSLBM_SWEEP_PLANES 1
#define QSLBM_SWEEP_RESIDENT 2
#define QSLBM_SWEEP_SPLIT 3
#define QSLBM_SWEEP_FUSED 4

/* Flow schemes.  SINGLE_STEP: the single-step update (Sec. III.E, V.A), tau < 1.
 * MACROSCOPIC: the tau = 1 scheme at particle speed c = 6 nu for tau >= 1
 * (Sec. V.G Eqs. "densities MAC", "momentum Mac"): the time step is rescaled
 * by gamma = 6 nu (Sec. VII form), rho and rho u come from the neighbours'
 * equilibria, the force enters as in the single-step scheme at tau = 1; needs
 * 6 nu >= 1 and gamma = 0 or 1; the automatic U0 drops its tau <= 1 bound. */
#define QSLBM_FLOW_SINGLE_STEP 0
#define QSLBM_FLOW_MACROSCOPIC 1

#define QSLBM_MAG_QS 0   /* quasi-static: N_mag tau_m = 1 sweeps per flow step  */
#define QSLBM_MAG_TIME 1 /* time-resolved: one update of Sec. III.D Eq. "single-
                            step algorithm for MHD de rosis" per flow step, with
                            tau_m = eta/c_m^2 + 1/2 (lattice speed 1); needs
                            1/2 < tau_m <= 7/6 (3-D) or 5/4 (2-D) and alpha = 1 */

/* Problem statement of the paper (Sec. II: Re, Rm, Ha with L = pipe radius;
 * Sec. IV: pipe, insulating walls, pressure gradient; Sec. VI: non-uniform
 * applied field).  qslbm_params_init fills the defaults noted here. */
typedef struct qslbm_params {
    int32_t dim;            /* 2 (D2Q9 + D2Q5) or 3 (D3Q19 or D3Q27 + D3Q7); default 3 */
    int32_t nx, ny, nz;     /* periodic box in lattice nodes; 2-D uses nz = 1      */
    int32_t geometry;       /* QSLBM_CHANNEL | QSLBM_PIPE | QSLBM_PERIODIC         */
    double diameter;        /* pipe diameter / wall distance D, lattice units      */
    double center[2];       /* wall centre (x, y); NaN = ((nx-1)/2, (ny-1)/2)      */
    double marker_spacing;  /* Lagrangian marker spacing; default 1.0              */
    double Re, Ha, Rm;      /* L = D/2; Ha = B0 L / sqrt(eta nu)                   */
    double U0;              /* velocity scale; 0 = min(0.05, Re/(6L), Re L/(2Ha^2)) */
    int32_t b0_kind;        /* QSLBM_B0_UNIFORM | QSLBM_B0_TANH | QSLBM_B0_FIELD    */
    double b0_dir[3];       /* unit direction of B^ext; default (1, 0, 0)          */
    double ramp_center;     /* zc of the tanh ramp                                 */
    double ramp_width;      /* w of the tanh ramp                                  */
    double force_amp;       /* F(t) = F0 (1 + amp sin(2 pi t / period)); 0 = const */
    double force_period;    /* period T in flow steps                              */
    int32_t n_mag;          /* sweeps per step; 0 = min(ceil(2 eta / c_m^2), cap)  */
    int32_t n_mag_cap;      /* cap for the automatic count; <= 0 = no cap; 270     */
    double nu_ref;          /* IB reference viscosity; 0 = nu (lambda = 1)         */
    double eta_ref;         /* IB reference resistivity; 0 = c_m^2 / 2 (QS sweeps),
                               eta (lambda_m = 1) for QSLBM_MAG_TIME              */
    int32_t precision;      /* QSLBM_FP32 (default) | QSLBM_FP64                   */
    int32_t strict_qs;      /* 1: induction flux from B^ext only; default 0        */
    uint64_t seed;          /* initial perturbation seed                           */
    double perturb;         /* initial |u| noise, fraction of U0, inside the wall  */
    int32_t init_kind;      /* QSLBM_INIT_REST (default) | QSLBM_INIT_POISEUILLE   */
    int32_t sweep_kernel;   /* QSLBM_SWEEP_AUTO (default) | _PLANES | _RESIDENT | _SPLIT | _FUSED */
    double alpha;           /* accelerated sweep (Sec. V.H, Eq. "magnetic field
                               quasi-static acelerated"): b <- b + (sweep(b) - b)/alpha;
                               1 (default; 0 also means 1) is the plain sweep; stable
                               for 1 - w_0 <= alpha <= 1 (3/4 in 3-D, 2/3 in 2-D) */
    int32_t mag_scheme;     /* QSLBM_MAG_QS (default) | QSLBM_MAG_TIME             */
    double gamma;           /* time step rescaled to dt/gamma (Sec. VII): equilibria,
                               relaxation times and forcing rescaled; forces and
                               resistivity per step over gamma; 1 (default; 0 also
                               means 1); the body-force period is in physical time */
    const double* b0_field; /* QSLBM_B0_FIELD: [3][ny][nx] binary64, read (copied) by
                               qslbm_create only; NULL otherwise                 */
    int32_t flow_q;         /* 3-D flow lattice: 19 (D3Q19; default, 0 also) or 27
                               (D3Q27 of Sec. III.A, Table I); 2-D: 0 or 9        */
    int32_t flow_scheme;    /* QSLBM_FLOW_SINGLE_STEP (default) | QSLBM_FLOW_MACROSCOPIC */
    void* stream;           /* cudaStream_t to queue work on, or NULL              */
} qslbm_params;

/* Lattice-unit values the parameters map to (lambda = nu/nu_ref,
 * lambda_m = eta/eta_ref, c_mag = 2 eta / c_m^2). */
typedef struct qslbm_units {
    double R, U0, nu, tau, eta, B0, F0, c_mag, lambda, lambda_m, cs2, cm2;
    int32_t n_mag, n_markers;
    int64_t nodes;
    int64_t device_bytes; /* device memory the handle holds */
    int64_t shell_nodes;  /* nodes inside the support of some wall marker */
    int32_t sweep_kernel; /* the QSLBM_SWEEP_* kernel in use (never AUTO)        */
    double tau_m;         /* relaxation time of the magnetic update (1 for QS)  */
    int32_t flow_q;       /* velocities of the flow lattice: 9, 19 or 27        */
    double gamma;         /* time-step rescaling in use (6 nu on the macroscopic
                             scheme)                                            */
    int32_t fused_rows;   /* QSLBM_SWEEP_FUSED: rows per band, 0 otherwise      */
    int32_t fused_bands;  /* bands per plane                                    */
    int32_t fused_chunk;  /* z planes each CTA marches per sweep                */
    int32_t fused_ctas;   /* CTAs per sweep launch                              */
    double sweep_us_fused; /* AUTO on a domain both FP32 sweep paths take: one   */
    double sweep_us_split; /* sweep of each timed at creation (microseconds); the
                              faster is kept (their results are bitwise equal);
                              0 when not timed                                   */
} qslbm_units;

/* Diagnostics (Sec. IV Eq. "Energy balance equations", Sec. V.H Eq. "Error l2
 * decay"), accumulated in binary64 on the device.  Averages run over the
 * nodes at least two lattice units inside the wall. */
typedef struct qslbm_obs {
    int64_t step;           /* flow steps taken                                   */
    double mass;            /* sum of rho over the box                            */
    double mass_drift;      /* (mass - initial mass) / initial mass               */
    double E_k, E_m;        /* <rho |u|^2 / 2>, <|B^ext + b|^2 / 2>               */
    double pump;            /* <F_body . u>                                       */
    double visc;            /* -nu <u . lap u>                                    */
    double joule;           /* -<u . (J x B)>                                     */
    double qs_residual;     /* RMS of eta lap b - div(u B - B u)                  */
    double steady_residual; /* |u - u_prev| / ((t - t_prev) |u|) over the averaging
                               region, u_prev from the previous qslbm_observables
                               call                                               */
    int32_t nan_flag;       /* 1 if any field value is not finite                 */
} qslbm_obs;

typedef struct qslbm_handle qslbm_handle;

/* Fill *p with the defaults listed in qslbm_params. */
void qslbm_params_init(qslbm_params* p);

/* Validate *p, map it to lattice units (Sec. II groups; U0 rule above), build
 * the wall markers and their IB weights d_j, s_j, s^m_j (Sec. V.C, V.E, V.F),
 * allocate the fields on the current CUDA device and initialise rho = 1,
 * b = 0 and u = seeded splitmix64 noise of size perturb * U0 inside the wall.
 * *p is copied.  On success *out owns the handle.
 * Errors: QSLBM_EINVAL (bad parameters, wall outside the box, markers not on
 * integer z planes, more than 4096 (FP32) or 2048 (FP64) markers on one plane,
 * the most whose corrections a per-plane IB kernel holds in shared memory;
 * qslbm_last_error gives the reason), QSLBM_ENOMEM, QSLBM_ECUDA, QSLBM_EARCH. */
int qslbm_create(const qslbm_params* p, qslbm_handle** out);

/* Lattice-unit values of the handle.  Errors: QSLBM_EINVAL (NULL argument). */
int qslbm_get_units(const qslbm_handle* h, qslbm_units* out);

/* Queue nsteps >= 0 flow steps (N_mag sweeps + IB on b each, force, flow
 * update, IB on u).  Asynchronous.  Errors: QSLBM_EINVAL, QSLBM_ECUDA. */
int qslbm_step(qslbm_handle* h, int64_t nsteps);

/* Queue nsweeps >= 0 magnetic sweeps (each followed by the IB corrector on b)
 * with u frozen; t does not advance.  Asynchronous. */
int qslbm_mag_sweeps(qslbm_handle* h, int32_t nsweeps);

/* Synchronise the handle's stream and compute the diagnostics into *out
 * (nullable).  rho [n], u [3n], b [3n] (each nullable) receive the fields in
 * binary64.  Errors: QSLBM_EINVAL, QSLBM_ECUDA, QSLBM_EUNSTABLE (the fields
 * hold a non-finite value; *out is still filled). */
int qslbm_observables(qslbm_handle* h, qslbm_obs* out, double* rho, double* u, double* b);

/* Copy the state out / in (binary64 host arrays as above; any may be NULL to
 * leave that field alone).  set_state also sets the step counter to t and
 * makes the uploaded velocity the reference of the steady residual.
 * Synchronous.  Errors: QSLBM_EINVAL, QSLBM_ECUDA. */
int qslbm_get_state(qslbm_handle* h, double* rho, double* u, double* b, int64_t* t);
int qslbm_set_state(qslbm_handle* h, const double* rho, const double* u, const double* b, int64_t t);

/* End-to-end step from and to host memory: upload the state (as set_state),
 * run nsteps flow steps, compute the diagnostics and download the state.
 * rho_in/u_in/b_in and rho_out/u_out/b_out follow the field layout above; the
 * outputs and *obs are nullable. */
int qslbm_step_host(qslbm_handle* h, const double* rho_in, const double* u_in, const double* b_in,
                    int64_t t_in, int64_t nsteps, double* rho_out, double* u_out, double* b_out,
                    qslbm_obs* obs);

/* Wait for all queued work of the handle.  Errors: QSLBM_ECUDA. */
int qslbm_sync(qslbm_handle* h);

/* Release the handle and its device memory (synchronises first). */
int qslbm_destroy(qslbm_handle* h);

/* Allocation-free diagnostics (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory when they need the
 * diagnostics: code recording a CUDA graph, where cudaMalloc is refused while
 * the stream is captured; code whose device memory belongs to another
 * allocator that already holds the pool; loops that must not enter the
 * driver's allocator).
 *
 * Computes the diagnostics of qslbm_observables for fields the caller passes,
 * writing into out[0..9], on the device, in this order: mass, mass_drift, E_k,
 * E_m, pump, visc, joule, qs_residual, steady_residual, nan_flag (1.0 or 0.0).
 *   h                 handle giving geometry, coefficients and the initial mass;
 *                     its own fields are not read or written
 *   drho, u, b        device arrays in the handle's precision (float for
 *                     QSLBM_FP32, double for QSLBM_FP64), layout
 *                     [component][z][y][x]; drho = rho - 1, u and b three
 *                     components each
 *   u_prev            device array like u: the velocity steps_since_prev steps
 *                     earlier (for the steady residual; 0 steps gives 0)
 *   fb                body force for the pumping term (F0 (1 + amp sin(...)))
 *   out               device pointer to 10 doubles, written by the call
 *   stream            cudaStream_t to queue the work on, or NULL
 * The partial sums live in one fixed array inside the library, sized for
 * QSLBM_STATIC_MAX_PLANES z planes (one reduction block per plane,
 * (4096 + 1) x 11 doubles, about 360 KB held by every GPU that loads the
 * library until the process exits).  A domain with more planes is rejected
 * with QSLBM_EINVAL (qslbm_last_error names the limit).  No device memory is
 * allocated or freed.  The first call on a device looks up that array's
 * device address and should be made before any stream capture starts.  Every
 * call on a device shares the array (each call overwrites what it uses, nothing
 * has to start at zero): calls that may run at the same time on the GPU
 * (unordered streams) race and must be serialised by the caller.
 * Asynchronous; errors: QSLBM_EINVAL (NULL argument, too many planes),
 * QSLBM_ECUDA. */
#define QSLBM_STATIC_MAX_PLANES 4096
int qslbm_observables_static(const qslbm_handle* h, const void* drho, const void* u, const void* b,
                             const void* u_prev, double fb, int64_t steps_since_prev, double* out, void* stream);

/* Self-check of the bounded wait (test support; the paper has no counterpart).
 * The resident sweep kernel waits on its neighbour planes' counters with a
 * routine that gives up after a limit instead of spinning for ever (the
 * kernel then flags QSLBM_ETIMEOUT).  This call runs that routine in one warp
 * on a counter in device memory: counter_set = 0 leaves the counter at 0, so
 * the wait can never be satisfied and must give up after limit_s seconds;
 * counter_set = 1 satisfies it at once.
 *   limit_s    the wait's limit, 0 < limit_s <= 2 seconds
 *   gave_up    out: 1 if the wait gave up, 0 if it was satisfied
 *   waited_s   out: time spent in the wait, by the GPU's global timer
 * Synchronous (default stream); allocates and frees 16 bytes of device memory.
 * Errors: QSLBM_EINVAL (NULL output, limit out of range), QSLBM_ECUDA. */
int qslbm_check_bounded_wait(double limit_s, int32_t counter_set, int32_t* gave_up, double* waited_s);

/* ------------------------------------------------------------------ batches
 * Many independent instances (3-D, one precision) advanced together: every
 * phase of a flow step is one fused launch over all instances' work, and the
 * steps are replayed from CUDA graphs (one of many steps, one of a single
 * step for the remainder).  The magnetic sub-iteration (Sec. V.G, with the IB
 * on b after each sweep, Sec. V.D) takes one of two routes per instance:
 *  - resident groups (FP32): an instance with a straight wall (the same ring
 *    on every plane) and planes of at most 5120 nodes runs all its N_mag
 *    sweeps in one cooperative launch shared by every such instance; each CTA
 *    holds a group of whole planes in shared memory, and the groups of an
 *    instance exchange their end planes through global memory with bounded
 *    waits (a wait that times out is reported as QSLBM_ETIMEOUT by
 *    qslbm_batch_handle and the server).  Instances are admitted smallest
 *    first while their groups fit co-resident on the device;
 *  - marching: every other instance (and any created with sweep_kernel =
 *    QSLBM_SWEEP_SPLIT) takes one persistent z-marching launch per sweep over
 *    the instances with N_mag > s, then one IB launch; the sweep's launch
 *    mode, tile shape and persistent grid are chosen by timing candidates on
 *    the batch when it is first built with such a member.
 * Each instance follows the same arithmetic as a handle created alone with
 * QSLBM_SWEEP_SPLIT (the same expressions in the same order). */
typedef struct qslbm_batch qslbm_batch;

typedef struct qslbm_batch_info_t {
    int32_t count, max_n_mag;
    int32_t sweep_threads, sweep_grid;  /* tuned marching launch: threads = 32 x the tile's rows
                                           (4, 8 or 16); grid 0 = one block per work item  */
    int32_t launches_per_step;
    int64_t nodes, node_sweeps_per_step, device_bytes, steps;
    double tune_us[32];                 /* microseconds per sweep of each candidate tried, in
                                           the order ordinary / programmatic launches x rows
                                           4, 8, 16 x grid 1, 2, 4, 8 CTAs per SM, one per
                                           item (0 when not timed)                          */
    int32_t resident_instances;         /* members whose sweeps run in the resident group kernel */
    int32_t resident_groups;            /* its CTAs (groups of whole planes)               */
    int32_t graph_steps;                /* flow steps per captured graph chunk             */
    int32_t march_chunk;                /* z planes per work item of the marching sweep    */
    int32_t sweep_pdl;                  /* 1: the marching sweep and its IB pass are launched
                                           with programmatic stream serialization           */
} qslbm_batch_info_t;

/* Create count instances from params[0..count-1] (their stream fields are
 * ignored; work goes to `stream`, NULL = a stream the batch creates).  All
 * must have dim = 3 and one precision (else QSLBM_EINVAL).  Errors as for
 * qslbm_create. */
int qslbm_batch_create(const qslbm_params* params, int32_t count, void* stream, qslbm_batch** out);

/* Queue nsteps flow steps of every instance (asynchronous; device errors
 * surface at qslbm_batch_handle).  Errors: QSLBM_EINVAL (NULL batch, negative
 * nsteps), QSLBM_ECUDA (a graph launch failed). */
int qslbm_batch_step(qslbm_batch* b, int64_t nsteps);

/* The handle of instance i (in creation order), after synchronising the
 * batch's stream: use it with qslbm_observables, qslbm_get_state,
 * qslbm_set_state and qslbm_get_units; stepping it on its own would leave the
 * batch out of step.  The batch owns it.  Errors: QSLBM_EINVAL (NULL
 * argument, i out of range), QSLBM_ECUDA, QSLBM_ETIMEOUT (a resident group's
 * neighbour wait gave up; the counters are reset). */
int qslbm_batch_handle(qslbm_batch* b, int32_t i, qslbm_handle** out);

/* Sizes, tuned launch and timing of the batch.  Errors: QSLBM_EINVAL (NULL). */
int qslbm_batch_info(const qslbm_batch* b, qslbm_batch_info_t* info);

/* Release every instance and the batch.  Errors: QSLBM_EINVAL (NULL). */
int qslbm_batch_destroy(qslbm_batch* b);

/* ------------------------------------------------------------------ serving
 * A request loop with continuous batching.  Requests (a problem and a stop
 * tolerance on the steady residual) may be submitted from any thread; each
 * qslbm_server_run admits queued requests whose device memory fits the
 * budget (in arrival order, or smallest first), advances every running
 * request by chunk_steps flow steps in the batched launches, and retires
 * requests whose FP64 steady residual fell below their tolerance (status
 * QSLBM_OK), that reached max_steps (QSLBM_ETIMEOUT), or whose fields went
 * non-finite (QSLBM_EUNSTABLE).  A request larger than the whole budget
 * finishes at once with QSLBM_EBUDGET.  Times are seconds on the server's
 * monotonic clock. */
typedef struct qslbm_server qslbm_server;

#define QSLBM_ADMIT_FIFO 0     /* queued requests in arrival order (first fit)          */
#define QSLBM_ADMIT_SMALLEST 1 /* fewest nodes first (ties in arrival order), first fit;
                                  in FP32, while any request runs, admission stops at the
                                  first request that would not fit beside the running
                                  ones in the batch's resident group kernel (so that the
                                  running requests keep its one launch per step)       */

typedef struct qslbm_server_config {
    int64_t hbm_budget_bytes; /* device memory the running requests may hold  */
    int32_t chunk_steps;      /* flow steps between residual checks            */
    int32_t max_running;      /* 0 = limited by the budget only                */
    int32_t precision;        /* QSLBM_FP32 | QSLBM_FP64 for every request     */
    void* stream;             /* cudaStream_t or NULL (the server creates one) */
    int32_t admit;            /* QSLBM_ADMIT_FIFO (0) | QSLBM_ADMIT_SMALLEST   */
} qslbm_server_config;

typedef struct qslbm_result {
    int64_t id;
    int32_t status;           /* QSLBM_OK, QSLBM_ETIMEOUT, QSLBM_EUNSTABLE, ... */
    int64_t steps;            /* flow steps taken                               */
    int64_t nodes;
    double residual;          /* last steady residual                           */
    double t_submit, t_admit, t_done;
    qslbm_obs obs;            /* diagnostics at retirement                      */
} qslbm_result;

typedef struct qslbm_server_stats_t {
    int32_t running, pending, sweep_threads, sweep_grid;
    int64_t chunks, rebuilds, steps, node_steps, device_bytes;
} qslbm_server_stats_t;

/* Errors: QSLBM_EINVAL (NULL argument, chunk_steps or hbm_budget_bytes not
 * positive, unknown precision or admission order), QSLBM_ENOMEM, QSLBM_ECUDA. */
int qslbm_server_create(const qslbm_server_config* cfg, qslbm_server** out);
/* Queue a request (dim 3; precision and stream are the server's).  keep_fields
 * keeps the finished fields on the device for qslbm_server_fields until
 * qslbm_server_release.  Thread-safe.  Its parameters are checked when it is
 * admitted (a refusal becomes its result's status).  Errors: QSLBM_EINVAL
 * (NULL argument, tol or max_steps not positive, dim != 3). */
int qslbm_server_submit(qslbm_server* s, const qslbm_params* p, double tol, int64_t max_steps, int32_t keep_fields,
                        int64_t* id);
/* One admission + chunk + retirement round (blocks until the chunk is done).
 * Errors: QSLBM_EINVAL (NULL server), QSLBM_ECUDA, QSLBM_ETIMEOUT (a resident
 * group's neighbour wait gave up), QSLBM_ENOMEM. */
int qslbm_server_run(qslbm_server* s, int32_t* n_running, int32_t* n_pending);
/* Move up to max finished results into out; *n = how many.  Errors:
 * QSLBM_EINVAL (NULL server or n, max < 0, NULL out with max > 0). */
int qslbm_server_poll(qslbm_server* s, qslbm_result* out, int32_t max, int32_t* n);
/* Fields of a finished request submitted with keep_fields (binary64 host
 * arrays as in qslbm_get_state); QSLBM_ENOTFOUND otherwise.  The first call
 * for a request allocates its host-copy staging buffer (56 B per node), which
 * counts against the HBM budget with the rest of its memory. */
int qslbm_server_fields(qslbm_server* s, int64_t id, double* rho, double* u, double* b);
/* Free a kept request's device memory and return it to the budget;
 * QSLBM_ENOTFOUND for an id that is not kept. */
int qslbm_server_release(qslbm_server* s, int64_t id);
/* Counters; device_bytes is the device memory the admitted and kept requests
 * hold, the figure admission compares with the budget. */
int qslbm_server_stats(const qslbm_server* s, qslbm_server_stats_t* st);
/* Release every running and kept request and the server (synchronises its
 * stream first).  Errors: QSLBM_EINVAL (NULL). */
int qslbm_server_destroy(qslbm_server* s);

/* Static string for a code, and the reason for the calling thread's last
 * refusal or failed CUDA call (empty if none). */
const char* qslbm_strerror(int code);
const char* qslbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QSLBM_H */
