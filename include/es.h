/*
 * es.h -- C ABI of libes, a single-GPU (sm_103a) implementation of the
 * Eulerian grid work of one coupled electrophoresis time step of
 * Bartuschat & Ruede, arXiv 1708.08741 (Algorithm 1, Sec. 5.7).
 *
 * One time step is the call sequence
 *     es_map_particles      particle -> grid mapping, PDF reconstruction,
 *                           potential stencil/RHS assembly
 *     es_potential_solve    multigrid solve of the Debye-Hueckel equation,
 *                           EDL field and electric body force
 *     es_lbm_step           fused TRT stream-collide with moving bounce-back
 *     es_forces             momentum-exchange force/torque plus q E_ext
 *     es_advance            rigid-body update
 * or es_step, which issues all five.
 *
 * Conventions for every function:
 *  - Return value: ES_OK (0) or a negative ES_E* status.  A failing call
 *    leaves a message retrievable with es_last_error().  No C++ exception
 *    crosses this boundary.
 *  - Units are lattice units: dx = dt = rho_0 = 1 (Sec. 4.4); eps is the
 *    fluid permittivity in those units.
 *  - Grid layout: cell (i, j, k) has linear index i + nx (j + ny k) (x
 *    fastest) and centre (i + 1/2, j + 1/2, k + 1/2) (Sec. 4.3, Eq.
 *    FineLattice with 0-based indices).
 *  - All work is issued on the CUDA stream given to es_create, in order, and
 *    does not wait for the GPU, except where a function says it does.
 *    Asynchronous kernel errors and device-side statuses (overlapping
 *    particles) surface at the next call that synchronises.
 *  - The context owns every device buffer it uses; callers' arrays are
 *    copied and never retained.
 *  - A context is not thread safe: one host thread at a time.
 */
#ifndef ES_H
#define ES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ES_OK 0
#define ES_EINVAL (-1)         /* invalid argument or parameter set        */
#define ES_ENOMEM (-2)         /* device or host allocation failed         */
#define ES_ECUDA (-3)          /* a CUDA runtime call or kernel failed      */
#define ES_ENOTCONVERGED (-4)  /* solver hit max_cycles above tolerance     */
#define ES_ENAN (-5)           /* residual norm is NaN or infinite          */
#define ES_EOVERLAP (-6)       /* two particles claim a cell, or a sphere cuts a wall */
#define ES_ETIMEOUT (-7)       /* a kernel's bounded wait for its asynchronous copies ran out */

/* arithmetic forms */
#define ES_FP64 0    /* everything in double precision                           */
#define ES_MIXED32 1 /* PDFs stored as FP32 deviations f_q - w_q, FP32 collision,
                        FP32 multigrid cycles inside a defect correction whose
                        potential and residual are float-float (two floats,
                        about 48 significant bits, evaluated on the FP32 pipe),
                        force/torque from FP32 link terms with the constant
                        2 w_q c_q part summed exactly (es_forces), FP64
                        rigid-body update                                     */
#define ES_MIXED16 2 /* as ES_MIXED32, with the PDFs stored as FP16 relative
                        deviations (f_q - w_q) / w_q                           */

/* particle electric boundary conditions (Sec. 5.5) */
#define ES_KIND_ZETA 0   /* prescribed zeta potential: Dirichlet             */
#define ES_KIND_CHARGE 1 /* prescribed total surface charge q: Neumann       */

/* potential condition on a non-periodic domain face (Sec. 5.4) */
#define ES_POT_ZERO_FLUX 0
#define ES_POT_DIRICHLET 1

/* fields for es_get_field / es_set_field; all exchanged as double except
 * OWNER (int32) and FLAGS (uint8).  Multi-component fields are component
 * major: component c of cell i at [c * N + i].                             */
#define ES_FIELD_PSI 0      /* N: EDL potential psi (boundary cells: zeta or 0) */
#define ES_FIELD_RHO 1      /* N: density of the stored state                   */
#define ES_FIELD_U 2        /* 3N: velocity u = sum c f - f_b/2 of the stored state
                               (the modified velocity of Eq. modified_velocity) */
#define ES_FIELD_FB 3       /* 3N: electric body force density f_b (Sec. 5.6)  */
#define ES_FIELD_PDF 4      /* 19N: populations the next es_lbm_step pulls from,
                               in the direction order of es_lattice            */
#define ES_FIELD_OWNER 5    /* N int32: particle index of an obstacle cell, -1 fluid */
#define ES_FIELD_FLAGS 6    /* N uint8: bit 0 obstacle cell, bit 1 fluid cell with a
                               D3Q19 neighbour that is an obstacle or beyond a wall */
#define ES_FIELD_PDF_LAST 7 /* 19N: populations the last es_lbm_step pulled from */

typedef struct {
    int dims[3];        /* cells per axis; each a multiple of 2^(levels-1)          */
    int periodic[3];    /* 1: periodic axis; 0: walls half-way outside the first
                           and last layer (LBM: wall_slip) with pot_bc on both faces */
    int pot_bc[6];      /* faces x-lo, x-hi, y-lo, y-hi, z-lo, z-hi of non-periodic axes */
    double pot_val[6];  /* Dirichlet values of those faces                          */
    double tau;         /* LBM relaxation time, nu = (tau - 1/2)/3 (Eq. kinVisc); > 1/2 */
    double kappa;       /* Debye-Hueckel parameter 1/lambda_D (Eq. DebyHuckApproxPot) */
    double eps;         /* fluid permittivity (Eq. ChrgDensDHA)                   */
    double E_ext[3];    /* applied field (Sec. 5.6)                               */
    double accel[3];    /* additional uniform body force density on the fluid      */
    double rho_p_ratio; /* particle / fluid density (1.195 in Sec. 6.1)           */
    int precision;      /* ES_FP64, ES_MIXED32 or ES_MIXED16                      */
    int levels;         /* multigrid levels, 1..12                                */
    int nu1, nu2;       /* pre- and post-smoothing red-black sweeps per level     */
    int coarse_sweeps;  /* red-black sweeps on the coarsest level                 */
    double omega;       /* smoother relaxation (1: Gauss-Seidel; the paper's SOR uses 1.7) */
    double res_rf;      /* residual reduction factor w.r.t. the first solve (Sec. 5.3) */
    int max_cycles;     /* cycle cap per es_potential_solve                        */
    int smoother;       /* ES_SMOOTH_TWO_PASS (0, default) or ES_SMOOTH_FUSED: how a
                           red-black sweep is executed; both compute the same sweep */
    int mg_storage;     /* ES_MG_NATIVE (0, default) or ES_MG_FP16: storage of the
                           finest level's multigrid correction (see below)        */
    int wall_slip[6];   /* LBM condition per face of a non-periodic axis (order of
                           pot_bc): 0 no-slip (resting bounce-back), 1 free-slip
                           (specular reflection; Sec. 4.1 uses both)             */
    double phi_t;       /* thermal voltage k_B T / (z e).  0 (default): the
                           Debye-Hueckel equation.  > 0: the symmetric nonlinear
                           Poisson-Boltzmann equation (Eq. SPBE),
                           -lap psi + kappa^2 phi_t sinh(psi / phi_t) = 0, solved by
                           Newton steps whose linear systems get coarse_sweeps
                           red-black SOR sweeps on the stencil re-linearised about
                           the current psi (Sec. 5.3); needs ES_FP64, levels == 1.
                           The charge density becomes -eps kappa^2 phi_t
                           sinh(psi / phi_t).                                      */
    int fine_layout;    /* ES_LAYOUT_AUTO (0, default) or ES_LAYOUT_NATURAL: storage of
                           the finest level's multigrid correction and right-hand
                           side (see below); both give the same iteration          */
    int near_list_cells; /* multigrid levels (dims[0] % 4 == 0 on the level) with more
                           cells than this smooth their near-boundary cells in
                           separate passes over per-colour cell lists, the others
                           inside the smoothing kernel; the same sweep either way.
                           0 selects the default ES_NEAR_LIST_CELLS; < 0 is
                           ES_EINVAL.  (The colour-split finest level always uses
                           the lists.)                                             */
    int sweep_staging;  /* colour-split finest level, rows of up to 512 cells:
                           ES_STAGE_REGISTERS (0, default) each thread loads its
                           neighbours' rows into registers, marching through z
                           planes; ES_STAGE_BULK a block stages the other
                           colour's rows and its right-hand side in shared memory
                           with bulk asynchronous copies (cp.async.bulk with
                           mbarrier completion), three planes ahead.  The same
                           sweep either way.                                    */
    int lbm_block[2];   /* thread-block shape of the stream-collide: cells along x
                           (a multiple of 32 in 32..256) by rows along y, at most
                           256 threads; {0, 0} selects {32, 4}.  The same result
                           for every shape (the autotuner times them).         */
    int fast_update_cells; /* reduced forms with the colour-split finest level: on
                           grids of at least this many cells a tolerance-driven
                           solve that starts within 5000 x tol updates the
                           residual after a correction in FP32 as r - A e (Sec.
                           5.3 defect correction, see es_potential_solve).  0
                           selects the default ES_FAST_UPDATE_CELLS; < 0 is
                           ES_EINVAL.                                              */
} es_params;

/* Defaults of near_list_cells and fast_update_cells (2^21 cells): below this
   size the separate passes cost more in launches and host round trips than
   they save. */
#define ES_NEAR_LIST_CELLS (1 << 21)
#define ES_FAST_UPDATE_CELLS (1 << 21)

/* Execution of one red-black Gauss-Seidel sweep (same arithmetic either way):
   TWO_PASS runs one in-place pass per colour; FUSED runs red and black in
   one pass over the level (out of place). */
#define ES_SMOOTH_TWO_PASS 0
#define ES_SMOOTH_FUSED 1

/* Storage of the finest level's correction e inside the V-cycle.  NATIVE:
   the solver's arithmetic type (double in ES_FP64, float otherwise).  FP16
   (reduced precisions only; two-pass smoother; dims[0] % 4 == 0; levels >=
   2): e is held as FP16 values s * e with s = sqrt(N) / ||r|| fixed for the
   V-cycles of one correction, and every operation still computes in float.
   The outer defect correction forms the residual of psi in float-float, so
   the rounding of the stored correction only slows the outer iteration; it
   does not move the converged potential. */
#define ES_MG_NATIVE 0
#define ES_MG_FP16 1

/* AUTO: in the reduced precisions, with the two-pass smoother, native
   correction storage, levels >= 2 and dims[0] % 8 == 0, the finest level's
   e and rhs are stored colour-split (all cells of colour (x+y+z) % 2 = 0,
   then all of colour 1, each in natural order), so that a red or black half
   sweep streams only its own colour; otherwise, and with NATURAL, cell
   x + nx (y + ny z) is element x + nx (y + ny z). */
#define ES_LAYOUT_AUTO 0
#define ES_LAYOUT_NATURAL 1

/* How the finest level's half sweep brings in its operands (sweep_staging). */
#define ES_STAGE_REGISTERS 0
#define ES_STAGE_BULK 1

typedef struct {
    double x[3]; /* centre                  */
    double v[3]; /* translational velocity  */
    double w[3]; /* angular velocity        */
    double R;    /* radius                  */
    int kind;    /* ES_KIND_ZETA or ES_KIND_CHARGE */
    double zeta; /* surface potential (ES_KIND_ZETA)  */
    double q;    /* total charge (ES_KIND_CHARGE)      */
} es_particle;

typedef struct {
    int cycles;       /* V-cycles applied                                  */
    double r_initial; /* residual L2 norm before the first cycle          */
    double r_final;   /* residual L2 norm after the last cycle            */
    double tol;       /* absolute tolerance res_rf * (norm at the first solve) */
} es_solve_info;

typedef struct es_ctx es_ctx;

/* Device allocator hooks: alloc returns device memory of at least `bytes`
 * (256-byte aligned) or NULL; free releases it.  `user` is passed through. */
typedef void* (*es_alloc_fn)(size_t bytes, void* user);
typedef void (*es_free_fn)(void* ptr, void* user);

/* Creates a simulation: validates the parameters (the PhysicalCheck role of
 * Sec. 5.1; ES_EINVAL on violation), allocates all device state with
 * cudaMalloc, sets the fluid at rest (f_q = w_q), psi = 0, copies the n
 * particles (host array, n >= 0) and binds the CUDA stream `stream`
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the
 * context, or NULL on failure.  Synchronises once at the end.            */
int es_create(const es_params* params, const es_particle* particles, int n, void* stream,
              es_ctx** out);

/* As es_create, with all device memory taken from alloc/free (for example a
 * framework's caching allocator).  alloc == NULL selects cudaMalloc.      */
int es_create_with_allocator(const es_params* params, const es_particle* particles, int n,
                             void* stream, es_alloc_fn alloc, es_free_fn free_fn, void* user,
                             es_ctx** out);

/* Synchronises the stream and releases everything; ctx may be NULL. */
int es_destroy(es_ctx* ctx);

/* Algorithm 1, "set electric BCs of particles" and "set velocity BCs of
 * particles" (Sec. 5.5, Sec. 4.2): maps every sphere onto the lattice (a
 * cell belongs to a sphere iff its centre lies inside), reconstructs the
 * PDFs of cells uncovered since the last mapping as f^eq(rho_0, u_s) with
 * the surface velocity at that mapping, writes the boundary values into psi
 * and assembles the quasi-constant stencil: boundary flags per multigrid
 * level and, per charged sphere, sigma = q / (number of its fluid faces).
 * Work is limited to each sphere's bounding box.  Overlap or a sphere that
 * cuts a wall is reported as ES_EOVERLAP by the next synchronising call. */
int es_map_particles(es_ctx* ctx);

/* Algorithm 1, "while residual >= tol: iterate" and the coupling block
 * (Sec. 5.3, Sec. 5.6): r = b - A psi with the 7-point finite-volume
 * stencil of Sec. 4.3 and the boundary treatment of Sec. 5.4 (FP64, or
 * float-float in the reduced forms); tol = res_rf * ||r|| of the first
 * solve of the run; while ||r|| >= tol, psi += V-cycle(r) (reduced forms:
 * several warm-started FP32 V-cycles per correction, and, on grids of at
 * least fast_update_cells cells starting within 5000 x tol, the residual
 * after a correction updated in FP32 as r - A e, re-formed in float-float if
 * that is not yet below tol).  forced_cycles >= 0 applies exactly that many cycles
 * and skips the tolerance test.  Then computes the EDL field grad psi
 * (Eq. ElPotGradComp), the charge density -kappa^2 eps psi (Eq.
 * ChrgDensDHA) and the body force f_b = rho_e (E_ext - grad psi).
 * Synchronises once per cycle to read the residual norm.  info may be
 * NULL.  Returns ES_ENOTCONVERGED after max_cycles, ES_ENAN on a NaN norm,
 * ES_EOVERLAP if the preceding mapping found overlapping spheres.        */
int es_potential_solve(es_ctx* ctx, int forced_cycles, es_solve_info* info);

/* Algorithm 1, "perform fused stream-collide step" (Sec. 4.1, Sec. 4.2):
 * one pull stream-collide sweep over all fluid cells with the TRT operator
 * (Eq. LBMcollideStep), incompressible equilibrium (Eq. EqPDF_TRT), Luo
 * forcing with the modified velocity (Eq. LBE_forcetermLuo, Eq.
 * modified_velocity) and velocity bounce-back at moving sphere cells (Eq.
 * LBMMovWall), resting bounce-back at no-slip walls and specular
 * reflection at free-slip walls (wall_slip).                              */
int es_lbm_step(es_ctx* ctx);

/* es_lbm_step for n resident runs at once (the paper has no counterpart:
 * serving many small independent runs).  One persistent launch steps every
 * run's stream-collide from a work table of the runs' fields and parameters
 * (tiles of 32 cells x 4 rows, any mix of grid sizes), each cell exactly as
 * es_lbm_step computes it, so a run gives the same bits alone and batched.
 * The launch goes on ctxs[0]'s stream after the work already issued on every
 * context's stream, and each context's later work waits for it (CUDA
 * events), so the contexts stay stream-ordered.  1 <= n <= ES_LBM_BATCH_MAX;
 * all contexts on one device, of one precision, without free-slip faces, no
 * context twice (ES_EINVAL otherwise). */
#define ES_LBM_BATCH_MAX 32
int es_lbm_step_batch(es_ctx* const* ctxs, int n);

/* Algorithm 1, "apply hydrodynamic force to particles" (Sec. 4.2, Eq.
 * LBMhydrodynForce, torque by the same sum with (x_s - X) x dF) plus the
 * electrostatic force F_C = q E_ext (Sec. 5.6), summed in a fixed order
 * (deterministic): in FP64, or in the reduced forms from FP32 link terms
 * (float-float block sums) plus the exactly summed constant part.  Uses the populations bounced by the last
 * es_lbm_step.  F and T receive n x 3 doubles each (particle major); either
 * may be NULL.  on_device != 0: F/T are device pointers (no
 * synchronisation); 0: host pointers (synchronises).  The sums are also
 * kept for es_advance.                                                    */
int es_forces(es_ctx* ctx, double* F, double* T, int on_device);

/* Algorithm 1, "pe moves particles": semi-implicit Euler with dt = 1,
 * V += F/m, X += V (wrapped on periodic axes), Omega += T/I with
 * m = rho_p_ratio (4/3) pi R^3 and I = (2/5) m R^2, using the force and
 * torque of the last es_forces / es_set_forces.                          */
int es_advance(es_ctx* ctx);

/* One whole time step: es_map_particles, es_potential_solve, es_lbm_step,
 * es_forces (kept on the device), es_advance.                             */
int es_step(es_ctx* ctx, int forced_cycles, es_solve_info* info);

/* Copies a field (ES_FIELD_*) to dst, converting PDFs to plain FP64 values.
 * bytes must equal the field size; on_device selects device or host dst.
 * Synchronises.                                                           */
int es_get_field(es_ctx* ctx, int which, void* dst, size_t bytes, int on_device);

/* Values of a field at n selected cells (linear indices idx, host array)
 * into the host array out, component major: out[k * n + i] is component k
 * of cell idx[i].  Fields as for es_get_field (OWNER and FLAGS converted to
 * double); 1 <= n <= 65536; indices must lie in [0, N).  Synchronises.   */
int es_gather(es_ctx* ctx, int which, const int64_t* idx, int n, double* out);

/* es_gather without any device allocation.  The paper has no counterpart:
 * this is a library convenience.  es_gather allocates its device staging
 * buffer on first use; callers that must not allocate device memory when
 * they read values back -- a real-time loop that cannot wait on an
 * allocator, or an application that hands out all device memory up front --
 * use this variant, which stages through a fixed array in the library's
 * device memory instead and calls no device allocator (no cudaMalloc,
 * cudaFree or allocator hook).
 *  - Same arguments, checks, field conversions and output layout as
 *    es_gather; 1 <= n <= ES_GATHER_NOALLOC_MAX (4096), larger n returns
 *    ES_EINVAL.
 *  - The context's device must be the current device (ES_EINVAL otherwise).
 *  - The array (640 KiB) is held by every GPU that loads the library until
 *    the process exits.  The first call on a device looks up the array's
 *    address on that device; make that first call before any stream
 *    capture.
 *  - All calls share the array and it keeps the last call's contents; no
 *    part of it needs to start at zero.  Calls whose GPU work overlaps (two
 *    streams or two host threads at once) race on it: serialise them.
 *  - Copies the indices from the caller's (pageable) host array and
 *    synchronises the context's stream, like es_gather, so that stream
 *    must not be one that is being captured into a graph.                 */
#define ES_GATHER_NOALLOC_MAX 4096
int es_gather_noalloc(es_ctx* ctx, int which, const int64_t* idx, int n, double* out);

/* Overwrites ES_FIELD_PSI, ES_FIELD_FB or ES_FIELD_PDF from doubles.      */
int es_set_field(es_ctx* ctx, int which, const void* src, size_t bytes, int on_device);

/* Host copies of the particle state (n must equal the context's count).
   es_set_particles changes positions, velocities, spins, zeta and charge;
   a sphere's radius and kind are fixed after creation (ES_EINVAL).  It
   copies src into a pinned staging buffer and returns without waiting for
   the device: src may be reused at once, and the new state is in place for
   every later call on the context's stream.  The surface charge density
   stays as the last mapping found it until the next es_map_particles.
   es_get_particles synchronises the context's stream. */
int es_get_particles(es_ctx* ctx, es_particle* dst, int n);
int es_set_particles(es_ctx* ctx, const es_particle* src, int n);

/* Overrides the kept force and torque (host arrays, n x 3) for es_advance. */
int es_set_forces(es_ctx* ctx, const double* F, const double* T, int n);

/* Waits for the stream and reports pending device statuses. */
int es_synchronize(es_ctx* ctx);

/* The library's own D3Q19 velocity (19 x 3 ints) and weight tables. */
int es_lattice(int* c57, double* w19);

/* ---- Per-kernel device time (instrumentation; the paper has no counterpart) ----
   Between es_profile_start and es_profile_stop the library brackets each
   launch of its grid-sized kernels (stream-collide, body force, smoothers,
   restriction, prolongation, coarse solve, outer residual, correction) with
   a pair of CUDA events on the context's stream.  es_profile_stop
   synchronises the stream and writes one record per kernel and multigrid
   level: launches, summed device time, and summed algorithmic bytes (the
   least traffic the launches' work needs, every input read once and every
   output written once; the formulas are stated beside each launch).  The
   events add two stream commands per bracketed launch and change no
   result.  es_profile_stop returns ES_EINVAL when profiling was not started;
   *n receives the number of records (at most max are written). */
typedef struct {
    char name[32];   /* kernel                                       */
    int level;       /* multigrid level; -1 for a fine-grid kernel   */
    int launches;
    double ms;       /* summed device time of the launches           */
    double bytes;    /* summed algorithmic bytes of the launches     */
} es_kernel_time;

int es_profile_start(es_ctx* ctx);
int es_profile_stop(es_ctx* ctx, es_kernel_time* out, int max, int* n);

/* Measured fused multiply-add throughput of the current device in GFLOP/s
 * (2 flops per FMA), the denominator of the arithmetic roofline of kernels
 * bound by their FP64 (precision ES_FP64) or FP32 (ES_MIXED32) pipe; the
 * paper has no counterpart (instrumentation).  Runs register-resident FMA
 * chains on every SM for a few milliseconds, timed with CUDA events on a
 * private stream; allocates and frees a small device buffer.  Synchronises
 * that stream.  ES_EINVAL for another precision or a NULL gflops, ES_ECUDA
 * if a CUDA call fails. */
int es_alu_peak(int precision, double* gflops);

/* Number of CUDA kernels this context has launched so far (telemetry). */
uint64_t es_kernel_launches(const es_ctx* ctx);

/* Device bytes a context with these parameters and n particles will hold. */
size_t es_device_bytes(const es_params* params, int n);

/* Message of the last failure on ctx (or of the last failed es_create when
 * ctx is NULL); never NULL.                                               */
const char* es_last_error(const es_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ES_H */
