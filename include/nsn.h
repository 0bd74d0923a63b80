/*
 * nsn.h -- C ABI of the GB300 (sm_103a) non-smooth Newton time stepper.
 *
 * Implements one time step of Algorithm 1 of Macklin, Erleben, Mueller,
 * Mueller, "Non-Smooth Newton Methods for Deformable Multi-Body Dynamics"
 * (ACM TOG 38(5), 2019) on one GPU:
 *   - per-row evaluation of Fischer-Burmeister contact rows with the
 *     effective-mass complementarity preconditioner (Sec. 4.2, 7, App. A.1),
 *     smooth isotropic friction rows with compliance W (Sec. 4.3, App. A.2),
 *     revolute joint rows (Sec. 3.1-3.2) and stable Neo-Hookean compliance
 *     rows (Sec. 9.1-9.2.2, App. B), plus the diagonal geometric-stiffness
 *     shift of particle masses (Sec. 8.3);
 *   - a matrix-free, Jacobi-preconditioned conjugate-residual solve (Sec. 8.2)
 *     of the Schur system [J H~^-1 J^T + C + eps I] dl = (1/h)(J H~^-1 g - h)
 *     (Eq. schur_system, Sec. 8.4), then du = H~^-1 (h J^T dl - g) and the
 *     damped update of Sec. 6.2 / 8.1.
 *
 * Conventions (shared with the input generators):
 *   - SI units; gravity and h in nsn_config.  Quaternions (w, x, y, z),
 *     angular velocity in the world frame (kinematic map G of Sec. 9.4).
 *   - Bodies receive ids 0..nb-1 in the order added.  -1 denotes the static
 *     world in constraint records.
 *   - Rows: contact c owns rows 3c (normal), 3c+1, 3c+2 (friction along the
 *     orthonormal basis of Duff et al. 2017 built from n); then joint j (in
 *     the order added, revolute and prismatic alike) owns 5 rows; then
 *     Neo-Hookean tet k owns 3 rows (principal stretches s1 >= s2 >= |s3|);
 *     then linear tet l owns 6 rows.  Multipliers are forces (N); impulses
 *     are h * lambda.
 *   - Revolute rows: 3 anchor-coincidence rows, 2 rows keeping a's axis
 *     orthogonal to the basis t1, t2 of b's axis (Sec. 3.1; the paper gives no
 *     joint functions).  Prismatic rows (the Fetch scenes of Sec. 10): t_k .
 *     (p_a - p_b) for k = 1, 2 (a's anchor stays on the line through b's
 *     anchor along b's axis), a_w . t_1, a_w . t_2, and n_a . t_2 with n_a the
 *     first basis vector of a's axis (no twist); both axes are normalised.
 *   - Linear tet rows (Sec. 9.2.1): the small strain of F = D_s D_m^-1 in the
 *     eigenbasis of the isotropic stiffness: (e_xx + e_yy + e_zz) / sqrt(3),
 *     (e_xx - e_yy) / sqrt(2), (e_xx + e_yy - 2 e_zz) / sqrt(6), and the
 *     engineering shears 2 e_yz, 2 e_xz, 2 e_xy; the paper's strain vector
 *     s rotated by a constant orthogonal matrix, which makes the compliance
 *     (V_e K_e)^-1 diagonal (1 / (V_e (3 lambda + 2 mu)), 1 / (2 V_e mu) twice,
 *     1 / (V_e mu) three times).
 *
 * Ownership: every host array passed in is copied; the caller keeps it.  All
 * device memory belongs to the context and is released by nsn_destroy.  The
 * *_device entry points take device pointers that must stay valid for the
 * call and be ordered on the context's stream.  A context is used from one
 * host thread at a time.
 *
 * Errors: every call returns an nsn_status; nothing aborts or throws across
 * the ABI.  nsn_last_error() returns a message for the last failure.
 */
#ifndef NSN_H
#define NSN_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsn_ctx nsn_ctx;

typedef enum {
  NSN_OK = 0,
  NSN_ERR_INVALID_ARG = 1,
  NSN_ERR_OUT_OF_MEMORY = 2,
  NSN_ERR_CUDA = 3,
  NSN_ERR_NOT_CONVERGED = 4,
  NSN_ERR_TIMEOUT = 5,
  NSN_ERR_BAD_STATE = 6,
  NSN_ERR_NONFINITE = 7
} nsn_status;

enum { NSN_RIGID = 0, NSN_PARTICLE = 1 };
enum { NSN_CONTACT = 0, NSN_REVOLUTE = 1, NSN_TET_NH = 2, NSN_PRISMATIC = 3, NSN_TET_LINEAR = 4 };
enum { NSN_NCP_FB = 0, NSN_NCP_MIN = 1 };
enum { NSN_R_NONE = 0, NSN_R_H2 = 1, NSN_R_EFFMASS = 2 };
enum { NSN_GS_OFF = 0, NSN_GS_PARTICLES = 1 };
enum { NSN_FP32 = 0, NSN_FP64 = 1 };

typedef struct {
  double h;               /* time step (Sec. 5) */
  double gravity[3];
  int32_t newton_iters;   /* N of Algorithm 1; cap when tol_rel > 0 */
  int32_t cr_iters;       /* M of Algorithm 1; cap when cr_tol_mode = 1 */
  double damping;         /* t of Sec. 8.1 (0.75 in the paper) */
  double eps;             /* identity shift of Sec. 8.4 (1e-6 in the paper) */
  double tol_rel;         /* stop Newton when merit <= tol_rel * merit(u=0, l=0); 0 = fixed */
  int32_t cr_tol_mode;    /* 1: stop CR at ||r||_P <= min(0.1, merit/merit0) ||r0||_P */
  int32_t ncp;            /* NSN_NCP_FB (paper default) or NSN_NCP_MIN */
  int32_t rscale;         /* complementarity preconditioner, Sec. 7 */
  int32_t geom_stiffness; /* NSN_GS_PARTICLES: Sec. 8.3 on particle DOFs */
  int32_t precision;      /* NSN_FP32 bulk arithmetic or NSN_FP64 throughout;
                             CR scalars and the merit are FP64 in both */
  int32_t use_graph;      /* 1: capture the step as one CUDA graph and replay it */
  int32_t cone_project;   /* 1: after each damped update (Sec. 8.1) set lambda_n :=
                             max(lambda_n, 0) and scale lambda_f into |lambda_f| <=
                             mu lambda_n.  Not in the paper (0 = the printed method):
                             on separating sliding contacts the damped update leaves
                             lambda_n > 0, the lagged W of Sec. 4.3 grows like
                             1/lambda_n and |lambda_f|/(mu lambda_n) grows every
                             iteration.  Solutions of the NCPs already lie in this set. */
  int32_t island_stop;    /* 1: islands (connected components of the bodies through
                             constraints, the static world excluded) are solved side by
                             side: each has its own merit, its own zero-iterate merit
                             for tol_rel, its own CR scalars (A of Eq. schur_system is
                             block diagonal by island, so this is CR on each island's
                             system alone) and its own warm-start acceptance; an island
                             that reaches tol_rel keeps its u and lambda, and the step
                             ends when all have stopped or after newton_iters */
  int32_t cr_resident;    /* island mode, 1 (default): islands of rigid bodies, contacts
                             and joints with at most res_max_rows rows run their CR of a
                             Newton iteration inside one thread block from shared memory
                             (the same recurrence and stop rules; HBM read once per
                             Newton iteration instead of once per CR iteration); 0: every
                             island in the streamed CR loop */
  int32_t res_max_rows;   /* row cap of a resident island and of a group of them, at most 2048
                             (default 384; <= 0: 384) */
  int32_t line_search;    /* 1: back-tracking line search on each Newton step (Sec. 8.1): the
                             trials t = 1, 1/2, 1/4, 1/8, 1/16 (each a merit evaluation at
                             lambda + t dlambda, u + t du), the first whose FP64 merit is
                             below the current iterate's is taken, else the damped step t =
                             damping; per island in island mode.  0 (default, the paper's
                             results): the damped step */
  int32_t best_iterate;   /* 1 (requires island_stop = 1): each island that has not stopped
                             returns the iterate of least merit among those its Newton
                             iterations evaluated (the start included) when the final
                             iterate's merit is larger -- a safeguard against a diverging
                             iteration, not in the paper.  0 (default): the last iterate */
} nsn_config;

/* Fills the paper's defaults: h = 1/60, g = (0, 0, -9.81), 4 x 20 iterations,
 * t = 0.75, eps = 1e-6, FB, effective-mass r, GS on particles, FP32, graph on,
 * no cone projection, one system (no islands). */
void nsn_default_config(nsn_config *cfg);

typedef struct {
  int32_t newton_done;    /* Newton iterations solved in the last step */
  int32_t cr_total;       /* CR iterations summed over those Newton iterations */
  double merit0;          /* ||[g; h]|| at the zero iterate u = 0, lambda = 0 */
  double merit_final;     /* ||[g; h]|| at the returned iterate */
  float ms;               /* device time of the last call (CUDA events) */
} nsn_stats;

/* Input records (packed, 4-byte fields). */
typedef struct {
  int32_t body_a, body_b;  /* body ids, -1 = static world (not both) */
  float pa[3];             /* point on a: body-local (rigid), ignored (particle), world (-1) */
  float pb[3];             /* point on b, same convention */
  float n[3];              /* unit world contact normal pointing from b towards a (Sec. 3.3) */
  float d;                 /* thickness d of C_n = n^T (a - b) - d >= 0 */
  float mu;                /* friction coefficient (Sec. 3.4) */
} nsn_contact;

typedef struct {
  int32_t body_a, body_b;  /* rigid bodies, -1 = world */
  float pa[3], pb[3];      /* anchors: body-local, or world for a static side */
  float axis_a[3];         /* hinge axis in a's frame (world if static) */
  float axis_b[3];         /* hinge axis in b's frame (world if static) */
  float compliance;        /* e of Sec. 3.2; 0 = hard */
} nsn_revolute;

typedef struct {
  int32_t v[4];            /* particle body ids */
  float rest[4][3];        /* rest positions of the 4 vertices */
  float E, nu;             /* Young's modulus, Poisson ratio (App. B) */
} nsn_tet;

/* Creates a context on the current CUDA device.  stream: a cudaStream_t to
 * order all work on, or NULL to create a private stream. */
nsn_status nsn_create(const nsn_config *cfg, void *stream, nsn_ctx **out);
nsn_status nsn_destroy(nsn_ctx *ctx);
const char *nsn_last_error(const nsn_ctx *ctx);

/* Appends n bodies (copied).  kind[n] NSN_RIGID/NSN_PARTICLE; pos n x 3;
 * quat n x 4 unit quaternions (NULL = identity); vel n x 3; omega n x 3 (NULL = 0);
 * mass[n] > 0; inertia n x 3 body-frame principal moments > 0 (rigid; may be
 * NULL if all are particles).  first_id receives the id of the first body. */
nsn_status nsn_add_bodies(nsn_ctx *ctx, int32_t n, const int32_t *kind, const float *pos,
                          const float *quat, const float *vel, const float *omega,
                          const float *mass, const float *inertia, int32_t *first_id);

/* Appends n constraint records of one type (nsn_contact; nsn_revolute for
 * NSN_REVOLUTE and NSN_PRISMATIC; nsn_tet for NSN_TET_NH and NSN_TET_LINEAR;
 * copied).  first_row receives the first row of the block within its type's
 * row range (joints of both kinds share one range).  Contacts: body ids of
 * any kind or -1.  Joints: rigid or -1; prismatic axes nonzero.  Tets: four
 * distinct particles with a non-degenerate rest shape, E > 0, 0 < nu < 0.5. */
nsn_status nsn_add_constraints(nsn_ctx *ctx, int32_t type, int32_t n, const void *records,
                               int32_t *first_row);

/* Removes all contacts (they are regenerated every step, Sec. 10). */
nsn_status nsn_clear_contacts(nsn_ctx *ctx);

/* Number of bodies / constraint rows (after all adds). */
nsn_status nsn_counts(nsn_ctx *ctx, int32_t *n_bodies, int32_t *n_rows);

/* Advances nsteps time steps (Algorithm 1) from the current state and commits
 * each.  stats (may be NULL) describes the last step.  Returns
 * NSN_ERR_NONFINITE if the merit became NaN/Inf. */
nsn_status nsn_step(nsn_ctx *ctx, int32_t nsteps, nsn_stats *stats);

/* State in ABI body order; any pointer may be NULL.  Host arrays:
 * pos nb x 3, quat nb x 4, vel nb x 3, omega nb x 3 (particles: quat, omega ignored). */
nsn_status nsn_get_state(nsn_ctx *ctx, float *pos, float *quat, float *vel, float *omega);
nsn_status nsn_set_state(nsn_ctx *ctx, const float *pos, const float *quat, const float *vel,
                         const float *omega);
/* Same with device pointers (float32), ordered on the context stream. */
nsn_status nsn_set_state_device(nsn_ctx *ctx, const float *pos, const float *quat, const float *vel,
                                const float *omega);
nsn_status nsn_get_state_device(nsn_ctx *ctx, float *pos, float *quat, float *vel, float *omega);
/* State in the bulk precision of the context (double copies of the FP64 build's
 * values, for verification); same layout as nsn_get_state. */
nsn_status nsn_get_state_f64(nsn_ctx *ctx, double *pos, double *quat, double *vel, double *omega);
/* Multipliers of the last step (R values, forces in N). */
nsn_status nsn_get_lambda(nsn_ctx *ctx, double *lambda);
/* Merit after each Newton iteration of the last step, then the final merit;
 * returns the count through *n (at most cap written). */
nsn_status nsn_get_merit_history(nsn_ctx *ctx, double *out, int32_t cap, int32_t *n);

/* ---- verification entry points (used by the parity tests) ----------------
 * nsn_linearize: runs the first n_before Newton iterations of a step from the
 * current state without committing, then evaluates rows, g, H~, b and the
 * Jacobi diagonal at that iterate and keeps that linear system.
 * nsn_apply_operator: y = (J H~^-1 J^T + C + eps I) x on the kept system
 * (R doubles in/out, host), using the same kernels as the CR loop.
 * nsn_solve: runs iters CR iterations on the kept system from dl = 0 and
 * returns dl (R) and du = H~^-1 (h J^T dl - g) (D, in body order, 6 per rigid
 * body [v, w], 3 per particle); either output may be NULL.
 * nsn_get_system: copies b (R), the Jacobi diagonal (R), h (R) and g (D). */
nsn_status nsn_linearize(nsn_ctx *ctx, int32_t n_before);
nsn_status nsn_apply_operator(nsn_ctx *ctx, const double *x, double *y);
nsn_status nsn_solve(nsn_ctx *ctx, int32_t iters, double *dlambda, double *du);
nsn_status nsn_get_system(nsn_ctx *ctx, double *b, double *diag, double *hvec, double *g);

/* Number of kernels executed by the last step of nsn_step.  Under the CUDA
 * graph (use_graph = 1) the Newton and CR loops are conditional WHILE nodes,
 * so this counts the loop bodies actually run; eager launch (use_graph = 0)
 * launches every iteration up to the caps, finished ones returning at once. */
nsn_status nsn_last_launch_count(nsn_ctx *ctx, int32_t *kernels_per_step);

/* The body pass's segment tile chosen for this scene: *body_lanes lanes per
 * body (4, 8 or 16).  Scenes of 100,000 rows or more are tuned when the layout
 * is built: the operator's body pass is timed with each tile on the scene
 * itself, and another tile replaces 8 only if it is at least 10% faster (8
 * lanes also give finer skip blocks of bodies late in a step); ms3 (may be
 * NULL) receives the three measured times in ms (zeros when not tuned).
 * Smaller scenes use 8. */
nsn_status nsn_tuning(nsn_ctx *ctx, int32_t *body_lanes, float *ms3);
/* Island-resident CR of this scene (nsn_config.cr_resident): info6[0] islands
 * solved by k_cr_resident (0 when off: not island mode, cr_resident = 0, or no
 * eligible island), [1] the groups they are packed into (runs of consecutive
 * eligible islands, at most 32 islands and res_max_rows rows each, one thread
 * block per group), [2] rows and [3] Jacobian entries of the largest group
 * (the shared-memory image's capacity), [4] dynamic shared memory per thread
 * block in bytes, [5] thread blocks of the persistent grid.  NULL:
 * NSN_ERR_INVALID_ARG. */
nsn_status nsn_resident_info(nsn_ctx *ctx, int32_t *info6);
/* Times k_cr_resident alone: the scene is linearized at the zero start of a
 * step (lambda = 0; the committed x, q, u are kept, lambda is not), so every
 * resident island takes part, and the kernel runs `iters` timed launches
 * (after one untimed) of up to cr_iters CR iterations each, on the context's
 * stream with CUDA events.  *ms: mean launch time; work4 (may be NULL): the
 * islands solved per launch and the row-, entry- and body-iterations of one
 * launch (iterations that applied A, summed over islands).  No resident
 * islands, or iters < 1: NSN_ERR_INVALID_ARG.  Call nsn_linearize again before
 * the nsn_apply_operator / nsn_solve_linear family. */
nsn_status nsn_time_resident(nsn_ctx *ctx, int32_t iters, float *ms, double *work4);
/* Forces the body pass's lanes per body (4, 8 or 16; 0 = tuned as above) from
 * the next use of the context on (the device layout is rebuilt, the state
 * kept).  Invalid values: NSN_ERR_INVALID_ARG. */
nsn_status nsn_set_body_lanes(nsn_ctx *ctx, int32_t lanes);

/* Times the two kernels of one Schur operator apply (Eq. schur_system,
 * matrix-free: body-segment pass J^T z, H~^-1, J y per entry; row pass with
 * C z + eps z and the fused CR dot products) on the context stream with CUDA
 * events, iters times on the system of the last step, and returns the mean
 * duration of each in milliseconds.  Requires a prior nsn_step. */
nsn_status nsn_time_operator(nsn_ctx *ctx, int32_t iters, float *ms_body_pass, float *ms_row_pass);

/* Layout sizes: [rigid bodies, particles, rows, pair rows, tets, rigid
 * entries, particle entries, device bytes held by the context]. */
nsn_status nsn_operator_sizes(nsn_ctx *ctx, int64_t *sizes8);

/* ---- warm starts and the learned warm start ----------------------------------
 * The paper starts every step from lambda^0 = 0 (Sec. 8.1) and notes that
 * warm starting can improve efficiency.  NSN_WARM_PREV starts from the
 * previous step's multipliers; NSN_WARM_LEARNED sets the contact rows'
 * lambda^0 from a per-contact network (16 features -> 128 -> 128 -> 128 -> 4,
 * ReLU, BF16 tensor-core GEMMs with FP32 accumulation; contact rows only,
 * joint and tet rows start at zero): outputs are the change of the normal and
 * two friction multipliers from their previous-step values (a contact new in
 * this step has zero there), over the contact's gravity-scaled effective mass
 * |g| / (1/m_a + 1/m_b), and a log preconditioner scale.
 * NSN_WARM_PREV keeps the previous step's multipliers only if the merit at
 * (u = 0, lambda^0) is not above the merit at the zero start.  NSN_WARM_LEARNED
 * falls back on the previous-step start: of the three candidates (network,
 * previous step, zero) the one of least merit at u = 0 is kept.  With
 * island_stop = 1 both choices are made island by island.  u^0 = 0 in all
 * modes.  The relative merit is always taken against the zero start. */
enum { NSN_WARM_ZERO = 0, NSN_WARM_PREV = 1, NSN_WARM_LEARNED = 2 };
/* OR-ed into the mode: warm-start the friction rows too.  By default only the
 * normal and joint rows are warm started and friction starts at zero: the
 * friction compliance W of Sec. 4.3 is a fixed point in lambda_f, and a stale
 * friction state seeds the oscillation of that fixed point. */
#define NSN_WARM_FRICTION 0x100
/* With NSN_WARM_LEARNED: the network's fourth output, the logarithm of a
 * per-contact preconditioner scale (clamped to [1/4, 4]), multiplies the
 * Jacobi preconditioner P of the contact's three rows in every CR solve of
 * the step; the scale is trained towards A_ii (A^-1)_ii of the contact's
 * normal row (the diagonal of the inverse over the Jacobi diagonal). */
#define NSN_WARM_PRECOND 0x200
#define NSN_MLP_NPARAM (128 * 16 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 4 * 128 + 4)
nsn_status nsn_set_warm_start(nsn_ctx *ctx, int32_t mode);
/* The previous step's multipliers as the next warm start reads them (R
 * values, ABI row order; after contacts were replaced, those carried over by
 * key, zero for new contacts). */
nsn_status nsn_get_prev_lambda(nsn_ctx *ctx, double *lambda);
/* Forgets the previous step's multipliers (sets them to zero), e.g. after
 * the state was reset: the next step's previous-step candidate is then the
 * zero start.  Enqueued on the context stream; allocates nothing. */
nsn_status nsn_clear_warm_start(nsn_ctx *ctx);
/* Islands of the current scene: *n_islands, and the island of each body
 * (host array of the body count, may be NULL).  Islands are numbered in the
 * order of their lowest body id; they do not depend on island_stop. */
nsn_status nsn_islands(nsn_ctx *ctx, int32_t *n_islands, int32_t *body_island);

/* Per island, for the last nsn_step with island_stop = 1 (host arrays of cap
 * >= n_islands entries, any may be NULL): merit at the zero iterate, merit at
 * the returned iterate, and the Newton iteration at which the island stopped
 * (-1: it did not reach tol_rel within newton_iters). */
nsn_status nsn_island_stats(nsn_ctx *ctx, int32_t cap, double *merit0, double *merit_final,
                            int32_t *stopped_at);

/* Device pointer to the per-island stop iterations above (n_islands int32,
 * owned by the context, valid until the scene changes; written by each step
 * on the context stream).  For on-device bookkeeping between steps. */
nsn_status nsn_island_stop_device(nsn_ctx *ctx, const int32_t **stopped_at);
/* Enqueues on the context stream a device-to-device copy of those n_islands
 * int32 into dst_device (a device buffer of the caller).  Allocates nothing. */
nsn_status nsn_island_stop_copy(nsn_ctx *ctx, int32_t *dst_device);

/* Decision log, for comparisons across precisions (verification): the
 * discrete choices of the method at each of the first `iters` Newton
 * iterations of each following step (iters = 0: off; the log is kept on the
 * device and rewritten by every step).  nsn_get_decisions copies the last
 * step's log: rows (iters x nsn_counts() rows, ABI row order) and islands
 * (iters x islands of nsn_islands), one byte each:
 *   contact normal row: bit 0 the Fischer-Burmeister kink C = lambda = 0
 *     (Sec. 4.2; min-map: the branch C <= r lambda), bit 1 / bit 2 the cone
 *     projection clamped lambda_n / scaled lambda_f in the update;
 *   friction rows: 0 inactive (mu lambda_n <= 0, Sec. 3.5), 1 inactive past
 *     the asymptote of W (App. A.2), 2 stick (W = 0), 3 sliding;
 *   joint rows: 0;  tet rows: eigenvalues of the Hessian clamped to keep it
 *     positive definite (Sec. 9.2.2), +4 when the tet is inverted;
 *   island: the line-search trial taken (Sec. 8.1; 0..4 for t = 1 .. 1/16,
 *     5 the damped step), 255 an island that had stopped;
 *   cr (iters x islands, uint16): the CR updates the island took before a
 *     stop test of Sec. 8.2 (or the cap) ended its CR, 0xffff for an island
 *     that had stopped.
 * 255 marks a row or iteration that was not evaluated.  Any output may be
 * NULL.  No logged step: NSN_ERR_BAD_STATE. */
nsn_status nsn_record_decisions(nsn_ctx *ctx, int32_t iters);
nsn_status nsn_get_decisions(nsn_ctx *ctx, uint8_t *rows, uint8_t *islands, uint16_t *cr);

/* Merits of the last warm-started step: zero start, warm start (the
 * network's candidate for NSN_WARM_LEARNED), and whether that candidate was
 * not chosen (island_stop = 1: the number of islands where it was not). */
nsn_status nsn_get_warm_stats(nsn_ctx *ctx, double *merit_zero, double *merit_warm, int32_t *rejected);
/* Network parameters (host, NSN_MLP_NPARAM floats): W1[128][16], b1[128],
 * W2[128][128], b2, W3[128][128], b3, W4[4][128], b4[4]; y = W x + b.  Setting
 * them resets the Adam state.  get_params also returns the last gradients. */
nsn_status nsn_mlp_set_params(nsn_ctx *ctx, const float *params, int32_t n);
nsn_status nsn_mlp_get_params(nsn_ctx *ctx, float *params, float *grads, int32_t n);
/* Y[n][4] = network(X[n][16]); device pointers, context stream; returns after
 * the call has finished.  Inference runs on the tensor cores (tcgen05, FP32
 * accumulators in tensor memory) with BF16 inputs, weights and activations;
 * X may have any 4-byte alignment.  A completion wait of the tensor cores
 * that exceeds its bound: NSN_ERR_TIMEOUT (the outputs are then incomplete).
 * nsn_mlp_time_forward: the same call repeated reps >= 1 times on the
 * context's stream between two CUDA events, *ms (host) = mean device time
 * of one call. */
nsn_status nsn_mlp_forward(nsn_ctx *ctx, const float *X, int32_t n, float *Y);
nsn_status nsn_mlp_time_forward(nsn_ctx *ctx, const float *X, int32_t n, float *Y, int32_t reps, float *ms);
/* One training step on a batch (device X[n][16], targets T[n][4], output
 * weights w[4]): loss 1/(2n) sum w_k (y_k - t_k)^2, backward on the tensor
 * cores, Adam (lr; lr = 0 only computes the gradients); *loss (host) gets the
 * batch loss. */
nsn_status nsn_mlp_train_step(nsn_ctx *ctx, const float *X, const float *T, const float *w, int32_t n, float lr,
                              float *loss);
/* Features of every contact at the current (committed) state and, if Ytarget
 * is not NULL, the current multipliers as training targets (device arrays
 * X[nc][16], Ytarget[nc][4], contacts in the order they were added). */
nsn_status nsn_contact_features(nsn_ctx *ctx, float *X, float *Ytarget);

/* ---- allocation-free operator apply -----------------------------------------
 * The paper has no counterpart.  This entry point serves callers that cannot
 * allocate device memory where they need an operator product: a host
 * application that owns the device's memory and gives the library a fixed
 * budget with nothing to spare, and a real-time control loop that must not
 * block in the device allocator (cudaMalloc can synchronise the device).
 *
 * Computes y = (J H~^-1 J^T + C + eps I) x for the system kept by the last
 * nsn_step (its final evaluation) or nsn_linearize, with the same kernels as
 * the CR loop.  x and y are caller-owned device arrays of nsn_counts() rows
 * (float32); stream is a cudaStream_t or NULL for the context stream.  A
 * stream other than the context stream must be ordered after the context
 * stream's last nsn_step / nsn_linearize (e.g. by waiting on an event recorded
 * there): the apply reads the Jacobian entries, compliances and inverse masses
 * that those calls wrote.  The call allocates nothing: the per-entry scratch
 * lives in a fixed static device array of NSN_NOALLOC_MAX_ENTRIES floats
 * (16 MiB), and x and y are permuted into the context's internal (island) row
 * order through two static arrays of NSN_NOALLOC_MAX_ENTRIES / 2 floats
 * (8 MiB each); every GPU loading the library holds them until the process
 * exits.  Scenes needing more row slots than NSN_NOALLOC_MAX_ENTRIES (2 per
 * contact or joint row, 4 per tet row) are rejected with NSN_ERR_INVALID_ARG.
 * All calls share the arrays and they keep the last call's contents; each
 * call first clears the slots it uses (the world side of a contact is read as
 * zero), with a memset on the stream, which allocates nothing.  Calls that
 * overlap on the GPU (different streams, or different contexts on one device)
 * race on the arrays.  The first call on a device (and the first after the
 * device's CUDA context changed) resolves the arrays' device addresses, under
 * a lock shared by all host threads; make that first call before any stream
 * capture.  FP32 contexts only. */
#define NSN_NOALLOC_MAX_ENTRIES (4 * 1024 * 1024)
nsn_status nsn_apply_operator_noalloc(nsn_ctx *ctx, const float *x, float *y, void *stream);

/* ---- contact generation (Sec. 3.3, Sec. 10) ---------------------------------
 * The paper creates a contact constraint when two features come within a
 * fixed distance of each other (Sec. 3.3), runs collision detection once per
 * time step with the unconstrained velocity to find candidates, and takes the
 * normal as the normalised vector between the closest points at the start of
 * the step (Sec. 10).  The collider does this for box and particle scenes:
 *   vertices: the 8 corners of every rigid body with a box shape (corner k has
 *             coordinate +half[i] on axis i where bit i of k is set, -half[i]
 *             otherwise), and every particle;
 *   shapes:   the static planes (all environments), and the rigid boxes of the
 *             vertex's own environment other than its own body and the
 *             excluded pairs (e.g. the two bodies of a joint).
 * Vertex p of body A is a candidate against shape B when p, or its predicted
 * position p + h (u_A(p) - u_B(p)) with u the unconstrained velocity field of
 * each body (v + omega x r), lies within `margin` of B (inside a box counts as
 * distance 0).  A contact record (the CONTACT layout of the scene arrays):
 * body_a = A, body_b = B or -1 for a plane; pa = the corner in A's frame (0
 * for a particle); pb = the closest point of B at the start of the step, in
 * B's frame, or the world foot point on a plane; n = the world normal from B
 * towards A: the plane normal, (p - closest point) / distance outside a box,
 * the outward normal of the face of least penetration inside it; d = 0; mu =
 * mu_env of A's environment.  Order: by vertex (body, then corner), then the
 * planes in order, then the boxes in body order.  Candidate, outside/inside
 * and nearest-face decisions are taken in FP32 with one rounding per
 * operation; closest points and normals in FP64, rounded to FP32.
 *
 * nsn_collider_create: the static scene.  kind (0 rigid, 1 particle), half
 * (n x 3 box half extents; a rigid body with any extent <= 0 has no shape and
 * no vertices) and env (environment id per body, non-decreasing, in
 * [0, n_envs)) for n_bodies bodies; mu_env (n_envs); planes (n_planes x 4:
 * unit normal n and offset o of the plane n.x = o, solid side n.x < o);
 * exclude (n_exclude x 2 body ids); margin > 0; h >= 0 the step of the
 * prediction; stream: a cudaStream_t for all work of the collider, or NULL.
 * Host arrays are copied; the caller keeps them.  Bad sizes, ids, order or
 * values, or more than 2^31 - 1 vertex-shape pairs (the sum over environments
 * of vertices x (planes + boxes)): NSN_ERR_INVALID_ARG; device memory:
 * NSN_ERR_OUT_OF_MEMORY.
 *
 * nsn_collider_run: host arrays.  pos (n x 3), quat (n x 4, w x y z), vel and
 * omega (n x 3, the unconstrained velocity, world frame) are copied in; at
 * most `capacity` contacts are copied out to c_body (capacity x 2), c_pa,
 * c_pb, c_n (capacity x 3), c_d, c_mu (capacity); *n_found = the number of
 * contacts found.  Returns when the results are on the host.  More contacts
 * than capacity: the first `capacity` are written and the call returns
 * NSN_ERR_OUT_OF_MEMORY with *n_found set (call again with a larger buffer).
 *
 * nsn_collider_run_async: the same with device arrays on the collider's
 * stream, nothing copied and nothing synchronised: the count goes to the
 * device int32 *found_dev (may be NULL), contacts past `capacity` are not
 * written.  The collider's scratch is shared by its calls: calls on one
 * collider are serialised by its stream, and a collider is used from one
 * host thread at a time.
 *
 * nsn_collider_info: info4 = {bodies, vertices, planes, thread blocks per
 * launch}.  Errors of a collider call: nsn_collider_last_error. */
typedef struct nsn_collider nsn_collider;
nsn_status nsn_collider_create(int32_t n_bodies, const int32_t *kind, const float *half, const int32_t *env,
                               int32_t n_envs, const float *mu_env, int32_t n_planes, const float *planes,
                               int32_t n_exclude, const int32_t *exclude, float margin, float h, void *stream,
                               nsn_collider **out);
nsn_status nsn_collider_destroy(nsn_collider *c);
nsn_status nsn_collider_run(nsn_collider *c, const float *pos, const float *quat, const float *vel,
                            const float *omega, int32_t capacity, int32_t *c_body, float *c_pa, float *c_pb,
                            float *c_n, float *c_d, float *c_mu, int32_t *n_found);
nsn_status nsn_collider_run_async(nsn_collider *c, const float *pos, const float *quat, const float *vel,
                                  const float *omega, int32_t capacity, int32_t *c_body, float *c_pa, float *c_pb,
                                  float *c_n, float *c_d, float *c_mu, int32_t *found_dev);
nsn_status nsn_collider_info(const nsn_collider *c, int32_t *info4);
const char *nsn_collider_last_error(const nsn_collider *c);

/* Time steps with contacts generated at the start of each (Sec. 10: collision
 * detection once per step, candidates from the unconstrained velocity,
 * normals between closest points at the start of the step).  For each of
 * nsteps steps: the collider runs on the context's current state (positions,
 * orientations, angular velocities, and linear velocities plus h g), its
 * contacts replace the context's contacts, and one step of nsn_step runs.
 * The collider describes the same bodies as the context (same count and
 * order); its contacts come with the collider's friction per environment.
 * Replacing the contacts rebuilds the context's layout on the host (the
 * islands and the row order change with the contacts); the previous step's
 * multipliers -- the NSN_WARM_PREV start and the learned start's fallback --
 * carry over contact by contact through the key (body_a, body_b, point on
 * a), which for a generated contact names the vertex and the shape, and row
 * by row for joints and tets.  stats: the last step.  Errors: those of the
 * collider (NSN_ERR_INVALID_ARG for a collider of another body count) and of
 * nsn_step.  The context's stream waits for the collider at each step. */
nsn_status nsn_collide_and_step(nsn_ctx *ctx, nsn_collider *col, int32_t nsteps, nsn_stats *stats);

/* Host wall time, in milliseconds, of the phases of the last rebuild and
 * step (std::chrono steady clock, measured by the calling thread; each
 * phase ends with the stream synchronisation it already performs):
 *   NSN_PHASE_COLLIDE  nsn_collide_and_step: state export, collider run,
 *                      contact download and records
 *   NSN_PHASE_SAVE     previous multipliers and the state read back
 *   NSN_PHASE_LAYOUT   host layout (islands, orders, entry lists, groups)
 *   NSN_PHASE_UPLOAD   device arrays written, state scattered
 *   NSN_PHASE_RESTORE  previous multipliers matched by contact key, written
 *   NSN_PHASE_CAPTURE  CUDA graph capture and instantiation of the step
 *   NSN_PHASE_STEP     the step's launches up to its final synchronisation
 * A phase that did not run in the last call keeps its previous value, except
 * that a rebuild resets SAVE..RESTORE and a step resets CAPTURE.  ms holds
 * NSN_PHASES doubles (host).  Errors: NSN_ERR_INVALID_ARG for null arguments. */
enum { NSN_PHASE_COLLIDE = 0, NSN_PHASE_SAVE, NSN_PHASE_LAYOUT, NSN_PHASE_UPLOAD, NSN_PHASE_RESTORE,
       NSN_PHASE_CAPTURE, NSN_PHASE_STEP, NSN_PHASES };
nsn_status nsn_get_phase_times(nsn_ctx *ctx, double *ms);

/* best_iterate: the number of islands of the last step that returned an
 * earlier iterate than their last (0 when the option is off).  Errors:
 * NSN_ERR_INVALID_ARG for null arguments. */
nsn_status nsn_best_restored(nsn_ctx *ctx, int32_t *n_islands);

#ifdef __cplusplus
}
#endif
#endif
