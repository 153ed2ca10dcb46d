/*
 * dg_mhd.h -- C ABI of the GB300 DG-MHD hot path.
 *
 * The operator is the modal discontinuous Galerkin scheme for ideal MHD of
 * Guillet, Pakmor, Springel, Chandrashekar & Klingenberg (2018):
 *   du/dt + sum_a d f_a(u)/dx_a = s                      (Sec. 2, eq. cns-eq)
 *   M_l dw_l/dt = (2/dx)[ int f_a . d_a phi_l - oint F*.n phi_l ] + int s.phi_l
 *                                                        (Sec. 3.5, eq. wdot)
 * with HLLD face fluxes (Sec. 4.1.2), Powell source terms on a locally
 * divergence-free (LDF) B basis (Sec. 4.1.3) or GLM cleaning (Sec. 4.1.5),
 * TVB-characteristic and positivity limiters (Sec. 4.2, 4.3), the CFL
 * timestep (Sec. 3.6, eq. cfl; Powell: eq. powell_dt) and SSP Runge-Kutta.
 *
 * Conventions shared by every call
 * --------------------------------
 * Pointers named w, wmean, rhs, rhs_mean, dt_dev are DEVICE pointers owned by
 * the caller. Pointers inside dg_mesh_desc and `nodal` of dg_mhd_project are
 * HOST or DEVICE as stated. `stream` is a cudaStream_t passed as void*
 * (NULL = legacy default stream). Every call is asynchronous on `stream`
 * unless stated; nothing synchronises the host except dg_mhd_status(ctx, 1)
 * and dg_mhd_init / dg_mhd_destroy.
 *
 * State layout (SoA, coalesced along cells): w[row][cell], row-major with the
 * cell index fastest, n_cells cells padded to `cell_stride` (a multiple of 4).
 * Rows: for the GLM scheme 9 Legendre variables x n(d) modes
 * (rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi; row = var*n + mode). For the
 * Powell scheme 5 Legendre hydro variables x n(d), then N_div LDF rows for B,
 * then (2D only) n(d) Legendre rows for B_z. Modes are ordered by total degree,
 * then k1 descending, then k2 descending; Legendre polynomials have l_k(1) = 1,
 * so mode 0 is the cell mean. LDF rows follow App. A.2 (curls of Legendre
 * potentials, stable-sorted by degree, unnormalised Gram-Schmidt).
 *
 * Precision: DG_PREC_FP64 -> w/rhs are double; wmean/rhs_mean unused (NULL).
 * DG_PREC_FP32MIX -> w/rhs are float and the degree-0 rows are ALSO held in
 * double in wmean[mean_row][cell] (mean rows = Legendre mode 0 of each
 * variable, then the degree-0 LDF rows, in row order); the double copy is
 * authoritative and the float mode-0 entries mirror it.
 *
 * Errors: every int-returning call returns a dg_status. Nothing throws or
 * aborts. Errors found on the device (non-finite state, positivity floor
 * used, c_h below the signal speed, timed-out wait) are latched in a device
 * status word and reported by dg_mhd_status.
 */
#ifndef DG_MHD_H
#define DG_MHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mhd_ctx dg_mhd_ctx;

typedef enum {
  DG_OK = 0,
  DG_E_ARG = -1,         /* bad argument (NULL, size, enum out of range)      */
  DG_E_MESH = -2,        /* invalid mesh description                           */
  DG_E_CUDA = -3,        /* a CUDA runtime call failed                         */
  DG_E_NONFINITE = -4,   /* NaN/Inf found in the state or the timestep        */
  DG_E_CH = -5,          /* GLM: c_h below the largest signal speed (Sec 4.1.5)*/
  DG_E_TIMEOUT = -6,     /* a bounded device wait gave up                      */
  DG_E_UNSUPPORTED = -7, /* combination not built (e.g. degree > 3)            */
  DG_W_FLOOR = 1         /* warning: positivity floor injected mass/energy     */
} dg_status;

enum { DG_DIVB_POWELL = 0, DG_DIVB_GLM = 1 };
enum { DG_PREC_FP64 = 0, DG_PREC_FP32MIX = 1 };
enum { DG_LIMIT_OFF = 0, DG_LIMIT_TVB = 1, DG_LIMIT_MLP = 2 };

/* Mesh (Sec. 3.1: non-overlapping cubic cells of an octree, Sec. 4.4).
 * Uniform (level == NULL): a periodic box of n[0] x n[1] (x n[2]) cells,
 * numbered x-fastest, cell size box_len / n[0].
 * Octree (level != NULL): n_leaves leaves of a periodic cube of side box_len;
 * leaf c has refinement level level[c] (cell size box_len / 2^level) and
 * integer coordinates ijk[c*dim + a] in [0, 2^level); the leaves must tile
 * the box without overlap and be 2:1 balanced across faces (DG_E_MESH
 * otherwise). Cells are numbered in the given order. Host memory, copied at
 * init. Faces: same-level, and coarse-fine faces integrated at the fine face's
 * Gauss points (coarse side at the mapped sub-face points, weights / 2^(dim-1)).
 * At most 2^31 - 65 cells (indices are 32-bit on the device): DG_E_MESH beyond. */
typedef struct {
  int dim;               /* 2 or 3                                             */
  int32_t n[3];          /* uniform: cells per axis (n[2] ignored for dim 2)   */
  double box_len;        /* uniform: n[0]*dx; octree: side of the cube         */
  int periodic;          /* must be 1                                          */
  int64_t n_leaves;      /* octree: number of leaves                           */
  const int8_t* level;   /* octree: n_leaves levels (NULL: uniform mesh)       */
  const int32_t* ijk;    /* octree: n_leaves*dim integer coordinates           */
  int partial;           /* octree, 1: a partition's local mesh -- the owned
                            leaves and their face neighbours (ghosts) of a
                            larger octree; they need not cover the cube, a face
                            with no leaf across it is left out (the ghosts'
                            results are the caller's to discard), regridding
                            calls return DG_E_UNSUPPORTED. 0: a full mesh    */
} dg_mesh_desc;

/* Parameters of Sec. 3.6, 4.1, 4.2, 4.3, 5.1 (defaults in brackets). */
typedef struct {
  double cfl;         /* C of eq. cfl                                [0.3]  */
  double cfl_glm;     /* C' of Sec. 4.1.5, C < C' < 1                 [0.9]  */
  double c_r;         /* c_p^2 / c_h                                 [0.18] */
  double c_h_fixed;   /* > 0: use this global c_h (AMR practice)      [0]    */
  double eta_powell;  /* eq. powell_dt threshold                      [0.2]  */
  double eps_hlld;    /* relative degeneracy test of the HLLD * states [1e-8]*/
  double Mtilde;      /* TVB threshold M~ (Sec. 4.2.1, 5.1)          [5]    */
  double beta;        /* minmod factor                               [2]    */
  double tvb_eps;     /* trigger threshold epsilon                   [1e-8] */
  double eps_rho;     /* positivity floors (Sec. 4.3, 5.1)           [1e-12]*/
  double eps_p;       /*                                             [1e-12]*/
  int precision;      /* DG_PREC_*                                   [FP64] */
  int limiter;        /* DG_LIMIT_*                                  [OFF]  */
  int positivity;     /* 1: positivity limiter on                    [0]    */
  int generic_kernels;/* 1: force the generic kernels even where a    [0]
                         specialised kernel exists (testing); 2: the
                         specialised kernels with the cell update's
                         contractions on the tensor core (3D GLM, degree
                         2, FP32 form; slower than the default CUDA-core
                         update on GB300, kept for comparison)               */
  int rk_order;       /* SSP-RK order of dg_mhd_step, 1..4 (Sec. 3.6); [3]
                         0: degree + 1 (at most 4), the paper's default      */
  int powell_q;       /* Powell face term q^dagger (Sec. 4.1.3):       [0]
                         0: q of the cell mean (eq. powellq-average, the
                         paper's default); 1: eq. powellq-interp, the layer
                         average between the trace and the HLLD interface
                         state, per face point (generic and octree
                         kernels; ignored with GLM and by
                         dg_mhd_rhs_noalloc)                                 */
} dg_mhd_params;

/* Fills *p with the defaults listed above. */
void dg_mhd_default_params(dg_mhd_params* p);

/* Builds the basis and quadrature tables (Sec. 3.2, 3.3, 3.5; App. A), the
 * face lists, and the device scratch for one mesh. degree d in 0..3;
 * divB_scheme DG_DIVB_*; gamma > 1. p NULL = defaults. On success *out owns
 * all device memory it allocated; release it with dg_mhd_destroy.
 * Uses the current CUDA device. Synchronous. */
int dg_mhd_init(const dg_mesh_desc* mesh, int degree, int divB_scheme, double gamma,
                const dg_mhd_params* p, dg_mhd_ctx** out);

/* Layout of the caller's buffers: rows per cell, degree-0 ("mean") rows per
 * cell, cells, and the cell stride (elements between consecutive rows). */
int dg_mhd_state_layout(const dg_mhd_ctx* ctx, int64_t* n_rows, int64_t* n_mean_rows,
                        int64_t* n_cells, int64_t* cell_stride);

/* L2 projection of point values onto the basis (eq. u-exp inverted with the
 * diagonal mass matrix, Sec. 3.1): nodal[var][q][cell] (DEVICE, double,
 * cell index fastest with stride cell_stride) holds the conserved variables at
 * the npts^dim tensor Gauss-Legendre points of each cell (last axis fastest);
 * npts in 1..8. Writes w (and wmean in FP32MIX). */
int dg_mhd_project(dg_mhd_ctx* ctx, const double* nodal, int npts, void* w, double* wmean,
                   void* stream);

/* The basis as a linear map from state rows to point values (HOST, no
 * context, no device work; Sec. 3.1 eq. u-exp, Sec. 3.2-3.3): for npts
 * reference points xi[p*dim + a] in [-1, 1]^dim of a cell,
 * out[(r*n_vars + v)*npts + p] = the value of conserved variable v at point p
 * of the field whose only non-zero weight is a 1 in state row r (the rows of
 * the state layout above: a Legendre row feeds its own variable, an LDF row
 * B_x, B_y (, B_z)). So u_v(xi_p) = sum_r out[r][v][p] w[r][cell]. Writes
 * *n_rows and *n_vars (9 GLM, 8 Powell) and, if out is non-NULL and cap >=
 * n_rows*n_vars*npts doubles, out (DG_E_ARG if too small; DG_E_ARG for dim
 * not 2 or 3, degree outside 0..3, an unknown scheme, npts outside
 * 0..2^24 or xi NULL with npts > 0). */
int dg_mhd_basis_values(int dim, int degree, int divB_scheme, int64_t npts, const double* xi, int64_t cap,
                        double* out, int* n_rows, int* n_vars);

/* The map the specialised Powell kernels use between the 3D LDF basis of B
 * (Sec. 3.3) and the Legendre coefficients of its components (HOST, no
 * context, no device work): A[(j*3 + c)*n_modes + l] = <phi_j,c, P_l> / <P_l, P_l>
 * for LDF function j of degree <= degree and component c, so the component
 * c of sum_j w_j phi_j has Legendre coefficients sum_j w_j A[j][c][l] (exact:
 * every component is a polynomial of total degree <= degree). Computed by
 * quadrature with degree + 1 Gauss points per axis; entries below 1e-13 are
 * zero. Writes *n_div, *n_modes and, if A is non-NULL and cap >=
 * n_div*3*n_modes doubles, A (DG_E_ARG if too small or for a degree outside
 * 0..3; DG_E_UNSUPPORTED if the expansion misses a function at the points). */
int dg_mhd_ldf_legendre(int degree, int64_t cap, double* A, int* n_div, int* n_modes);

/* Sets the GLM wave speed c_h and damping rate c_h^2/c_p^2 used by
 * dg_mhd_rhs (Sec. 4.1.5). dg_mhd_dt and dg_mhd_step set them on the device
 * themselves; this call is for evaluating the operator at chosen values. */
int dg_mhd_set_glm(dg_mhd_ctx* ctx, double c_h, double damping_rate, void* stream);

/* One application of the spatial operator, eq. wdot: rhs = dw/dt for every
 * cell (projection, volume integral, HLLD face fluxes, Powell or GLM terms).
 * w is not modified. rhs has the layout of w. */
int dg_mhd_rhs(dg_mhd_ctx* ctx, const void* w, const double* wmean, void* rhs, double* rhs_mean,
               void* stream);

/* One stage of an SSP Runge-Kutta step (Sec. 3.6): out = a u0 + b (w + dt
 * L(w)) with L the operator of dg_mhd_rhs and dt the context's current step
 * (from dg_mhd_dt or dg_mhd_set_dt); the SSP-RK3 step of dg_mhd_step is
 * stage(w -> s1; 0, 1), stage(s1 -> s2; 3/4 w, 1/4), stage(s2 -> w; 1/3 w,
 * 2/3) with the limiter applied to s1 and s2. u0 may be NULL when a == 0; out
 * may alias u0 (not w). FP32MIX: wmean, outmean and (with u0) u0mean are the
 * FP64 means. Layouts as dg_mhd_rhs. */
int dg_mhd_stage(dg_mhd_ctx* ctx, const void* w, const double* wmean, const void* u0, const double* u0mean,
                 void* out, double* outmean, double a, double b, void* stream);

/* Sets the step length from a DEVICE double (for instance the minimum over
 * the ranks of a partitioned run, after an all-reduce) and, for GLM, the
 * cleaning speed and damping rate derived from it (Sec. 4.1.5), as dg_mhd_step
 * does with a given dt. Asynchronous on stream. */
int dg_mhd_set_dt(dg_mhd_ctx* ctx, const double* dt_dev, void* stream);

/* The context's current GLM cleaning speed c_h and damping rate (Sec. 4.1.5)
 * into host doubles; synchronises the device. 0 until a timestep, dg_mhd_set_glm
 * or dg_mhd_set_dt has set them (or c_h_fixed at init). */
int dg_mhd_glm_speeds(dg_mhd_ctx* ctx, double* c_h, double* damping_rate);

/* Cells that count in the timestep minimum of dg_mhd_dt (eq. cfl, eq.
 * powell_dt): mask (DEVICE, n_cells bytes, copied) holds 1 for the cells a
 * partition's rank owns, 0 for its ghost cells, whose face neighbours may be
 * missing or stale; NULL restores all cells. */
int dg_mhd_set_owned(dg_mhd_ctx* ctx, const uint8_t* mask, void* stream);

/* Limiters of Sec. 4.2-4.3 in place on w: TVB-characteristic slope limiter
 * (with the LDF slope fix of Sec. 4.2.4 for Powell) if enabled, then the
 * positivity limiter if enabled. troubled (DEVICE, nullable) receives 1 for
 * cells whose slopes the TVB limiter modified, else 0. */
int dg_mhd_limit(dg_mhd_ctx* ctx, void* w, double* wmean, uint8_t* troubled, void* stream);

/* Global timestep: eq. cfl from cell means, and eq. powell_dt for Powell
 * (|div B| from the face jumps of App. C eq. divb-cell). Writes dt to the
 * DEVICE scalar *dt_dev and, for GLM, sets c_h and the damping rate. */
int dg_mhd_dt(dg_mhd_ctx* ctx, const void* w, const double* wmean, double* dt_dev, void* stream);

/* One SSP-RK step (Sec. 3.6) of order rk_order in place on w (and wmean):
 * 1 forward Euler, 2 and 3 the Shu-Osher SSPRK(2,2) and SSPRK(3,3), 4 the
 * ten-stage SSPRK(10,4) of Ketcheson (2008) in its two-register form (ten
 * operator evaluations of dt/6 each). Scratch: the context's stage buffers.
 * dt_dev: DEVICE scalar with the step, or NULL to compute it from the limited
 * input with dg_mhd_dt (then read it back with dg_mhd_last_dt). Limiters, if
 * enabled, are applied to every stage input before it is evaluated (Sec. 4.3).
 * GLM: with dt_dev given, c_h follows from it before the first limiter pass;
 * with dt computed, the first limiter pass uses the c_h of the previous step. */
int dg_mhd_step(dg_mhd_ctx* ctx, void* w, double* wmean, const double* dt_dev, void* stream);

/* Device address of the timestep computed by the last dg_mhd_dt/step call. */
const double* dg_mhd_last_dt(const dg_mhd_ctx* ctx);

/* Reads the device status word. sync = 1: synchronise the stream first and
 * clear the word after reading. Returns DG_OK, a latched error or DG_W_FLOOR. */
int dg_mhd_status(dg_mhd_ctx* ctx, int sync);

/* Positivity diagnostics (Sec. 4.3): cells rescaled by the positivity limiter
 * (tau < 1) and the mass and energy injected by the mean floors, accumulated
 * since the last reset. Synchronises the device; reset = 1 clears them. */
int dg_mhd_counters(dg_mhd_ctx* ctx, int64_t* pos_cells, double* inj_mass, double* inj_energy, int reset);

/* Workload of the positivity limiter in the FP32 form (measurement support,
 * no counterpart in the paper): cells whose FP32 screen could not clear them
 * and that therefore went through the full procedure, summed over limiter
 * passes since the last reset (FP64 contexts run the procedure on every cell
 * and count 0). Synchronises the device; reset = 1 clears the count. */
int dg_mhd_positivity_listed(dg_mhd_ctx* ctx, int64_t* listed, int reset);

/* Divergence diagnostics of App. C on a uniform mesh (DG_E_UNSUPPORTED on
 * octrees), from the state w (and wmean in the FP32 form):
 * res (DEVICE, 4 doubles): [0] ||div B||_1 = (1/V) sum_K V_K |div B|_K
 * (eq. divb-total) with |div B|_K of eq. divb-cell: the L1 norm of div B over
 * the cell (the scheme's Gauss points) plus the face jumps |B^n_F - B^n_K|
 * over its boundary, both divided by V_K; [1] the volume average and [2] the
 * maximum of the normalised divergence |div B|_K dx / |mean B|_K
 * (eq. divb-normalized; 0 where the mean field vanishes); [3] the maximum of
 * |(div B)_K|, the signed divergence (1/V_K) oint B^n_F dS (eq. divb-gauss,
 * read with the cell volume). per_cell (DEVICE, 3 rows of cell_stride
 * doubles, or NULL): |div B|_K, (div B)_K and the normalised divergence.
 * Uses the context's face scratch; asynchronous on stream. */
int dg_mhd_divb(dg_mhd_ctx* ctx, const void* w, const double* wmean, double* res, double* per_cell, void* stream);

/* Troubled-cell statistics of the TVB limiter (Sec. 4.2 judges a detector by
 * its sensitivity and specificity; these counts give its workload), summed
 * since the last reset: limiter passes that ran the TVB procedure, cells that
 * went through it (flagged by the learned indicator, or every cell with the
 * plain detector), and cells whose slopes it changed. Any pointer may be
 * NULL. Synchronises the device; reset = 1 clears the counts. */
int dg_mhd_limiter_counts(dg_mhd_ctx* ctx, int64_t* passes, int64_t* flagged, int64_t* limited, int reset);

/* Learned troubled-cell indicator. The paper makes troubled-cell detection
 * a separate step of limiting, judged by sensitivity and specificity (Sec. 4.2);
 * the network is not in the paper. With limiter = DG_LIMIT_MLP, a network
 * (nin -> 64 -> 64 -> 1, ReLU, sigmoid; BF16 weights, FP32 accumulation on the
 * tensor cores) flags cells, and only flagged cells go through the TVB
 * procedure. Features of a cell, nin = 8 n(d) + 10*dim: Legendre coefficients
 * of the 8 MHD variables (LDF B mapped exactly to per-component Legendre
 * coefficients), variable v divided by |mean_v| + max_nb |mean_nb,v - mean_v|
 * + 1e-12, then rho_nb/rho - 1 for neighbours -x, +x, -y, +y (, -z, +z), then
 * for each direction the 8 degree-1 coefficients divided by M~ dx. Octree
 * meshes: the neighbour mean on a side is the average of the leaves across it
 * (as in the octree TVB procedure) and dx the leaf's own size.
 * theta (DEVICE, FP32, flat): W1[64][nin], b1[64], W2[64][64], b2[64],
 * w3[64], b3. */
/* X[cell*ldx + k] (DEVICE float, ldx >= nin; padding written as 0). */
int dg_mhd_mlp_features(dg_mhd_ctx* ctx, const void* w, const double* wmean, float* X, int ldx, void* stream);
/* Copies theta (DEVICE) into the context as BF16; flag = sigmoid > threshold.
 * Synchronous. nin must equal 8 n(d) + 10*dim. */
int dg_mhd_mlp_set_weights(dg_mhd_ctx* ctx, const float* theta, int nin, float threshold);
/* Features + inference for every cell: flags (nullable, uint8) and prob
 * (nullable, float) per cell (DEVICE). */
int dg_mhd_mlp_infer(dg_mhd_ctx* ctx, const void* w, const double* wmean, uint8_t* flags, float* prob,
                     void* stream);
/* Mean weighted binary cross-entropy -(pw y log p + (1-y) log(1-p)) over n
 * samples and its gradient (FP32 forward and backward, same layout as theta).
 * X, y (uint8 labels), theta, grad, loss: DEVICE. Synchronous; allocates. */
int dg_mhd_mlp_loss_grad(const float* X, int ldx, const uint8_t* y, int64_t n, int nin, const float* theta,
                         float pos_weight, float* grad, double* loss, void* stream);
/* Adam training (beta 0.9/0.999, eps 1e-8) on shuffled mini-batches, theta
 * updated in place; last_loss (host, nullable) receives the mean loss of the
 * last epoch. Synchronous; allocates its scratch. */
int dg_mhd_mlp_train(const float* X, int ldx, const uint8_t* y, int64_t n, int nin, float* theta, int epochs,
                     int batch, float lr, float pos_weight, uint64_t seed, double* last_loss, void* stream);

/* Measurement support (no counterpart in the paper). Kernel kinds:
 * 0 face flux, 1 cell update, 2 timestep, 3 TVB limiter, 4 projection,
 * 5 positivity limiter, 6 learned indicator (features + inference).
 * dg_mhd_profile(ctx, 1) resets the counters and, from then on, records a
 * CUDA event pair on the launch stream around every kernel launch;
 * dg_mhd_profile(ctx, 0) stops recording (launches are still counted).
 * dg_mhd_profile_read synchronises the device and returns, for one kind, the
 * summed event-timed device milliseconds and the number of launches since the
 * last reset. dg_mhd_launch_count returns all launches since the last reset. */
int dg_mhd_profile(dg_mhd_ctx* ctx, int enable);
/* Throughput probe of the current device (measurement support, no counterpart
 * in the paper; synchronous: one warm-up and one timed launch, CUDA events on
 * `stream`). kind 0: packed FP32 FMA (fma.rn.f32x2), 1: FP64 FMA, 2: TF32
 * tensor-core MMA (tcgen05 kind::tf32, M = 128, N = 256, K = 8, FP32
 * accumulators in tensor memory, one block per SM), 3: device-memory copy of
 * `bytes` (a multiple of 16) from src to dst (caller-owned DEVICE buffers,
 * 16-byte aligned; ignored for kinds 0-2). *rate: flop/s (kinds 0-2, 2 flop per
 * FMA) or bytes/s read plus written (kind 3); *ms: the timed launch.
 * DG_E_ARG for a bad kind or copy size, DG_E_TIMEOUT if the MMA probe's
 * bounded wait ran out. */
int dg_mhd_probe(int kind, const void* src, void* dst, int64_t bytes, double* rate, double* ms, void* stream);
int dg_mhd_profile_read(dg_mhd_ctx* ctx, int kind, double* total_ms, int64_t* launches);
int64_t dg_mhd_launch_count(const dg_mhd_ctx* ctx);

/* dg_mhd_rhs without any device allocation (the paper has no counterpart:
 * this is a deployment variant of dg_mhd_rhs).
 * For callers that cannot call cudaMalloc -- a framework whose pool owns all
 * device memory, code that must not trigger the device synchronisation that
 * cudaMalloc/cudaFree can cause, or an embedding that fixes the device
 * footprint at start-up. No context is needed: mesh, degree, scheme, gamma and
 * p (NULL = defaults; only eps_hlld is read, DG_E_ARG unless it lies in
 * [0, 1)) describe the problem, and c_h > 0 and damping_rate >= 0 set the GLM
 * terms (ignored for Powell). The caller passes the FP64 state w and the FP64
 * output rhs (DEVICE, layout of dg_mhd_rhs with cell_stride = n_cells rounded
 * up to a multiple of 32; the library cannot check their sizes).
 * status_dev (nullable, DEVICE int owned by the caller) receives the call's
 * device status word in stream order: 0, or bit 1 set when rhs holds a NaN or
 * an infinity (dg_mhd_status's DG_E_NONFINITE).
 * All scratch (basis tables, device scalars, face fluxes) lives in one static
 * device array of 4 Mi doubles (32 MiB) that every GPU loading the library
 * keeps until the process exits; the call looks up its device address
 * (cudaGetSymbolAddress) on the current device every time. With lazy module
 * loading (the CUDA default) the first call on a device loads this library's
 * module, which can allocate device memory and synchronise: make one warm-up
 * call per device at start-up, before any stream capture. The host copies of
 * the tables it uploads are built once per (dim, degree, scheme) and kept
 * until exit. Problems whose scratch exceeds the array return DG_E_ARG (about
 * 16 thousand cells at degree 2 in 3D). Every call rewrites the shared array
 * (tables and scalars are re-uploaded and the status word cleared), so calls
 * that overlap on the GPU -- two streams, two host threads -- race and must be
 * serialised by the caller. */
int dg_mhd_rhs_noalloc(const dg_mesh_desc* mesh, int degree, int divB_scheme, double gamma,
                       const dg_mhd_params* p, double c_h, double damping_rate, const double* w,
                       double* rhs, int* status_dev, void* stream);

/* ---- Dynamic regridding of octree meshes (Sec. 5, adaptive mesh refinement) ----
 * A regrid step: dg_mhd_amr_marks -> copy the marks to the host ->
 * dg_mhd_regrid_plan (new leaves and their sources) -> dg_mhd_init on the new
 * leaves -> copy the sources to the device -> dg_mhd_remap from the old
 * context's state into the new context's state -> destroy the old context.
 *
 * Smoothness indicator (Sec. 5): s_max[c] = max over the monitored conserved
 * components u (bit v of field_mask, v < 8, 9 with GLM psi; in the Powell form
 * the B components are those of the LDF rows) and the directions a of
 * S_a(u) = sum_{k=1..d} 2^(2k-1) int_[-1,1]^dim (d^k u / dxi_a^k)^2, in FP64.
 * w, wmean: the state (layout of dg_mhd_rhs; wmean nullable); s_max: DEVICE
 * FP64 array of n_cells. Any mesh. DG_E_ARG for an empty or out-of-range mask. */
int dg_mhd_smoothness(dg_mhd_ctx* ctx, const void* w, const double* wmean, int field_mask, double* s_max,
                      void* stream);

/* Refinement marks of an octree context (Sec. 5): marks[c] (DEVICE int8,
 * n_cells) = +1 if s_max[c] > 2 s_tilde and level < max_level; -1 for every
 * member of a group of 2^dim sibling leaves whose restriction (the L2
 * projection of the group onto the parent's basis) has S_a(u) < s_tilde / 2
 * for every monitored u and direction, whose parent level is >= min_level and
 * none of whose members is marked +1; 0 otherwise. s_max: caller-owned DEVICE
 * FP64 scratch of n_cells (receives the smoothness indicator). Uniform
 * contexts: DG_E_UNSUPPORTED. */
int dg_mhd_amr_marks(dg_mhd_ctx* ctx, const void* w, const double* wmean, int field_mask, double s_tilde,
                     int min_level, int max_level, int8_t* marks, double* s_max, void* stream);

/* New leaf list from the marks (HOST arrays; synchronous, host only):
 * refinement of the leaves marked +1 (up to level 17), 2:1 balance across
 * faces by refining every leaf two levels coarser than a face neighbour until
 * none is, then coarsening of the sibling groups with all members marked -1
 * where the parent keeps the balance, to a fixed point. Writes *n_new and, if
 * new_level, new_ijk and src are non-NULL and cap >= *n_new, the new leaves
 * in Morton order (level, ijk[n_new*dim]) and per new leaf its source
 * src[2i] = kind | octant << 4 (kind 0 copy, 1 prolongation from the old leaf
 * src[2i+1] into child `octant`, 2 restriction of old sibling group src[2i+1])
 * -- the array dg_mhd_remap takes. DG_E_ARG if cap is too small (*n_new is
 * still set: call with NULL arrays to query the size). */
int dg_mhd_regrid_plan(const dg_mhd_ctx* ctx, const int8_t* marks, int64_t cap, int8_t* new_level,
                       int32_t* new_ijk, int32_t* src, int64_t* n_new);

/* The same planning without a context (HOST arrays; synchronous, no device
 * work): the leaves (dim, n, level[n], ijk[n*dim], any order) must tile the
 * periodic unit cube without overlap, be 2:1 balanced across faces and have
 * levels <= 17 (DG_E_MESH otherwise; DG_E_ARG for dim not 2 or 3, n < 1 or a
 * mark outside {-1, 0, 1}). marks[c] in the given leaf order; the output and
 * its size query are those of dg_mhd_regrid_plan, the groups numbered as
 * dg_mhd_sibling_groups numbers them (the numbering a context built on the
 * same leaves uses). */
int dg_mhd_regrid_plan_mesh(int dim, int64_t n, const int8_t* level, const int32_t* ijk, const int8_t* marks,
                            int64_t cap, int8_t* new_level, int32_t* new_ijk, int32_t* src, int64_t* n_new);

/* The groups of 2^dim sibling leaves of a mesh (HOST arrays, no context; the
 * mesh rules of dg_mhd_regrid_plan_mesh): the children of one cube, all of
 * them leaves, sorted by (parent level, parent i, j, k); groups[g*2^dim + o]
 * = index of the leaf in octant o (o = sum_a bit_a << a, bit_a the lowest bit
 * of its coordinate a). Writes *n_groups and, if groups is non-NULL and
 * cap >= *n_groups, the groups (DG_E_ARG if cap is too small). These are the
 * groups the restriction sources of a plan and the -1 marks refer to. */
int dg_mhd_sibling_groups(int dim, int64_t n, const int8_t* level, const int32_t* ijk, int64_t cap,
                          int32_t* groups, int64_t* n_groups);

/* The faces a context builds for an octree mesh (HOST arrays, no context; Sec.
 * 3.5 surface integrals, coarse-fine faces as in dg_mesh_desc): the mesh rules
 * of dg_mesh_desc (DG_E_MESH otherwise; DG_E_ARG for dim not 2 or 3). Cells in
 * the given order, per cell its axes in order, the lower side first; a
 * same-level face is listed once by its right (upper) cell, a coarse-fine face
 * by its fine cell. Face f: face_left[f] / face_right[f] = the cells below /
 * above it along the axis (periodic wrap), face_meta[f] = axis | kind << 2 |
 * sub << 4, kind 0 same level, 1 coarse cell on the left, 2 on the right, sub
 * = the fine cell's coordinate parities across the face (bit j for the j-th
 * other axis in increasing order). Writes *n_faces and, if the three arrays
 * are non-NULL and cap >= *n_faces, the faces (DG_E_ARG if cap is too small).
 * partial = 1: the leaves of a partition's local mesh (owned and ghost cells,
 * see dg_mesh_desc.partial): they need not cover the cube; a face with no leaf
 * across it is left out. */
int dg_mhd_octree_faces(int dim, int64_t n, const int8_t* level, const int32_t* ijk, int partial, int64_t cap,
                        int32_t* face_left, int32_t* face_right, int32_t* face_meta, int64_t* n_faces);

/* The tables a context's regridding calls use (HOST, no context, no device
 * work), concatenated in out (doubles) with the six sizes in sizes[6]; n =
 * Legendre modes, nd = LDF rows (0 for GLM), no = 2^dim:
 *   QL [dim a][n][n]       smoothness form of a Legendre field along a:
 *                          S_a = w^T QL[a] w (Sec. 5, sum_k 2^(2k-1) int (d_a^k u)^2
 *                          over the reference cell, by the (d+1)-point rule);
 *   QB [dim c][dim a][nd][nd]  the same for component c of the LDF field;
 *   PL [no][n][n], PB [no][nd][nd]  L2 prolongation: child row from parent rows;
 *   RL [no][n][n], RB [no][nd][nd]  L2 restriction: parent row from child o's rows.
 * DG_E_ARG for dim not 2 or 3, degree outside 0..3, an unknown scheme, or cap
 * below the total (call with out NULL to get the sizes). */
int dg_mhd_regrid_tables(int dim, int degree, int divB_scheme, int64_t cap, double* out, int64_t* sizes);

/* State of the new context from the old one (asynchronous on stream): per new
 * leaf a copy, an L2 prolongation (parent octant onto the child's basis; the
 * LDF rows under the vector inner product of eq. innerp) or an L2 restriction
 * (the 2^dim children onto the parent's basis). src: DEVICE copy of the plan's
 * src array; w_old/wmean_old and w_new/wmean_new: the two contexts' state
 * buffers (wmean both NULL or both non-NULL; FP32 form: the means are
 * remapped in FP64 and mirrored into the float rows). Both contexts must have
 * the same dimension, degree, scheme and precision, the old one an octree.
 * Source entries out of range are skipped and latch DG_E_ARG in the new
 * context's status word. */
int dg_mhd_remap(const dg_mhd_ctx* old_ctx, dg_mhd_ctx* new_ctx, const int32_t* src, const void* w_old,
                 const double* wmean_old, void* w_new, double* wmean_new, void* stream);

/* Releases every device allocation of ctx. ctx may be NULL. */
void dg_mhd_destroy(dg_mhd_ctx* ctx);

/* Static string for a dg_status value. */
const char* dg_mhd_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* DG_MHD_H */
