/*
 * deer.h - C ABI of the GB300 (sm_103a) parallel-Newton library.
 *
 * The library evaluates a nonlinear recurrence s_t = f_t(s_{t-1}), t = 1..T, from a
 * fixed s_0 (Sec. 2.1 of the paper; inputs x_t are curried into f_t) by the parallel
 * Newton iteration of Algorithm alg:deer: every iteration linearises f at the current
 * guess for all t at once, solves the resulting linear recurrence with a parallel
 * associative scan (Eq. deer_lds, bin_op_affine) and tests the residual
 * r_t = s_t - f_t(s_{t-1}) (Eq. r_def).
 *
 * Conventions for every entry point:
 *   - Tensor pointers are DEVICE memory owned by the caller, row-major and contiguous,
 *     unless an argument says "host". The library never allocates device memory; it
 *     uses the caller's workspace (size from the *_workspace_bytes queries).
 *   - Floating-point buffers (params, s0, x, s, gradients) are float64 when
 *     prec = DEER_FP64 or DEER_MIXED_BF16 and float32 when prec = DEER_FP32.
 *   - A trajectory batch is packed: sequence b owns rows offsets[b] .. offsets[b+1]-1 of
 *     s [N][d] and x [N][d_in] (N = offsets[B]); row offsets[b] + t - 1 holds s_t.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream). The
 *     solver reads one small status word back per iteration and returns after the
 *     stream has drained; results are then valid.
 *   - Errors are returned as a deer_status; nothing aborts or traps. A solve that
 *     reaches its iteration cap returns DEER_NOT_CONVERGED with the last iterate in s.
 *   - Calls are reentrant given distinct workspaces; two calls that share a workspace
 *     must not overlap on the GPU.
 */
#ifndef DEER_H_
#define DEER_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* deer_stream_t; /* identical to cudaStream_t */

typedef enum {
  DEER_OK = 0,
  DEER_NOT_CONVERGED = 1,     /* iteration cap reached; the last iterate is in s_out */
  DEER_ERR_INVALID = -1,      /* bad pointer, size, enum value or combination */
  DEER_ERR_CUDA = -2,         /* a CUDA call failed (see deer_last_cuda_error) */
  DEER_ERR_NONFINITE = -3,    /* a residual became NaN/Inf (reset heuristic off) */
  DEER_ERR_WORKSPACE = -4,    /* workspace missing, too small or misaligned (256 B) */
  DEER_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
  DEER_ERR_UNSUPPORTED = -6   /* combination not built (e.g. dense ELK, d too large) */
} deer_status;

/* Built-in recurrences f (the registry; f runs in hand-written CUDA). */
typedef enum {
  /* Brusselator kinetics dx = a-(b+1)x+x^2y, dy = bx-x^2y, explicit Euler, d = 2.
     params per sequence: [a, b]. */
  DEER_F_BRUSSELATOR_EULER = 0,
  /* Mass-action reaction network, explicit Euler / classical RK4. params per sequence:
     rate constants k[R]; topology per sequence: int32 [R][4] = (i1, i2, p1, p2) with -1
     for an absent slot; reaction r has rate k_r c_i1 c_i2 (c_i2 -> 1 if i2 < 0),
     consumes i1, i2 and produces p1, p2. Species indices must lie in [0, d). */
  DEER_F_MASSACTION_EULER = 1,
  DEER_F_MASSACTION_RK4 = 2,
  /* GRU cell, zero biases: z = sig(Wz x + Uz h), r = sig(Wr x + Ur h),
     h~ = tanh(Wh x + Uh (r*h)), h' = (1-z) h + z h~. params (shared, stride 0):
     [Wz, Wr, Wh] each [d][d_in], then [Uz, Ur, Uh] each [d][d]. */
  DEER_F_GRU = 3,
  /* Affine recurrence s_t = A s_{t-1} + x_t (x may be NULL). params (shared): A [d][d]. */
  DEER_F_LINEAR = 4,
  /* Mean-field RNN of the predictability threshold experiment (Sec. ssc:exp_thresh):
     s_t = W tanh(s_{t-1}) + u_t with u_t the row of x (input size d; x may be NULL for
     u = 0). params: W [d][d], per sequence (params_stride >= d*d) or shared. The thesis
     draws W_ij ~ N(0, g^2/d) with W_ii = 0; any W is accepted. d in {1,2,4,8,16,32}. */
  DEER_F_RNN_TANH = 5,
  /* Discretised Langevin dynamics (Eq. langevin) in a two-component Gaussian-mixture
     potential phi(s) = -log(w1 N(s; m1, diag v1) + w2 N(s; m2, diag v2)):
     s_t = s_{t-1} - dt grad phi(s_{t-1}) + sqrt(2 dt) w_t, with w_t the row of x (input
     size d; standard normal draws; x may be NULL for the noise-free drift). Its Jacobian is
     I - dt Hess phi. params per sequence (params_stride >= 4d+2) or shared:
     [m1 (d) | m2 (d) | v1 (d) | v2 (d) | w1 | w2] with v > 0, w >= 0, w1 + w2 > 0.
     d in {1,2,4,8,16,32}. */
  DEER_F_LANGEVIN_2WELL = 6,
  /* Lorenz-96 dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F (indices modulo d), one fixed
     step dt of the fifth-order solution of the Dormand-Prince 5(4) pair (no step-size
     control: f_t must be one fixed map). params: [F], per sequence (params_stride >= 1) or
     shared. d in {4, 5, 8}. */
  DEER_F_LORENZ96_DP5 = 7,
  /* Input-selected permutation, the group word problem as a linear recurrence
     (Prop. cayley): s_t[i] = s_{t-1}[x_t[i]] with x_t the row of x holding d source
     indices stored as exact integers in [0, d) (input size d; x required). A_t is the
     corresponding permutation (selection) matrix. An index that is not an integer in
     [0, d) makes that entry NaN, which the solver reports as DEER_ERR_NONFINITE.
     params: unused (any non-NULL pointer). d in {2,4,5,8,16,32}. */
  DEER_F_PERMUTE = 8
} deer_fkind;

/* Transition matrix A~_t of the linear recurrence solved per iteration
   (Table fxd_pt_sum of the paper). */
typedef enum {
  DEER_JAC_FULL = 0,     /* Newton / DEER: df_t/ds_{t-1}, dense d x d (d <= 32) */
  DEER_JAC_DIAG = 1,     /* quasi-Newton / quasi-DEER: its diagonal (Eq. quasi_lds) */
  DEER_JAC_IDENTITY = 2, /* Picard: I */
  DEER_JAC_ZERO = 3      /* Jacobi: 0 */
} deer_jac;

typedef enum {
  DEER_DAMP_NONE = 0,
  DEER_DAMP_ELK = 1,   /* Kalman-filter step, lambda = damp_param (Sec. 4.3): diagonal modes
                          (quasi-ELK) and the full Jacobian for d <= 8 (dense ELK) */
  DEER_DAMP_SCALE = 2, /* scale-ELK: A~ <- (1 - k) A~, k = damp_param in [0, 1] (Sec. 4.5.1) */
  DEER_DAMP_CLIP = 3   /* clip-ELK: diag A~ clipped to [-rho, rho], rho = damp_param (Sec. 4.5.2) */
} deer_damp;

/* Initial guess s^(0) of the iteration (Sec. 3.3.3: zeros, a copy of s_0, one Jacobi step
   or iid standard normal draws; any guess converges, Prop. global_convergence). */
typedef enum {
  DEER_INIT_ZEROS = 0,  /* s^(0)_t = 0 */
  DEER_INIT_S0 = 1,     /* s^(0)_t = s_0 */
  DEER_INIT_JACOBI = 2, /* s^(0)_t = f_t(0): one Jacobi step from zero */
  DEER_INIT_USER = 3,   /* s_out holds the guess on entry (warm start) */
  DEER_INIT_RANDN = 4   /* iid N(0, 1) entries from a counter-based generator: entry e of the
                           packed s array (e = row * d + i) is
                           sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller, evaluated in float64), with
                           u1 = ((z(2e+1) >> 11) + 1) 2^-53 and u2 = (z(2e+2) >> 11) 2^-53,
                           where z(n) is the n-th output (n >= 1) of SplitMix64 started at
                           deer_options.seed: z(n) = mix(seed + n * 0x9E3779B97F4A7C15),
                           mix(z) = z ^ (z >> 31) after z ^= z >> 30, z *= 0xBF58476D1CE4E5B9,
                           z ^= z >> 27, z *= 0x94D049BB133111EB (all modulo 2^64). The same
                           seed and packing give the same guess on every call. */
} deer_init;

typedef enum {
  DEER_FP64 = 0,       /* everything float64 */
  DEER_FP32 = 1,       /* everything float32; per-sequence residual max/merit reported in
                          float64 */
  DEER_MIXED_BF16 = 2  /* float64 state, dynamics value and residual; the Jacobian is formed
                          in float32 and stored as bf16 E = A - I, and the dense scan composes
                          (I + E) with float32 accumulation in correction form. While a
                          sequence's scaled residual is above 1e-4 (and in the first
                          iteration) its dynamics value is evaluated in float32, whose
                          rounding is far below that residual; such an iterate reports at
                          least 1e-6 and cannot pass the test, so convergence is always
                          decided on a float64 residual. State entries beyond 1e18 count as
                          overflow for the reset heuristic. Mass-action kinetics with d = 16
                          or 32 and DEER_JAC_FULL (no damping or scale-ELK); not available
                          in deer_grad or deer_solve_noalloc. */
} deer_prec;

typedef struct {
  int32_t kind;            /* deer_fkind */
  int32_t d;               /* state size */
  int32_t d_in;            /* input size (GRU; LINEAR uses d); 0 when f takes no input */
  int32_t n_reactions;     /* R (mass-action only) */
  double dt;               /* integrator step (Brusselator, mass-action) */
  const void* params;      /* device; layout per kind above */
  int64_t params_stride;   /* elements between consecutive sequences' params; 0 = shared */
  const int32_t* topology; /* device; mass-action only */
  int64_t topology_stride; /* int32 elements between sequences' topologies; 0 = shared */
} deer_dynamics;

typedef struct {
  int32_t max_iters;  /* iteration cap; <= 0 means the longest T (sufficient by
                         Prop. global_convergence) */
  double tol;         /* a sequence passes the test when its scaled residual
                         max_{t,i} |r_t,i| / max(1, |s_t,i|) <= tol (r_t = s_t - f_t(s_{t-1}),
                         Eq. r_def; the absolute residual wherever |s| <= 1), evaluated in
                         float64 on the iterate about to be updated; it converges after
                         `confirm` consecutive passing iterates */
  int32_t jac;        /* deer_jac */
  int32_t damp;       /* deer_damp */
  double damp_param;  /* lambda (ELK), k (scale) or rho (clip) */
  int32_t init;       /* deer_init */
  int32_t prec;       /* deer_prec */
  int32_t reset;      /* reset heuristic (Sec. 3.2): entries that are non-finite or exceed
                         1e30 (float64) / 1e18 (float32) after a scan are set to 0 */
  int32_t chunk;      /* scan chunk length; 0 = automatic. Power of two in [8, 1024]. */
  int32_t confirm;    /* a sequence converges when `confirm` consecutive iterates pass the
                         test (<= 1 means one). With 2 the returned iterate has had one more
                         Newton step after first passing, which removes the smooth part of
                         the remaining error when the test sits near float32 roundoff. */
  int32_t window;     /* sliding window (Sec. 3.2; parallel Newton converges from the front,
                         so a converged prefix can be left alone): 0 = every iteration
                         covers each sequence whole; 1 = after each test, the whole chunks
                         before a sequence's first row whose scaled residual exceeds tol
                         (in any of the last `confirm` + 1 iterates) are frozen and later
                         iterations solve only from there, starting from the frozen
                         state. The fixed point is the same; iterates differ from the
                         unwindowed iteration once rows are frozen. Applies to undamped
                         steps (damp = DEER_DAMP_NONE); damped steps converge linearly and
                         always cover each sequence whole. */
  uint64_t seed;      /* generator seed of DEER_INIT_RANDN (ignored otherwise) */
  double* history;    /* optional DEVICE buffer [history_len][4] (NULL = none): the
                         convergence test of iteration i (i = 0 tests the initial guess)
                         writes row i = (i, sum over the sequences it tested of their merit
                         1/2 ||r||^2, the largest scaled residual among them, the number of
                         sequences still active after it). Rows of tests that did not run
                         are left untouched; tests past history_len are not recorded. */
  int32_t history_len;
  int32_t compensate;  /* DEER_FP32 with mass-action kinetics and the full Jacobian (d = 4, 8,
                          16, 32): 1 keeps, for every state entry, a float32 compensation
                          term in the workspace (the state is the unevaluated sum s + lo,
                          |lo| <= ulp(s)/2), forms the residual from the pair in increment
                          form ((s_t - s_{t-1}) - inc_t + (lo_t - lo_{t-1}), inc_t = f(s_{t-1})
                          - s_{t-1} from the integrator) and adds each Newton correction to
                          the pair with error-free transformations. Near equilibrium the
                          per-step increments of these trajectories fall below half a float32
                          ulp of the state, where a plain float32 state loses them and the
                          loss adds up along the conserved directions (errors of 1e-4 at
                          T = 16384); with the pair the returned s is the float32 rounding of
                          a trajectory accurate to the float32 rounding of the increments.
                          Costs 8 more bytes per state entry per iteration. 0 = plain float32
                          state. Ignored for other kinds, modes and precisions. Default 1. */
  int64_t jac_bytes_max; /* the most bytes the stored step Jacobians may take (0 = no
                          bound). deer_grad / deer_grad_ex: below B T d^2 values the reverse
                          recursion runs over time windows of
                          W = jac_bytes_max / (B d^2 sizeof(real)) rows from the end of the
                          sequences: each window's Jacobians are formed when it is reached
                          (each one once), its rows of the trajectory, cotangents and inputs
                          are gathered into the workspace, and the adjoint entering it from
                          the later window joins the cotangent of its last row; the gradient
                          is the same up to rounding. deer_solve / deer_solve_batched with
                          DEER_MIXED_BF16 and d = 16: when the bf16 Jacobians of all rows
                          (N d^2 2 bytes) exceed it, none is stored: each chunk's aggregate is
                          formed while the chunk is linearised, and the scan's final pass
                          linearises it again (the same arithmetic from the same iterate)
                          to apply the correction. Never leaving the chip, the Jacobians are
                          then kept in float32 and composed to float32 accuracy (tf32 tensor-
                          core products with a three-term split) instead of bf16, which keeps
                          Newton's rate of convergence over long horizons; state, residual
                          and test stay float64. The workspace queries shrink accordingly. */
  int32_t device_loop; /* 1 = run the Newton loop of Algorithm 1 on the device: after the
                          first iteration, the iterations are one CUDA graph, a gate node
                          and a conditional while node whose body is one iteration (scan,
                          linearisation, convergence check; the check sets the condition
                          for the next), launched once per call with no host
                          synchronisation between iterations. Every kernel then reads the
                          active-set sizes the last check wrote to device memory, and the
                          grids are sized for the whole problem (blocks past the active set
                          exit at once). Results are identical to the host loop's. Ignored
                          (host loop) while per-phase profiling is on. The call still blocks
                          until the loop ends. Default 0. */
  int32_t no_block_solve; /* 0 (default): where every sequence is short enough for one
                          thread-block cluster (up to 8 blocks) to hold its iterate in
                          registers (d = 1 or 2: up to 8192 steps; d = 4: up to 2048) and
                          the step is the full Jacobian without damping or with scale
                          damping (no mixed precision, no compensated state, no history
                          record), the whole Newton loop runs in one kernel, one cluster per
                          sequence: linearisation, convergence test and a cluster-wide scan
                          per iteration through distributed shared memory, no launch or host
                          synchronisation between iterations, every cluster stopping on its
                          own convergence (for the Brusselator, Euler, mass-action, linear,
                          mean-field RNN and Langevin kinds). The sliding window is moot
                          there (each cluster iterates its whole sequence). 1 = always the
                          multi-kernel loop. */
} deer_options;

typedef struct {
  int32_t iters;      /* linear-recurrence solves applied to this sequence */
  int32_t converged;  /* 1 if the convergence test of deer_options.tol passed on
                         `confirm` consecutive iterates */
  double merit;       /* 1/2 ||r||^2 (unscaled residual, Eq. merit) of the last iterate
                         tested (the returned one, unless the iteration cap stopped the
                         solve after its last scan) */
  double max_resid;   /* scaled residual max_{t,i} |r_t,i| / max(1, |s_t,i|) of that
                         iterate (the quantity compared with tol) */
} deer_info;

/* Fills `opt` with defaults: cap T, tol 1e-10, FULL, no damping, INIT_S0, FP64, auto chunk,
   confirm 1, no window, seed 0, no history, compensated float32 state. */
void deer_default_options(deer_options* opt);

/* Workspace bytes needed by deer_solve / deer_solve_batched for `batch` sequences
   holding `total_steps` rows in all. Returns 0 for an invalid configuration. */
size_t deer_workspace_bytes(const deer_dynamics* f, int64_t batch, int64_t total_steps,
                            const deer_options* opt);

/* Solve `batch` sequences of equal length T. s0 [batch][d]; x [batch*T][d_in] or NULL;
   s_out [batch*T][d] (holds the guess on entry when init = DEER_INIT_USER).
   info: host array [batch] or NULL. */
deer_status deer_solve(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                       const void* x, void* s_out, const deer_options* opt, void* workspace,
                       size_t workspace_bytes, deer_stream_t stream, deer_info* info);

/* Ragged batch: offsets is a HOST array [batch+1] (offsets[0] = 0, non-decreasing; empty
   sequences allowed). Sequences converge independently: a converged sequence is masked
   out of later iterations. Other arguments as deer_solve. */
deer_status deer_solve_batched(const deer_dynamics* f, int64_t batch, const int64_t* offsets,
                               const void* s0, const void* x, void* s_out,
                               const deer_options* opt, void* workspace, size_t workspace_bytes,
                               deer_stream_t stream, deer_info* info);

/* Workspace bytes for deer_grad. */
size_t deer_grad_workspace_bytes(const deer_dynamics* f, int64_t batch, int64_t T,
                                 const deer_options* opt);

/* Gradient of a loss l(s_1..s_T) at the converged trajectory s_star [batch*T][d] by the
   adjoint (Eq. bptt / unrolled_bwds): a reverse linear recurrence
   lambda_T = g_T, lambda_{t-1} = g_{t-1} + A_t^T lambda_t solved with a reverse parallel
   scan, then dl/dtheta = sum_t lambda_t^T df_t/dtheta(s_{t-1}) and dl/ds0 = A_1^T lambda_1.
   dl_ds [batch*T][d] holds g_t = dl/ds_t. dl_dparams [batch][params per sequence] (mass-
   action: d/dk; Brusselator: d/d(a,b); not available for shared-parameter kinds);
   dl_ds0 [batch][d] or NULL. Uses opt->prec (FP64 or FP32) and opt->chunk. */
deer_status deer_grad(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                      const void* x, const void* s_star, const void* dl_ds, void* dl_dparams,
                      void* dl_ds0, const deer_options* opt, void* workspace,
                      size_t workspace_bytes, deer_stream_t stream);

/* deer_grad plus the gradient with respect to the inputs curried into f_t (Sec. 2.1):
   dl_dx [batch*T][d_in] (the layout of x) receives lambda_t^T df_t/dx_t evaluated at
   s_{t-1}, or NULL. Available for the kinds with differentiable inputs: the GRU (through
   its three gates), the affine recurrence and the mean-field RNN (additive inputs), and
   the Langevin kind (noise draws, scaled by sqrt(2 dt)); DEER_ERR_UNSUPPORTED for the
   others or when x is NULL. Same workspace as deer_grad. */
deer_status deer_grad_ex(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                         const void* x, const void* s_star, const void* dl_ds,
                         void* dl_dparams, void* dl_ds0, void* dl_dx,
                         const deer_options* opt, void* workspace, size_t workspace_bytes,
                         deer_stream_t stream);

/* Largest Lyapunov exponent along trajectories (Ch. 5, Algorithm alg:LLE_estimate): for
   each of `batch` sequences of T steps, the unit vector u_0 = u0[b] is pushed through the
   step Jacobians J_t = df_t/ds evaluated at s_{t-1} (s_0 for t = 1) and renormalised
   every step, u_t = J_t u_{t-1} / ||J_t u_{t-1}||, and lle_out[b] = (1/T) sum_t
   log ||J_t u_{t-1}||. A positive value predicts slow parallel-Newton convergence over
   long horizons (Ch. 5). s: DEVICE trajectory [batch*T][d] (a rollout or a converged
   solve); u0: DEVICE [batch][d], unit vectors; lle_out: DEVICE float64 [batch]; buffers in
   float64 for DEER_FP64, float32 for DEER_FP32 (lle_out always float64); d <= 32. The
   Jacobians are materialised in the workspace (size from deer_lle_workspace_bytes). */
size_t deer_lle_workspace_bytes(const deer_dynamics* f, int64_t batch, int64_t T,
                                int32_t prec);
deer_status deer_lle(const deer_dynamics* f, int64_t batch, int64_t T, const void* s0,
                     const void* x, const void* s, const void* u0, double* lle_out,
                     int32_t prec, void* workspace, size_t workspace_bytes,
                     deer_stream_t stream);

/* Sequential rollout s_t = f_t(s_{t-1}) on the GPU (the comparison baseline: one
   trajectory per thread or thread group, no parallelism over t). offsets: DEVICE array
   [batch+1] for a ragged batch, or NULL for `batch` sequences of length T. Needs no
   workspace. */
deer_status deer_rollout(const deer_dynamics* f, int64_t batch, int64_t T,
                         const int64_t* offsets, const void* s0, const void* x, void* s_out,
                         int32_t prec, deer_stream_t stream);

/* deer_solve for callers that cannot allocate device memory when they solve: code that
   runs while the allocator must not be touched (a cudaMalloc synchronises the device),
   loops with a hard latency budget, embedders with a fixed memory pool. There is no
   counterpart in the paper; this is a packaging of deer_solve. It takes no workspace: the
   library keeps one fixed scratch area of deer_noalloc_scratch_bytes() (32 MiB) per device
   in a __device__ array, present on every GPU that loads the library until the process
   exits. Problems whose workspace (deer_workspace_bytes plus one deer_info per sequence)
   does not fit are rejected with DEER_ERR_WORKSPACE (deer_last_cuda_error says how many
   bytes they needed). Every call looks up the array's address on the current device
   (cudaGetSymbolAddress, which allocates nothing), so a context that was reset and
   recreated since an earlier call is handled. Like deer_solve's host-driven loop, it reads a
   status word back and synchronises its stream once per Newton iteration (`device_loop` is
   ignored), so it cannot be called while the stream is being captured into a CUDA graph. Every call reuses the same array and clears
   what must start at zero, so calls that overlap on the GPU (other streams or threads)
   race and must be serialised by the caller. Arguments and results as deer_solve (without
   mixed precision, dense ELK or the sliding window, which return DEER_ERR_UNSUPPORTED, and
   always with a plain float32 state: `compensate` is ignored); nothing is allocated on the
   device or the host. */
deer_status deer_solve_noalloc(const deer_dynamics* f, int64_t batch, int64_t T,
                               const void* s0, const void* x, void* s_out,
                               const deer_options* opt, deer_stream_t stream,
                               deer_info* info);
size_t deer_noalloc_scratch_bytes(void);

/* Tensor-core kernels (on by default): where a step of the path has a tensor-core kernel
   and a SIMT one with the same results up to rounding, the tensor-core one runs when this
   is on: the GRU d = 64 float32 linearisation (tcgen05, three products per step split to
   float32 accuracy) and the d = 32 float32 dense chunk products (warp-level tf32 MMAs split
   to float32 accuracy). 0 = SIMT kernels; 1 = the default tensor-core kernels (the d = 16
   mixed-precision chunk products as warp-level bf16 MMAs, one chunk per warp); 2 = as 1,
   but the d = 16 mixed-precision chunk products run as tcgen05 MMAs with the accumulator
   in tensor memory, 8 chunks per CTA stacked block-diagonally (1/8 of the issued
   multiply-adds useful: the measured alternative). Process-wide, thread-safe; affects
   calls made after it returns. */
void deer_set_tensor_cores(int32_t on);
int32_t deer_get_tensor_cores(void);

/* Peak arithmetic rate of the current GPU, measured (the denominators of the rooflines of
   the ALU- and tensor-bound kernels; there is no counterpart in the paper): what = 0 FP32
   FMA (the faster of scalar and packed two-wide FMA chains), 1 FP64 FMA, 2 dense tcgen05
   MMAs of kind::tf32, 3 dense tcgen05 MMAs of kind::f16 with bf16 operands (M = 128,
   N = 256, float32 accumulation in tensor memory). Every SM works (the SM count is read
   from the device); the work is counted exactly (2 flop per multiply-add) and timed with
   CUDA events on `stream`, best of five launches after two warm-ups. *flops_per_s
   receives flop/s. Synchronises the stream; allocates nothing (the tensor-memory columns
   of the MMA kernel are released before it returns). DEER_ERR_TIMEOUT if the MMA
   kernel's bounded wait gave up, DEER_ERR_INVALID for another `what`. */
deer_status deer_measure_peak(int32_t what, deer_stream_t stream, double* flops_per_s);

/* Number of kernels this library enqueued since load (all entry points, all threads). */
int64_t deer_kernel_launch_count(void);

/* Self-test of the bounded device waits (the failure path behind DEER_ERR_TIMEOUT): runs
   the single-pass look-back scan over one sequence of two tiles whose first tile is never
   scanned, so the second tile's wait for its predecessor's flag runs out at the spin limit
   (a fraction of a second); the kernel then records the timeout and finishes, leaving the
   context usable. Allocates and frees about 100 KB of device memory; synchronises the
   stream. Returns DEER_ERR_TIMEOUT when the wait gave up as designed (the expected
   result), DEER_OK if it did not, DEER_ERR_CUDA on a CUDA error. */
deer_status deer_selftest_wait_timeout(deer_stream_t stream);

/* Per-phase device time of deer_solve / deer_solve_batched, measured with CUDA events on
   the solver's stream while profiling is enabled (off by default; costs one extra stream
   synchronisation per iteration). Phase p: 0 set-up, 1 linearise + residual, 2
   convergence check, 3 scan. rows[p] counts the trajectory rows the phase processed
   (rows of converged sequences are skipped). Process-wide, thread-safe. */
typedef struct {
  int64_t launches[4];
  double ms[4];
  int64_t rows[4];
} deer_profile;
void deer_profile_enable(int32_t on);
void deer_profile_reset(void);
void deer_profile_read(deer_profile* out);

const char* deer_status_string(int32_t status);
const char* deer_last_cuda_error(void);
int32_t deer_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DEER_H_ */
